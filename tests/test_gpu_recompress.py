"""GPU recompression of input H^2-matrices (orthogonalized bases, Fig. 1;
coarsening with the matrix's own block tree, Fig. 7) against the oracle's
recompression and the dense matrix; exact mode; a recompressed operand in a
product; sampled rows at the n = 32768 sphere size."""
import numpy as np
import pytest

import paper_2309_09061_gb300 as P
import synth
from oracle import h2_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    return P.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kernel", [P.H2_K_LAPLACE, P.H2_K_YUKAWA])
@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED])
def test_recompress_against_oracle(kernel, precision):
    eps = 1e-4
    pts = synth.sphere(900, 17)
    A = P.h2_build_interp(pts, kernel, 16, 2.0, 3)
    D = P.h2_to_dense(A)
    stats = P.h2_recompress(A, eps, precision)
    C = P.h2_to_dense(A)
    Co = O.recompress(O.build_interp(O.build_structure(pts, 16, 2.0, 3), kernel), eps).to_dense()
    assert rel(C, Co) <= 10 * eps
    assert rel(C, D) <= eps
    assert 0 < stats["max_rank_b"] < 27


def test_recompress_exact_mode():
    pts = synth.sphere(700, 2)
    A = P.h2_build_interp(pts, P.H2_K_YUKAWA, 16, 2.0, 3)
    D = P.h2_to_dense(A)
    P.h2_recompress(A, 0.0)
    assert rel(P.h2_to_dense(A), D) <= 1e-12


def test_recompress_double_layer():
    eps = 1e-5
    pts = synth.cube_surface(700, 5)
    nrm = synth.cube_surface_normals(pts)
    A = P.h2_build_interp(pts, P.H2_K_DLP, 16, 1.5, 3, normals=nrm)
    D = P.h2_to_dense(A)
    P.h2_recompress(A, eps)
    assert rel(P.h2_to_dense(A), D) <= eps


def test_recompressed_operand_in_product():
    pts = synth.sphere(900, 17)
    A = P.h2_build_interp(pts, P.H2_K_LAPLACE, 16, 2.0, 3)
    C = P.h2_clone(A)
    P.h2_recompress(C, 1e-8)
    DC = P.h2_to_dense(C)
    Z = P.h2_clone(A)
    P.h2_mul_add(Z, C, C, 1e-6)
    assert rel(P.h2_to_dense(Z), P.h2_to_dense(A) + DC @ DC) <= 2e-6


def test_recompress_full_size_sphere():
    """n = 32768 sphere, leaf 64, eta 2, order 4 (rank 64), eps 1e-6: sampled
    rows of the recompressed matrix against the Chebyshev matrix's rows, and
    lower ranks."""
    n, eps = 32768, 1e-6
    pts = synth.sphere(n, 2309090611)
    A = P.h2_build_interp(pts, P.H2_K_LAPLACE, 64, 2.0, 4)
    rows = np.unique(synth.splitmix64(79, 24) % n).astype(np.int64)
    ref = P.h2_rows(A, rows).cpu().numpy()
    stats = P.h2_recompress(A, eps)
    got = P.h2_rows(A, rows).cpu().numpy()
    assert rel(got, ref) <= 10 * eps
    assert stats["max_rank_b"] < 64


def test_recompress_arguments():
    with pytest.raises(P.H2Error) as e:
        P.h2_recompress(P.h2_build_interp(synth.sphere(256, 1), 0, 16, 2.0, 2), -1.0)
    assert e.value.code == -1
