"""GPU matrix-vector product against the oracle's and against dense."""
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


@pytest.mark.parametrize("trans", [False, True])
def test_matvec_against_oracle(trans):
    import torch
    n = 1000  # ragged leaves
    pts = synth.sphere(n, 3)
    X = P.h2_build_interp(pts, P.H2_K_YUKAWA, 20, 2.0, 3)
    Xo = O.build_interp(O.build_structure(pts, 20, 2.0, 3), O.K_YUKAWA)
    x = synth.normal01(9, n * 5).reshape(n, 5)
    xd = torch.as_tensor(np.ascontiguousarray(x.T), device="cuda")   # (5, n) row-major = n x 5 column-major
    yd = torch.empty_like(xd)
    P.h2_matvec(X, xd, yd, trans=trans)
    got = yd.cpu().numpy().T
    ref = Xo.matvec(x, trans)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_rows_of_product_against_dense():
    n = 1024
    pts = synth.sphere(n, 8)
    Z = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, 32, 2.0, 3)
    P.h2_mul_add(Z, Z, Y, 1e-6)
    rows = [0, 5, 511, 1023]
    got = P.h2_rows(Z, rows).cpu().numpy()
    D = P.h2_to_dense(Z)
    assert np.abs(got - D[rows]).max() <= 1e-13 * np.abs(D).max()
