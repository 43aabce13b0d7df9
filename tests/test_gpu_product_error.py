"""GPU eps_2 (Sec. 7: relative spectral error by power iteration) of computed
products, through h2_product_error, against the oracle's power iteration on the
same operator (the GPU result's dense expansion with the oracle's X, Y, Z0)
from the same start vector; and at the full n = 32768 sphere workload."""
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


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED])
def test_eps2_against_oracle(precision):
    n, leaf, eta, order, eps = 1024, 32, 2.0, 3, 1e-5
    pts = synth.sphere(n, 21)
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, leaf, eta, order)
    Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, leaf, eta, order)
    Z0 = P.h2_build_interp(pts, P.H2_K_LAPLACE, leaf, eta, order)
    Zr = P.h2_clone(Z0)
    P.h2_mul_add(Zr, X, Y, eps, precision)
    x0 = synth.normal01(99, n)
    e, nrm = P.h2_product_error(Zr, Z0, X, Y, x0=x0, steps=20)
    st = O.build_structure(pts, leaf, eta, order)
    DX = O.build_interp(st, O.K_LAPLACE).to_dense()
    DY = O.build_interp(st, O.K_YUKAWA).to_dense()
    eo, no = O.spectral_error(P.h2_to_dense(Zr), DX, DX, DY, x0, 20)
    assert abs(nrm - no) <= 1e-10 * no
    assert abs(e - eo) <= 1e-6 * eo
    assert 0.0 < e <= 2 * eps


def test_eps2_of_exact_product():
    """Exact mode (eps = 0, Sec. 3) reproduces Z0 + X Y to rounding: eps_2 at
    rounding level."""
    n = 512
    pts = synth.sphere(n, 4)
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 16, 2.0, 2)
    Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, 16, 2.0, 2)
    Zr = P.h2_clone(X)
    P.h2_mul_add(Zr, X, Y, 0.0, P.H2_FP64)
    e, nrm = P.h2_product_error(Zr, X, X, Y, steps=20)
    assert nrm > 0.0 and e <= 1e-12


def test_eps2_full_size_sphere():
    """n = 32768 sphere workload (leaf 64, eta 2, order 4, eps 1e-6, X = Y = Z):
    eps_2 of the FP64 and mixed products, 20 steps (Sec. 7)."""
    n, eps = 32768, 1e-6
    pts = synth.sphere(n, 2309090611)
    G = P.h2_build_interp(pts, P.H2_K_LAPLACE, 64, 2.0, 4)
    errs = {}
    for prec in (P.H2_FP64, P.H2_MIXED):
        Zr = P.h2_clone(G)
        P.h2_mul_add(Zr, G, G, eps, prec)
        errs[prec], nrm = P.h2_product_error(Zr, G, G, G, steps=20)
        assert nrm > 0.0
        Zr.free()
    # FP64: within the truncation tolerance; mixed: FP32 products add a few 1e-7
    assert 0.0 < errs[P.H2_FP64] <= eps
    assert 0.0 < errs[P.H2_MIXED] <= 10 * eps


def test_eps2_argument_errors():
    pts = synth.sphere(256, 1)
    A = P.h2_build_interp(pts, 0, 16, 2.0, 2)
    B = P.h2_build_interp(synth.sphere(256, 2), 0, 16, 2.0, 2)
    with pytest.raises(P.H2Error) as e:
        P.h2_product_error(A, A, A, B)
    assert e.value.code == -2
    with pytest.raises(P.H2Error) as e:
        P.h2_product_error(A, A, A, A, steps=0)
    assert e.value.code == -1
