"""GPU "+Z" with Z's own bases (V_Z and W_Z preserved in phase A beside V_X
and W_Y): Z from an earlier product (adaptive bases) and Z of another
Chebyshev order, against the oracle's general-Z product and the dense
Z + X Y, in every precision; exact mode."""
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


N, LEAF, ETA, ORDER = 900, 16, 2.0, 3


def operands():
    pts = synth.sphere(N, 31)
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, LEAF, ETA, ORDER)
    Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, LEAF, ETA, ORDER)
    return pts, X, Y


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED, P.H2_TC])
def test_other_order_z_against_oracle(precision):
    eps = 1e-5
    pts, X, Y = operands()
    Z = P.h2_build_interp(pts, P.H2_K_LAPLACE, LEAF, ETA, 2)
    DZ = P.h2_to_dense(Z)
    P.h2_mul_add(Z, X, Y, eps, precision)
    st3 = O.build_structure(pts, LEAF, ETA, ORDER)
    st2 = O.build_structure(pts, LEAF, ETA, 2)
    Xo, Yo, Zo = O.build_interp(st3, O.K_LAPLACE), O.build_interp(st3, O.K_YUKAWA), O.build_interp(st2, O.K_LAPLACE)
    Zg = P.h2_to_dense(Z)
    assert rel(Zg, O.mul_add(Zo, Xo, Yo, eps).result.to_dense()) <= 10 * eps
    assert rel(Zg, DZ + Xo.to_dense() @ Yo.to_dense()) <= 2 * eps


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED])
def test_adaptive_z_plus_product(precision):
    """Z = X + X Y from a first product (adaptive bases), then Z + X Y."""
    eps = 1e-5
    pts, X, Y = operands()
    Z = P.h2_clone(X)
    P.h2_mul_add(Z, X, Y, 1e-8, precision)
    DZ = P.h2_to_dense(Z)
    P.h2_mul_add(Z, X, Y, eps, precision)
    DX, DY = P.h2_to_dense(X), P.h2_to_dense(Y)
    assert rel(P.h2_to_dense(Z), DZ + DX @ DY) <= 2 * eps


def test_adaptive_z_exact_mode():
    pts, X, Y = operands()
    Z = P.h2_clone(X)
    P.h2_mul_add(Z, X, Y, 1e-8, P.H2_FP64)
    DZ = P.h2_to_dense(Z)
    P.h2_mul_add(Z, X, Y, 0.0, P.H2_FP64)
    assert rel(P.h2_to_dense(Z), DZ + P.h2_to_dense(X) @ P.h2_to_dense(Y)) <= 1e-12
