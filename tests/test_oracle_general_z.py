"""Pins of "+Z" with Z's own bases (reading: V_Z and W_Z preserved in phase A
beside V_X and W_Y): exact mode reproduces Z + X Y to rounding for Z with
adaptive bases (an earlier product) and for Z of another Chebyshev order; the
truncated product stays within eps; equal bases take the original path."""
import numpy as np
import pytest

import synth
from oracle import h2_oracle as O
from tests.oracle_cases import structure


def _ops(order=3):
    st = structure(order=order)
    return st, O.build_interp(st, O.K_LAPLACE), O.build_interp(st, O.K_YUKAWA)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_same_basis_detects_equal_chebyshev_bases():
    st, X, Y = _ops()
    X2 = O.build_interp(st, O.K_YUKAWA)
    assert O.same_basis(X.V, X2.V) and O.same_basis(X.W, Y.W)
    Z1 = O.mul_add(X, X, Y, 1e-6).result
    assert not O.same_basis(Z1.V, X.V)


@pytest.mark.parametrize("eps", [0.0, 1e-5])
def test_adaptive_z_plus_product(eps):
    st, X, Y = _ops()
    Z1 = O.mul_add(X, X, Y, 1e-8).result  # adaptive isometric bases, ranks != 27
    DZ, DX, DY = Z1.to_dense(), X.to_dense(), Y.to_dense()
    res = O.mul_add(Z1, X, Y, eps)
    assert res.rowsA.RbarZ is not None and res.colsA.RbarZ is not None
    err = rel(res.result.to_dense(), DZ + DX @ DY)
    assert err <= (1e-12 if eps == 0.0 else 2 * eps)


def test_other_order_z():
    """Z interpolated with order 2 on the same points, tree and block tree."""
    st3, X, Y = _ops(order=3)
    st2 = O.build_structure(st3.points, st3.leaf, st3.eta, 2)
    Z = O.build_interp(st2, O.K_LAPLACE)
    res = O.mul_add(Z, X, Y, 0.0)
    assert rel(res.result.to_dense(), Z.to_dense() + X.to_dense() @ Y.to_dense()) <= 1e-12


def test_equal_bases_keep_the_original_path():
    st, X, Y = _ops()
    res = O.mul_add(O.build_interp(st, O.K_LAPLACE), X, Y, 1e-6)
    assert res.rowsA.RbarZ is None and res.colsA.RbarZ is None
