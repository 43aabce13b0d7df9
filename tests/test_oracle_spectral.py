"""Pins of the oracle's spectral-error estimate (Sec. 7, eps_2 by power
iteration) against closed forms and a library spectral norm."""
import numpy as np

import synth
from oracle import h2_oracle as O
from tests.oracle_cases import structure


def test_power_norm_diagonal_closed_form():
    d = np.array([5.0, -3.0, 1.0, 0.5])
    D = np.diag(d)
    est = O.power_norm(lambda x: D @ x, lambda y: D.T @ y, np.ones(4), 20)
    assert abs(est - 5.0) <= 5.0 * (3.0 / 5.0) ** 38
    assert est <= 5.0 + 1e-15  # a lower bound (Rayleigh quotient of A^* A)


def test_power_norm_matches_library_norm():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((40, 30))
    est = O.power_norm(lambda x: A @ x, lambda y: A.T @ y, synth.normal01(3, 30), 400)
    assert abs(est - np.linalg.norm(A, 2)) <= 1e-10 * np.linalg.norm(A, 2)


def test_spectral_error_of_exact_and_truncated_products():
    st = structure(order=3)
    X = O.build_interp(st, O.K_LAPLACE)
    Y = O.build_interp(st, O.K_YUKAWA)
    DX, DY = X.to_dense(), Y.to_dense()
    D0 = DX.copy()
    x0 = synth.normal01(7, D0.shape[0])
    e, p = O.spectral_error(D0 + DX @ DY, D0, DX, DY, x0)
    assert e <= 1e-13 and p > 0.0  # rounding only: Dr is formed, P is applied
    eps = 1e-4
    R = O.mul_add(X, X, Y, eps).result.to_dense()
    e, p = O.spectral_error(R, D0, DX, DY, x0, steps=60)
    exact = np.linalg.norm(R - D0 - DX @ DY, 2) / np.linalg.norm(D0 + DX @ DY, 2)
    assert 0.0 < e <= exact * (1 + 1e-12) and e >= 0.5 * exact  # lower bound, converged within a factor 2
    assert exact <= eps  # the truncation bound of Sec. 5 in the spectral norm
