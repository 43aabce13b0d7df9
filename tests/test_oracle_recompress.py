"""Pins of the oracle's recompression of an input H^2-matrix (orthogonalized
bases, Fig. 1; coarsening with the matrix's own block tree, Fig. 7): the
orthogonal factors are isometric and reproduce the bases, exact mode
reproduces the matrix, truncation stays within eps and lowers the ranks."""
import numpy as np
import pytest

import synth
from oracle import h2_oracle as O
from tests.oracle_cases import structure


def test_orthogonalize():
    st = structure(order=3)
    V = O.build_interp(st, O.K_LAPLACE).V
    Q, R = O.orthogonalize(V)
    for t in range(st.tree.nclusters):
        E, B = Q.expand(t), V.expand(t)
        assert np.abs(E.T @ E - np.eye(E.shape[1])).max() < 1e-13
        assert np.abs(E @ R[t] - B).max() < 1e-12 * max(1.0, np.abs(B).max())


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kernel", [O.K_LAPLACE, O.K_YUKAWA])
def test_recompress_exact_and_truncated(kernel):
    st = structure(order=3)
    A = O.build_interp(st, kernel)
    D = A.to_dense()
    assert rel(O.recompress(A, 0.0).to_dense(), D) <= 1e-12
    eps = 1e-4
    C = O.recompress(A, eps)
    assert rel(C.to_dense(), D) <= eps
    assert max(C.V.rank.values()) < max(A.V.rank.values())  # the Chebyshev rank 27 is not needed at 1e-4
    for t in range(st.tree.nclusters):
        E = C.V.expand(t)
        if E.shape[1]:
            assert np.abs(E.T @ E - np.eye(E.shape[1])).max() < 1e-12


def test_recompress_double_layer():
    pts = synth.cube_surface(600, 5)
    nrm = synth.cube_surface_normals(pts)
    st = O.build_structure(pts, 16, 1.5, 3)
    A = O.build_interp_dlp(st, nrm)
    D = A.to_dense()
    assert rel(O.recompress(A, 1e-5).to_dense(), D) <= 1e-5
