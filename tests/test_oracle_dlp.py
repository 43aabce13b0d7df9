"""Pins of the oracle's double-layer operator (the second workload of Sec. 7,
here as point collocation of <n(y), x - y> / (4 pi |x - y|^3) on the cube
surface): closed forms, derivative exactness of the normal-derivative basis,
interpolation convergence, and the product in exact and truncated mode."""
import math

import numpy as np
import pytest

import synth
from oracle import h2_oracle as O


def test_dlp_closed_form():
    x = np.array([[0.5, 0.5, 0.5]])
    y = np.array([[1.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
    ny = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    g = O.dlp_matrix(x, y, ny)
    assert abs(g[0, 0] + 1.0 / math.pi) < 1e-15  # <n, x - y> = -1/2, |x - y|^3 = 1/8
    assert abs(g[0, 1] + 1.0 / math.pi) < 1e-15
    assert O.dlp_matrix(y, y, ny)[0, 0] == 0.0  # coinciding points


def test_normals_of_cube_surface():
    p = synth.cube_surface(500, 3)
    nrm = synth.cube_surface_normals(p)
    assert np.allclose(np.abs(nrm).sum(axis=1), 1.0)
    # the normal points away from the cube centre
    assert np.all(((p - 0.5) * nrm).sum(axis=1) > 0.49)


def test_lagrange_derivative_exact_on_polynomials():
    nodes = O.cheb_nodes_1d(-0.3, 1.1, 5)
    x = np.linspace(-0.3, 1.1, 13)
    p = lambda t: t ** 4 - 2.0 * t ** 2 + t - 1.0
    dp = lambda t: 4.0 * t ** 3 - 4.0 * t + 1.0
    D = O.lagrange_1d_deriv(nodes, x)
    assert np.abs(D @ p(nodes) - dp(x)).max() < 1e-12


def test_normal_derivative_basis_exact_on_polynomials():
    """sum_nu p(xi_nu) d/dn l_nu(x) = grad p(x) . n for p of degree < m per axis."""
    m, lo, hi = 3, np.array([0.0, 0.1, -0.2]), np.array([1.0, 0.7, 0.4])
    rng = np.random.default_rng(4)
    x = lo + (hi - lo) * rng.random((20, 3))
    nrm = rng.standard_normal((20, 3))
    p = lambda q: (1 + q[:, 0]) * (2 - q[:, 1] ** 2) * (q[:, 2] + 3)
    grad = lambda q: np.stack([(2 - q[:, 1] ** 2) * (q[:, 2] + 3), (1 + q[:, 0]) * (-2 * q[:, 1]) * (q[:, 2] + 3),
                               (1 + q[:, 0]) * (2 - q[:, 1] ** 2)], axis=1)
    Dn = O.lagrange_3d_normal(lo, hi, m, x, nrm)
    val = Dn @ p(O.box_nodes(lo, hi, m))
    assert np.abs(val - (grad(x) * nrm).sum(axis=1)).max() < 1e-12


def _dlp(n=600, leaf=16, eta=1.5, order=3, seed=5):
    pts = synth.cube_surface(n, seed)
    nrm = synth.cube_surface_normals(pts)
    st = O.build_structure(pts, leaf, eta, order)
    return st, nrm


def test_fat_boxes():
    st, _ = _dlp()
    lo, hi = O.fat_boxes(st.tree)
    for t in range(st.tree.nclusters):
        ext = hi[t] - lo[t]
        assert ext.min() >= O.DLP_FAT * ext.max() * (1 - 1e-12)
        # contains the bounding box, same centre
        assert np.all(lo[t] <= st.tree.lo[t]) and np.all(hi[t] >= st.tree.hi[t])
        assert np.allclose(lo[t] + hi[t], np.asarray(st.tree.lo[t]) + np.asarray(st.tree.hi[t]))


def test_dlp_interpolation_converges():
    errs = []
    for m in (2, 3, 4):
        st, nrm = _dlp(order=m)
        G = O.build_interp_dlp(st, nrm).to_dense()
        K = O.dlp_matrix(st.points, st.points, nrm)
        errs.append(np.linalg.norm(G - K) / np.linalg.norm(K))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-2


def test_dlp_exact_product_sphere():
    """On the unit sphere with radial normals every block of the double-layer
    operator is nonzero; with V != W (Lagrange rows, normal-derivative columns)
    exact mode (eps = 0) reproduces K + K K to rounding."""
    pts = synth.sphere(600, 5)
    st = O.build_structure(pts, 16, 2.0, 3)
    K = O.build_interp_dlp(st, pts.copy())
    D = K.to_dense()
    R = O.mul_add(K, K, K, 0.0).result.to_dense()
    ref = D + D @ D
    assert np.linalg.norm(R - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("eps", [0.0, 1e-4])
def test_dlp_product_cube_surface(eps):
    """K + K K for the non-symmetric double-layer operator on the cube surface
    (clusters on one face are flat; the interpolation boxes are widened, see
    fat_boxes): exact mode reproduces it to rounding, the truncated product
    stays within eps."""
    st, nrm = _dlp()
    K = O.build_interp_dlp(st, nrm)
    D = K.to_dense()
    assert np.linalg.norm(D - D.T) > 0.1 * np.linalg.norm(D)  # genuinely non-symmetric
    R = O.mul_add(K, K, K, eps).result.to_dense()
    ref = D + D @ D
    err = np.linalg.norm(R - ref) / np.linalg.norm(ref)
    assert err <= (1e-12 if eps == 0.0 else eps)
