"""Pins of the oracle's input side against closed forms and definitions:
SplitMix64 test vector, Chebyshev nodes, cluster and block tree invariants
(Sec. 2, Def. "Cluster tree", Def. "Block tree"), polynomial exactness of the
interpolation (Example "Integral operator")."""
import math

import numpy as np
import pytest

import synth
from oracle import h2_oracle as O
from tests.oracle_cases import structure


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 for seed 0 (Steele, Lea, Flood 2014 reference code).
    z = synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_point_sets():
    p = synth.sphere(1000, 3)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-15)
    c = synth.cube(1000, 3)
    assert c.min() >= 0.0 and c.max() < 1.0
    s = synth.cube_surface(1000, 3)
    on_face = np.any((s == 0.0) | (s == 1.0), axis=1)
    assert on_face.all()


def test_chebyshev_nodes_and_cardinality():
    x = O.cheb_nodes_1d(-1.0, 1.0, 3)
    assert np.allclose(np.sort(x), [-math.sqrt(3) / 2, 0.0, math.sqrt(3) / 2], atol=1e-15)
    nodes = O.cheb_nodes_1d(0.2, 1.7, 5)
    assert np.allclose(O.lagrange_1d(nodes, nodes), np.eye(5), atol=1e-14)
    # Lagrange polynomials sum to one (they reproduce the constant)
    xs = np.linspace(0.2, 1.7, 11)
    assert np.allclose(O.lagrange_1d(nodes, xs).sum(axis=1), 1.0, atol=1e-13)


@pytest.mark.parametrize("geometry,n,leaf", [("sphere", 512, 16), ("cube", 777, 20), ("cube_surface", 1000, 32)])
def test_cluster_tree(geometry, n, leaf):
    pts = synth.make_points(geometry, n, 5)
    tr = O.build_cluster_tree(pts, leaf)
    assert sorted(tr.perm.tolist()) == list(range(n))
    assert tr.size[0] == n and tr.off[0] == 0
    L = tr.depth
    assert math.ceil(n / 2 ** L) <= leaf and (L == 0 or math.ceil(n / 2 ** (L - 1)) > leaf)
    for t in range(tr.nclusters):
        if tr.is_leaf(t):
            assert tr.level[t] == L and 0 < tr.size[t] <= leaf
            continue
        a, b = tr.children[t]
        assert tr.off[a] == tr.off[t] and tr.off[b] == tr.off[a] + tr.size[a]
        assert tr.size[a] == tr.size[t] // 2 and tr.size[a] + tr.size[b] == tr.size[t]
        raw = pts[tr.indices(t)]
        axis = int(np.argmax(raw.max(0) - raw.min(0)))
        assert pts[tr.indices(a), axis].max() <= pts[tr.indices(b), axis].min()
        for c in (a, b):  # boxes contain their points
            q = pts[tr.indices(c)]
            assert np.all(q >= tr.lo[c] - 1e-15) and np.all(q <= tr.hi[c] + 1e-15)


@pytest.mark.parametrize("eta", [0.0, 1.5, 2.0])
def test_block_tree_partition(eta):
    st = structure(eta=eta)
    tr, bt = st.tree, st.blocks
    n = len(tr.perm)
    cover = np.zeros((n, n), dtype=np.int32)
    for (t, s), k in bt.kind.items():
        if k == O.SPLIT:
            assert not tr.is_leaf(t) and not tr.is_leaf(s)
            assert not O.admissible(tr, tr, t, s, eta)
            continue
        cover[tr.off[t]:tr.off[t] + tr.size[t], tr.off[s]:tr.off[s] + tr.size[s]] += 1
        if k == O.ADM:
            dm = max(O.box_diam(tr.lo[t], tr.hi[t]), O.box_diam(tr.lo[s], tr.hi[s]))
            assert dm <= eta * O.box_dist(tr.lo[t], tr.hi[t], tr.lo[s], tr.hi[s])
            assert tr.level[t] == tr.level[s]
        else:
            assert tr.is_leaf(t) and tr.is_leaf(s)
    assert (cover == 1).all()  # leaves partition I x J exactly once
    if eta == 0.0:
        assert O.ADM not in bt.kind.values()


def test_interp_polynomial_exact():
    """A kernel of degree 2 per coordinate is reproduced exactly by order-3
    interpolation (identity theorem for polynomials)."""
    st = structure(order=3)
    G = O.build_interp(st, O.K_POLY2).to_dense()
    K = O.kernel_matrix(O.K_POLY2, st.points, st.points)
    assert np.linalg.norm(G - K) / np.linalg.norm(K) < 1e-13


def test_transfers_against_direct_lagrange():
    """V_t expanded through the transfer matrices (Eq. transfer) equals the
    Lagrange polynomials of t evaluated directly at the points of t."""
    st = structure(order=3)
    V = O.interp_basis(st.tree, st.points, 3)
    tr = st.tree
    for t in range(tr.nclusters):
        if tr.level[t] in (0, tr.depth):
            continue
        direct = O.lagrange_3d(tr.lo[t], tr.hi[t], 3, st.points[tr.indices(t)])
        assert np.abs(V.expand(t) - direct).max() < 1e-10 * max(1.0, np.abs(direct).max())


def test_interp_converges_laplace():
    errs = []
    for m in (2, 3, 4):
        st = structure(order=m)
        G = O.build_interp(st, O.K_LAPLACE).to_dense()
        K = O.kernel_matrix(O.K_LAPLACE, st.points, st.points)
        errs.append(np.linalg.norm(G - K) / np.linalg.norm(K))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


def test_kernels_closed_form():
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    g = O.kernel_matrix(O.K_LAPLACE, x, x)
    assert g[0, 0] == 0.0 and abs(g[0, 1] - 1.0 / (4 * math.pi * 5.0)) < 1e-17
    y = O.kernel_matrix(O.K_YUKAWA, x, x)
    assert y[1, 1] == 0.0 and abs(y[1, 0] - math.exp(-5.0) / 5.0) < 1e-17
    assert np.array_equal(O.kernel_matrix(O.K_DELTA, x, x), np.eye(2))


@pytest.mark.parametrize("trans", [False, True])
def test_matvec_against_dense(trans):
    """The forward/backward transformation matvec equals the dense product."""
    st = structure(order=3)
    X = O.build_interp(st, O.K_YUKAWA)
    res = O.mul_add(O.build_interp(st, O.K_LAPLACE), O.build_interp(st, O.K_LAPLACE), X, 1e-4).result
    for M in (X, res):  # interpolation bases and adaptive bases of a product
        D = M.to_dense()
        x = synth.normal01(5, D.shape[0] * 3).reshape(-1, 3)
        ref = (D.T if trans else D) @ x
        assert np.abs(M.matvec(x, trans) - ref).max() <= 1e-12 * np.abs(ref).max()
    rows = [0, 7, 100]
    assert np.allclose(X.rows_of(rows), X.to_dense()[rows], rtol=0, atol=1e-13 * np.abs(X.to_dense()).max())
