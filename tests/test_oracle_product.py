"""Pins of the oracle's product algorithm against definitions, brute force and
closed forms (Sec. 3-6).  X is the Laplace matrix, Y the Yukawa matrix, Z the
Laplace matrix, so that X Y is not symmetric and a transposed operand shows."""
import math

import numpy as np
import pytest

import synth
from oracle import h2_oracle as O
from tests.oracle_cases import block, product, rel, structure


# ---- prep quantities pinned by their defining identities -------------------

def test_basis_products_definition():
    st = structure(order=3)
    V = O.interp_basis(st.tree, st.points, 3)
    P = O.basis_products(V, V)
    for s in range(st.tree.nclusters):
        D = V.expand(s).T @ V.expand(s)
        assert np.abs(P[s] - D).max() <= 1e-12 * np.abs(D).max()


def test_basis_weights_definition():
    """Def. "Basis weight": W_r = Q_r R_r with Q_r isometric, so R^* R = W^* W."""
    st = structure(order=3)
    V = O.interp_basis(st.tree, st.points, 3)
    R = O.basis_weights(V)
    for r in range(st.tree.nclusters):
        W = V.expand(r)
        assert R[r].shape == (min(W.shape), W.shape[1]) or R[r].shape[0] <= W.shape[1]
        assert np.abs(R[r].T @ R[r] - W.T @ W).max() <= 1e-11 * np.abs(W.T @ W).max()


def _ancestors(tree, s):
    out = []
    while s >= 0:
        out.append(s)
        s = tree.parent[s]
    return out


def test_total_weights_definition():
    """Def. "Total weights": P_s Z_s stacks, for s and all its ancestors s*, the
    scaled blocks R_r S_{s*r}^* / ||S_{s*r} R_r^*||_2 moved to s by the
    transfer matrices, so Z_s^* Z_s is their Gram matrix.  Computed here from
    dense expansions, without the top-down recursion."""
    st = structure(order=2)
    Y = O.build_interp(st, O.K_YUKAWA)
    RW = O.basis_weights(Y.W)
    Zt = O.total_weights(Y, RW)
    tree = st.tree
    rowb = st.blocks.row_blocks()
    for s in range(tree.nclusters):
        Vs = Y.V.expand(s)
        gram = np.zeros((Y.V.rank[s], Y.V.rank[s]))
        for a in _ancestors(tree, s):
            Va = Y.V.expand(a)
            # coefficients moving V_a restricted to s into V_s: Va|_s = Vs T
            rows = slice(tree.off[s] - tree.off[a], tree.off[s] - tree.off[a] + tree.size[s])
            T = np.linalg.lstsq(Vs, Va[rows], rcond=None)[0]
            for r in rowb[a]:
                if st.blocks.kind[(a, r)] != O.ADM:
                    continue
                W = Y.W.expand(r)
                nrm = np.linalg.norm(Y.S[(a, r)] @ W.T, 2)  # = ||S R^*||_2
                B = T @ Y.S[(a, r)] @ W.T / nrm
                gram += B @ B.T
        assert np.abs(Zt[s].T @ Zt[s] - gram).max() <= 1e-9 * max(1.0, np.abs(gram).max())


# ---- exact mode (eps = 0): the induced representation is exact (Sec. 3) ----

@pytest.mark.parametrize("geometry,n,leaf,order", [("sphere", 512, 16, 2), ("cube_surface", 400, 16, 2),
                                                   ("cube", 300, 20, 3)])
def test_exact_mode_reproduces_dense_product(geometry, n, leaf, order):
    st, X, Y, Z, res, Xd, Yd, Zd = product(0.0, geometry, n, leaf, 2.0, order)
    ref = Zd + Xd @ Yd
    assert rel(res.induced.to_dense(False), ref) < 1e-12
    assert rel(res.result.to_dense(False), ref) < 1e-12


def test_eta_zero_is_dense_gemm():
    """eta = 0: nothing is admissible, every block is dense and the product is
    the dense matrix product at any eps."""
    st, X, Y, Z, res, Xd, Yd, Zd = product(1e-2, eta=0.0)
    assert O.ADM not in res.result.blocks.kind.values()
    assert rel(res.result.to_dense(False), Zd + Xd @ Yd) < 1e-13


def test_constant_kernel_closed_form():
    """g = 1: G = 1 1^T, so Z + G G = (n + 1) 1 1^T."""
    n = 384
    st, X, Y, Z, res, Xd, Yd, Zd = product(1e-6, n=n, kx=O.K_CONST, ky=O.K_CONST, kz=O.K_CONST)
    F = res.result.to_dense()
    assert np.abs(F - (n + 1)).max() < 1e-10 * (n + 1)


def test_identity_factor():
    """X = I (the delta kernel on distinct points): Z + I Y = Z + Y within eps."""
    eps = 1e-6
    st, X, Y, Z, res, Xd, Yd, Zd = product(eps, kx=O.K_DELTA)
    assert np.array_equal(Xd, np.eye(Xd.shape[0]))
    assert rel(res.result.to_dense(False), Zd + Yd) < eps


# ---- truncated mode: the error bounds of Sec. 5 and Sec. 6 ------------------

@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_truncated_error_bounds(eps):
    st, X, Y, Z, res, Xd, Yd, Zd = product(eps)
    ref = Zd + Xd @ Yd
    F = res.result.to_dense(False)
    assert rel(F, ref) < eps
    tr = st.tree
    c = math.sqrt(tr.depth + 1)
    for (t, r), k in st.blocks.kind.items():
        if k == O.SPLIT:
            continue
        B = block(ref, tr, t, r)
        assert np.linalg.norm(block(F, tr, t, r) - B) <= c * eps * np.linalg.norm(B) + 1e-300


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_phase_a_leaf_bound(eps):
    """Leaf clusters (Fig. 4 with Sec. 5): the scaled remainder is truncated at
    eps in the spectral norm and Z_s^* Z_s dominates every scaled block, so
    ||(I - Q_t Q_t^*) X_ts Y_sr||_2 <= eps ||X_ts V_Y,s||_2 ||S_Y,sr W_Y,r^*||_2
    for every dense (t,s) and admissible (s,r)."""
    st, X, Y, Z, res, Xd, Yd, Zd = product(eps)
    tr, kind = st.tree, st.blocks.kind
    rowb = st.blocks.row_blocks()
    Q = res.rowsA.Q
    worst = 0.0
    for t in range(tr.nclusters):
        if not tr.is_leaf(t):
            continue
        Qt = Q.leaf[t]
        for s in rowb[t]:
            if kind[(t, s)] != O.DENSE:
                continue
            XV = block(Xd, tr, t, s) @ Y.V.leaf[s]
            for r in rowb[s]:
                if kind[(s, r)] != O.ADM:
                    continue
                B = block(Xd, tr, t, s) @ block(Yd, tr, s, r)
                err = np.linalg.norm(B - Qt @ (Qt.T @ B), 2)
                bound = np.linalg.norm(XV, 2) * np.linalg.norm(Y.S[(s, r)] @ Y.W.expand(r).T, 2)
                worst = max(worst, err / bound)
    assert worst <= eps * (1 + 1e-6)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_phase_b_leaf_bound(eps):
    """Leaf clusters of build_basis (Fig. 7): C_t is truncated at eps after
    scaling each target block b by 1/||G|_b||_F, so every T^XY leaf (t,r) in b
    satisfies ||(I - Q'_t Q'_t^*) G|_{t x r}||_2 <= eps ||G|_b||_F."""
    st, X, Y, Z, res, Xd, Yd, Zd = product(eps)
    G = res.induced
    Gd = G.to_dense(False)
    tr = st.tree
    cmap = O.coarse_map(G, st.blocks)
    Qn = res.rowsB.Q
    worst = 0.0
    for (t, r), b in cmap.items():
        if not tr.is_leaf(t) or G.blocks.kind[(t, r)] == O.SPLIT:
            continue
        Qt = Qn.leaf[t]
        B = block(Gd, tr, t, r)
        err = np.linalg.norm(B - Qt @ (Qt.T @ B), 2)
        worst = max(worst, err / np.linalg.norm(block(Gd, tr, *b)))
    assert worst <= eps * (1 + 1e-6)


@pytest.mark.parametrize("eps", [0.0, 1e-4])
def test_bases_isometric_and_range_preserved(eps):
    """Def. "Isometric cluster basis" for every new basis; the induced row basis
    keeps range(V_X,t) and the induced column basis range(W_Y,r) (Sec. 4)."""
    st, X, Y, Z, res, Xd, Yd, Zd = product(eps)
    for basis in (res.rowsA.Q, res.colsA.Q, res.rowsB.Q, res.colsB.Q):
        for t in range(st.tree.nclusters):
            Qt = basis.expand(t)
            if Qt.shape[1]:
                assert np.abs(Qt.T @ Qt - np.eye(Qt.shape[1])).max() < 1e-12
    for t in range(st.tree.nclusters):
        Qt, VX = res.rowsA.Q.expand(t), X.V.expand(t)
        assert np.abs(Qt @ (Qt.T @ VX) - VX).max() < 1e-11 * np.abs(VX).max()
        Wt, WY = res.colsA.Q.expand(t), Y.W.expand(t)
        assert np.abs(Wt @ (Wt.T @ WY) - WY).max() < 1e-11 * np.abs(WY).max()


def test_product_tree_refines_target():
    st, X, Y, Z, res, Xd, Yd, Zd = product(1e-4)
    kind = res.product_tree.kind
    for b, k in st.blocks.kind.items():
        assert b in kind
        if k == O.DENSE:
            assert kind[b] == O.DENSE


# ---- planted mistakes: the pins above must catch them ----------------------

def test_planted_mistakes_are_caught(monkeypatch):
    st = structure(order=2)
    V = O.interp_basis(st.tree, st.points, 2)
    good = O.basis_weights(V)

    def weights_with_adjoint_transfer(W):  # the literal R F^* of Fig. 1
        tree, R = W.tree, {}
        for r in sorted(range(tree.nclusters), key=lambda c: -tree.level[c]):
            if tree.is_leaf(r):
                R[r] = O.qr_r(W.leaf[r], W.rank[r])
            else:
                R[r] = O.qr_r(np.vstack([R[c] @ W.transfer[c].T for c in tree.children[r]]), W.rank[r])
        return R

    bad = weights_with_adjoint_transfer(V)
    r = st.tree.children[0][0]
    W = V.expand(r)
    assert np.abs(good[r].T @ good[r] - W.T @ W).max() < 1e-11 * np.abs(W.T @ W).max()
    assert np.abs(bad[r].T @ bad[r] - W.T @ W).max() > 1e-3 * np.abs(W.T @ W).max()

    # a rank rule that drops too much must break the sharp leaf bound
    eps = 1e-4
    monkeypatch.setattr(O, "choose_rank", lambda sigma, e: int(np.count_nonzero(sigma > 30 * e)))
    X, Y, Z = (O.build_interp(st, k) for k in (O.K_LAPLACE, O.K_YUKAWA, O.K_LAPLACE))
    res = O.mul_add(Z, X, Y, eps)
    ref = Z.to_dense(False) + X.to_dense(False) @ Y.to_dense(False)
    G = res.induced.to_dense(False)
    worst = 0.0
    for t in range(st.tree.nclusters):
        if st.tree.is_leaf(t):
            Qt = res.rowsB.Q.leaf[t]
            for (a, b), blk in O.coarse_map(res.induced, st.blocks).items():
                if a == t and res.induced.blocks.kind[(a, b)] != O.SPLIT:
                    B = block(G, st.tree, a, b)
                    worst = max(worst, np.linalg.norm(B - Qt @ (Qt.T @ B), 2)
                                / np.linalg.norm(block(G, st.tree, *blk)))
    assert worst > eps
