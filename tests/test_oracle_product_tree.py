"""Brute-force pins of the product block tree T^XY (Sec. 6) built by the
oracle: its leaves tile I x K exactly once, and for every leaf (t, r) the
triples (a, s, b) met on the way from the root to (t, r), restricted to t x r,
add up to the dense product (XY)|t x r.  A dropped or doubled triple breaks
the sum.  The map from T^XY nodes to the admissible target blocks of phase B
is checked against containment of index ranges."""
import numpy as np
import pytest

from oracle import h2_oracle as O
import synth


def _setup(geometry, n, leaf, seed):
    pts = synth.make_points(geometry, n, seed)
    st = O.build_structure(pts, leaf, 2.0, 3)
    X = O.build_interp(st, O.K_LAPLACE)
    Y = O.build_interp(st, O.K_YUKAWA)
    return X, Y, O.build_product_tree(X, Y)


def _rng(tree, c):
    return slice(tree.off[c], tree.off[c] + tree.size[c])


def _leaf_sums(X, Y, P):
    """For every leaf of T^XY: the sum of its and its ancestors' triples on t x r."""
    Xd, Yd = X.to_dense(False), Y.to_dense(False)
    rows, mid, cols = X.rows, X.cols, Y.cols
    parent = {}
    for node, ch in P.children.items():
        for c in ch:
            parent[c] = node
    out = {}
    for node, kind in P.kind.items():
        if kind == O.SPLIT:
            continue
        t, r = node
        acc = np.zeros((rows.size[t], cols.size[r]))
        a = node
        while True:
            for s in P.triples[a]:
                acc += Xd[_rng(rows, t), _rng(mid, s)] @ Yd[_rng(mid, s), _rng(cols, r)]
            if a not in parent:
                break
            a = parent[a]
        out[node] = acc
    return out, Xd @ Yd


@pytest.mark.parametrize("geometry,n,leaf", [("cube", 300, 16), ("sphere", 257, 20), ("cube_surface", 400, 24)])
def test_leaves_tile_and_triples_sum_to_the_product(geometry, n, leaf):
    X, Y, P = _setup(geometry, n, leaf, 2309090631)
    sums, XY = _leaf_sums(X, Y, P)
    cover = np.zeros(XY.shape, dtype=int)
    for (t, r), acc in sums.items():
        cover[_rng(X.rows, t), _rng(Y.cols, r)] += 1
        ref = XY[_rng(X.rows, t), _rng(Y.cols, r)]
        assert np.allclose(acc, ref, rtol=1e-12, atol=1e-12 * np.abs(XY).max())
    assert (cover == 1).all()


def test_dropped_triple_is_detected():
    X, Y, P = _setup("cube", 300, 16, 2309090632)
    # plant a mistake in the oracle's tree: drop one triple of a node with several
    node = next(k for k, v in P.triples.items() if len(v) > 1)
    P.triples[node] = P.triples[node][1:]
    sums, XY = _leaf_sums(X, Y, P)
    bad = [k for k, acc in sums.items()
           if not np.allclose(acc, XY[_rng(X.rows, k[0]), _rng(Y.cols, k[1])], rtol=1e-12,
                              atol=1e-12 * np.abs(XY).max())]
    assert bad


@pytest.mark.parametrize("geometry,n,leaf", [("cube", 300, 16), ("sphere", 257, 20)])
def test_coarse_map_by_index_ranges(geometry, n, leaf):
    """Every T^XY node inside an admissible target block of T_IK maps to exactly
    that block (containment of index ranges), and no other node is mapped."""
    pts = synth.make_points(geometry, n, 2309090633)
    st = O.build_structure(pts, leaf, 2.0, 3)
    X = O.build_interp(st, O.K_LAPLACE)
    res = O.mul_add(O.build_interp(st, O.K_LAPLACE), X, O.build_interp(st, O.K_YUKAWA), 1e-4)
    G = res.induced
    cmap = O.coarse_map(G, st.blocks)
    tree = st.tree
    targets = [b for b, k in st.blocks.kind.items() if k == O.ADM]

    def inside(node, blk):
        (t, r), (bt, br) = node, blk
        return (tree.off[bt] <= tree.off[t] and tree.off[t] + tree.size[t] <= tree.off[bt] + tree.size[bt]
                and tree.off[br] <= tree.off[r] and tree.off[r] + tree.size[r] <= tree.off[br] + tree.size[br])

    for node in G.blocks.kind:
        holders = [b for b in targets if inside(node, b)]
        assert len(holders) <= 1  # admissible target blocks are disjoint
        if holders:
            assert cmap.get(node) == holders[0]
        else:
            assert node not in cmap
