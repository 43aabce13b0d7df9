"""Block-by-block GPU parity on the target block tree T_IK.

A whole-matrix norm can hide an error confined to a few blocks of small norm
(near-field blocks, low-rank blocks of coarse levels).  These tests compare
every leaf block b = (t, r) of T_IK separately, in all precision modes:

* against the oracle's result:   ||Zg|_b - Zo|_b||_F <= 10 eps ||Zo|_b||_F
  (the spec parity target, per block);
* against the exact Z + X Y:      ||Zg|_b - (Z + XY)|_b||_F <= sqrt(L+1) eps ||(Z + XY)|_b||_F
  (the block-relative error control of Sec. 5 and Sec. 6: the truncation
  errors of the L+1 levels are pairwise orthogonal, so they add in squares).

The oracle's own result is pinned to the same per-block bound on the CPU
(tests/test_oracle_product.py)."""
import math

import numpy as np
import pytest

import paper_2309_09061_gb300 as P
import synth
from oracle import h2_oracle as O

pytestmark = pytest.mark.gpu

PRECISIONS = [P.H2_FP64, P.H2_MIXED, P.H2_TF32X3, P.H2_TF32, P.H2_BF16X3, P.H2_AUTO]
# one TF32 product is meant for eps >= 1e-3, BF16 pieces for eps >= 1e-4
MIN_EPS = {P.H2_TF32: 1e-3, P.H2_BF16X3: 1e-4}

CASES = {
    # sphere, Laplace, leaf 32, eta 2, order 3 (rank 27), eps 1e-4: the n = 2048 workload
    "sphere-n2048": ("sphere", 2048, O.K_LAPLACE, O.K_LAPLACE, 32, 2.0, 3, 1e-4, 2309090610),
    # the same at eps 1e-3, the tolerance of one-term TF32 products
    "sphere-n2048-e3": ("sphere", 2048, O.K_LAPLACE, O.K_LAPLACE, 32, 2.0, 3, 1e-3, 2309090610),
    # cube volume, Yukawa, eta 1.5 (the n = 131072 workload's geometry and kernel, scaled down)
    "cube-n4096-yukawa": ("cube", 4096, O.K_YUKAWA, O.K_YUKAWA, 32, 1.5, 3, 1e-5, 2309090612),
    # X != Y (Laplace x Yukawa) on the cube surface, ragged leaves
    "cube_surface-n3000-mixed-kernels": ("cube_surface", 3000, O.K_LAPLACE, O.K_YUKAWA, 24, 2.0, 3, 1e-5, 31),
    # the n = 32768 workload's parameters at n = 4096 (leaf 64, order 4, rank 64): phase A's
    # upper levels have jobs wider than 64 rows, which the tensor-core modes run on tcgen05
    "sphere-n4096-order4": ("sphere", 4096, O.K_LAPLACE, O.K_LAPLACE, 64, 2.0, 4, 1e-5, 2309090611),
}
# cases whose tensor-core products must include tcgen05 launches
TC_CASES = {"sphere-n4096-order4"}


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    return P.load()


_cache = {}


def oracle_case(name):
    if name not in _cache:
        geometry, n, kx, ky, leaf, eta, order, eps, seed = CASES[name]
        pts = synth.make_points(geometry, n, seed)
        st = O.build_structure(pts, leaf, eta, order)
        X = O.build_interp(st, kx)
        Y = X if ky == kx else O.build_interp(st, ky)
        res = O.mul_add(X, X, Y, eps)  # Z = X
        Xd = X.to_dense(False)
        Yd = Xd if ky == kx else Y.to_dense(False)
        ref = Xd + Xd @ Yd  # tree order
        _cache[name] = (pts, st, res.result.to_dense(False), ref)
    return _cache[name]


def blocks(st):
    tr = st.tree
    for (t, r), k in st.blocks.kind.items():
        if k == O.SPLIT:
            continue
        yield (slice(tr.off[t], tr.off[t] + tr.size[t]), slice(tr.off[r], tr.off[r] + tr.size[r]), k)


@pytest.mark.parametrize("name,precision", [(c, p) for c in CASES for p in PRECISIONS
                                             if CASES[c][7] >= MIN_EPS.get(p, 0.0)])
def test_every_block(name, precision):
    geometry, n, kx, ky, leaf, eta, order, eps, seed = CASES[name]
    pts, st, Zo, ref = oracle_case(name)
    X = P.h2_build_interp(pts, kx, leaf, eta, order)
    Y = X if ky == kx else P.h2_build_interp(pts, ky, leaf, eta, order)
    Z = P.h2_clone(X)
    stats = P.h2_mul_add(Z, X, Y, eps, precision)
    if name in TC_CASES and precision in (P.H2_TF32X3, P.H2_AUTO):
        assert stats["fam_launches"][P.FAMILIES.index("gemm_tc")] > 0
    perm = Z.structure()[0]
    assert np.array_equal(perm, st.tree.perm)
    Zg = P.h2_to_dense(Z)[np.ix_(perm, perm)]  # original order -> tree order
    c = math.sqrt(st.tree.depth + 1)
    worst_o, worst_x, nb = 0.0, 0.0, 0
    for rs, cs, kind in blocks(st):
        g, o, x = Zg[rs, cs], Zo[rs, cs], ref[rs, cs]
        no, nx = np.linalg.norm(o), np.linalg.norm(x)
        do, dx = np.linalg.norm(g - o), np.linalg.norm(g - x)
        worst_o = max(worst_o, do / (no + 1e-300))
        worst_x = max(worst_x, dx / (nx + 1e-300))
        assert do <= 10 * eps * no + 1e-300, (name, kind, do / no)
        assert dx <= c * eps * nx + 1e-300, (name, kind, dx / nx)
        nb += 1
    assert nb == sum(1 for k in st.blocks.kind.values() if k != O.SPLIT)
    print(f"{name} precision {precision}: {nb} blocks, worst vs oracle {worst_o / eps:.2f} eps, "
          f"worst vs Z + XY {worst_x / eps:.2f} eps")
