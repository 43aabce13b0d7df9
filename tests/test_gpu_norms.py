"""GPU block norms (h2_block_norms): the power iteration whose estimates scale
the blocks before every truncation (Sec. 5 and Sec. 6 choose ranks relative
to block norms), checked block by block against the exact spectral norms of
the oracle's couplings and dense blocks (LAPACK SVD through numpy).

The estimates are lower bounds (up to rounding): an underestimate raises a
block's weight, which only makes its truncation more conservative.  The tests
bound how far below the exact norm they may fall."""
import numpy as np
import pytest

import paper_2309_09061_gb300 as P
import synth
from oracle import h2_oracle as O

pytestmark = pytest.mark.gpu

CASES = {
    # the n = 2048 workload (sphere, Laplace, leaf 32, eta 2, order 3)
    "sphere-n2048": ("sphere", 2048, O.K_LAPLACE, 32, 2.0, 3, 2309090610),
    # cube volume, Yukawa, eta 1.5, order 4 (rank 64 couplings)
    "cube-n4096-yukawa": ("cube", 4096, O.K_YUKAWA, 32, 1.5, 4, 2309090612),
}
# largest relative shortfall below the exact norm: FP64 iteration (stops at a
# relative change of 1e-10) and FP32 iteration (stops at 1e-5)
TOL = {P.H2_FP64: 1e-6, P.H2_MIXED: 1e-3}


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    return P.load()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED])
def test_block_norms_against_exact(name, precision):
    geometry, n, kern, leaf, eta, order, seed = CASES[name]
    pts = synth.make_points(geometry, n, seed)
    A = P.h2_build_interp(pts, kern, leaf, eta, order)
    t, s, kind, nrm = P.h2_block_norms(A, precision)
    st = O.build_structure(pts, leaf, eta, order)
    G = O.build_interp(st, kern)
    tr = st.tree
    # clusters are matched by (first tree position, size), which identifies them
    _, off, size, _, _ = A.structure()
    key_o = {(int(tr.off[c]), int(tr.size[c])): c for c in range(tr.nclusters)}
    cl = [key_o[(int(off[c]), int(size[c]))] for c in range(len(off))]
    worst, checked = 0.0, 0
    for b in range(len(kind)):
        ko = st.blocks.kind[(cl[t[b]], cl[s[b]])]
        if kind[b] == 2:
            assert ko == O.SPLIT
            assert nrm[b] == 0.0
            continue
        if kind[b] == 0:
            assert ko == O.ADM
            exact = np.linalg.norm(G.S[(cl[t[b]], cl[s[b]])], 2)
        else:
            assert ko == O.DENSE
            exact = np.linalg.norm(G.N[(cl[t[b]], cl[s[b]])], 2)
        # a lower bound up to rounding, and close to the norm
        assert nrm[b] <= exact * (1.0 + 1e-6 if precision == P.H2_MIXED else 1.0 + 1e-12), (b, nrm[b], exact)
        short = (exact - nrm[b]) / exact
        worst = max(worst, short)
        assert short <= TOL[precision], (b, int(kind[b]), nrm[b], exact)
        checked += 1
    assert checked == int(np.sum(kind != 2)) > 0
    print(f"{name} precision {precision}: {checked} blocks, largest shortfall {worst:.2e}")
    A.free()
