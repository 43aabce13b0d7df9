"""The 64-product batch at its real size (n log-uniform in [2048, 65536] on the
sphere and the cube surface, orders 3-5, Laplace kernel, leaf 64, eta 2,
eps 1e-5) in the fast form.  Every product of h2_mul_add_batched agrees
with the same product run alone on sampled rows within eps / 10 (the batched
call shares launches between the products, so summation orders differ), and
four products (the
smallest and the largest of each geometry) agree with the oracle's
G + G G on sampled rows within 10 eps."""
import numpy as np
import pytest

import bench
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
    lib = P.load()
    # full sizes take the library's own device memory: its stream-ordered pool reuses
    # freed memory across the streams of a call (PyTorch keeps a pool per stream, and
    # the n = 131072 cube at eps 1e-6 needs over 250 GB at its peak)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    prev = P.allocator()
    P.set_allocator("library")
    yield lib
    P._allocator = prev


def test_batch_of_64_products():
    eps = bench.BATCH["eps"]
    members = bench.batch_members()
    assert len(members) == 64
    pts = [synth.make_points(g, n, seed) for g, n, m, seed in members]
    Gs = [P.h2_build_interp(p, P.H2_K_LAPLACE, bench.BATCH["leaf"], bench.BATCH["eta"], m)
          for p, (g, n, m, seed) in zip(pts, members)]
    Zs = [P.h2_clone(G) for G in Gs]
    _, codes = P.h2_mul_add_batched(Zs, Gs, Gs, eps, P.H2_AUTO)
    assert codes == [0] * 64
    rows = {}
    for i, (G, Z, (g, n, m, seed)) in enumerate(zip(Gs, Zs, members)):
        idx = np.unique(synth.splitmix64(91 + i, 12) % n).astype(np.int64)
        rows[i] = idx
        got = P.h2_rows(Z, idx).cpu().numpy()
        Z1 = P.h2_clone(G)
        P.h2_mul_add(Z1, G, G, eps, P.H2_AUTO)
        alone = P.h2_rows(Z1, idx).cpu().numpy()
        Z1.free()
        # the batched call groups the products' GEMM batches into shared launches, whose
        # split-K choices (hence summation orders) differ from a lone product's: the
        # two results agree to the rounding of the products' arithmetic, far below eps
        assert float(np.linalg.norm(got - alone) / np.linalg.norm(alone)) <= 0.1 * eps, i
    # oracle on the smallest and the largest member of each geometry
    picks = []
    for geom in ("sphere", "cube_surface"):
        ids = [i for i, mb in enumerate(members) if mb[0] == geom]
        picks += [min(ids, key=lambda i: members[i][1]), max(ids, key=lambda i: members[i][1])]
    for i in picks:
        g, n, m, seed = members[i]
        Go = O.build_interp(O.build_structure(pts[i], bench.BATCH["leaf"], bench.BATCH["eta"], m), O.K_LAPLACE)
        Rg = Go.rows_of(rows[i])
        ref = Rg + Go.matvec(Rg.T, trans=True).T
        got = P.h2_rows(Zs[i], rows[i]).cpu().numpy()
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert err <= 10 * eps, (i, n, m, err)
    for Z in Zs:
        Z.free()
    for G in Gs:
        G.free()
