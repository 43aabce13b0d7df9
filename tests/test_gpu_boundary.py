"""GPU tests of the boundary's contract items: device memory from the caller's
allocator (PyTorch's caching allocator through the h2_opts callbacks), points
given in device memory, and every precision mode of the enum against the
FP64 oracle."""
import numpy as np
import pytest

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
    return P.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED, P.H2_TF32X3])
def test_product_with_torch_memory_only(precision):
    """With PyTorch's allocator every device buffer of the calls -- the
    handles and all scratch, in both streams of the product -- comes from
    torch: the library's own device memory stays at zero throughout (its peak
    is read after the calls), torch's allocator saw the calls, and the buffers
    go back to torch when the handles are freed."""
    import torch
    prev = P.allocator()
    ta = P.set_allocator("torch")
    try:
        torch.cuda.synchronize()
        cur0, _ = P.h2_library_memory(reset_peak=True)
        pts = synth.sphere(2048, 2309090610)
        X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
        Z = P.h2_clone(X)
        P.h2_mul_add(Z, X, X, 1e-4, precision)
        got = P.h2_to_dense(Z)
        cur, peak = P.h2_library_memory()
        assert cur == cur0 and peak == cur0, (cur0, cur, peak)
        assert ta.calls > 0
        held = ta.live
        assert held >= int(Z.info()["device_bytes"])
        X.free()
        Z.free()
        assert ta.live == 0
        assert held > 0
        st = O.build_structure(pts, 32, 2.0, 3)
        G = O.build_interp(st, O.K_LAPLACE)
        want = O.mul_add(G, G, G, 1e-4).result.to_dense()
        assert rel(got, want) <= 1e-3
    finally:
        P._allocator = prev


def test_library_allocator_counts_its_memory():
    """With the library's own sources the diagnostic sees the handle's buffers."""
    prev = P.allocator()
    P.set_allocator("library")
    try:
        cur0, _ = P.h2_library_memory()
        X = P.h2_build_interp(synth.sphere(1024, 5), P.H2_K_LAPLACE, 32, 2.0, 3)
        cur1, _ = P.h2_library_memory()
        assert cur1 - cur0 >= int(X.info()["device_bytes"])
        X.free()
    finally:
        P._allocator = prev


def test_points_in_device_memory():
    """Points (and normals) given as CUDA tensors build the same matrix as host
    arrays, bit for bit."""
    import torch
    pts = synth.cube_surface(1500, 7)
    nrm = synth.cube_surface_normals(pts)
    A = P.h2_build_interp(pts, P.H2_K_DLP, 32, 2.0, 3, normals=nrm)
    B = P.h2_build_interp(torch.tensor(pts, device="cuda"), P.H2_K_DLP, 32, 2.0, 3,
                          normals=torch.tensor(nrm, device="cuda"))
    assert np.array_equal(P.h2_to_dense(A), P.h2_to_dense(B))
    C = P.h2_build_interp(torch.tensor(pts, device="cuda"), P.H2_K_LAPLACE, 32, 2.0, 3)
    D = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    assert np.array_equal(P.h2_to_dense(C), P.h2_to_dense(D))


# precision modes and the tolerances they are meant for (H2_AUTO picks by eps)
MODES = [
    (P.H2_TF32, 1e-3), (P.H2_TF32, 3e-3), (P.H2_BF16X3, 1e-4), (P.H2_BF16X3, 3e-4), (P.H2_TF32X3, 1e-5),
    (P.H2_TF32X3, 1e-6), (P.H2_AUTO, 1e-3), (P.H2_AUTO, 1e-4), (P.H2_AUTO, 1e-5), (P.H2_AUTO, 1e-6),
    (P.H2_AUTO, 1e-8),
]


@pytest.mark.parametrize("precision,eps", MODES)
def test_precision_modes_against_oracle(precision, eps):
    """Every mode of the enum: X != Y (Laplace x Yukawa) on the cube surface,
    against the oracle within 10 eps and against Z + XY within 2 eps."""
    pts = synth.cube_surface(2000, 13)
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, 32, 2.0, 3)
    Z = P.h2_clone(X)
    P.h2_mul_add(Z, X, Y, eps, precision)
    st = O.build_structure(pts, 32, 2.0, 3)
    Xo, Yo = O.build_interp(st, O.K_LAPLACE), O.build_interp(st, O.K_YUKAWA)
    want = O.mul_add(Xo, Xo, Yo, eps).result.to_dense()
    ref = Xo.to_dense() + Xo.to_dense() @ Yo.to_dense()
    got = P.h2_to_dense(Z)
    assert rel(got, want) <= 10 * eps
    assert rel(got, ref) <= 2 * eps


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED, P.H2_TF32X3])
def test_autotuned_products_against_oracle(precision):
    """h2_opts.autotune: the first calls run the candidate schedules of each
    batch key in turn (split-K variants; for FP32-class products also the
    other kernel), later calls the fastest.  Every call's result matches the
    oracle within 10 eps and Z + XY within eps."""
    eps = 1e-5
    pts = synth.sphere(2048, 2309090610)
    st = O.build_structure(pts, 32, 2.0, 3)
    G = O.build_interp(st, O.K_LAPLACE)
    want = O.mul_add(G, G, G, eps).result.to_dense()
    ref = G.to_dense() + G.to_dense() @ G.to_dense()
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    P.set_autotune(True)
    try:
        for _ in range(6):  # 8 candidates x 2 timings per key need a few calls to settle
            Z = P.h2_clone(X)
            P.h2_mul_add(Z, X, X, eps, precision)
            got = P.h2_to_dense(Z)
            assert rel(got, want) <= 10 * eps
            assert rel(got, ref) <= eps
            Z.free()
    finally:
        P.set_autotune(False)
