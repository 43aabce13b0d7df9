"""The allocation-free dense expansion.

h2_to_dense_noalloc serves callers that cannot allocate device memory while
they run (code under another allocator's control, or a phase that forbids
cudaMalloc): all of its scratch lives in one fixed device array inside the
library.  Its result must equal the one of h2_to_dense, call after call,
although the array keeps the previous call's contents.  This file is
collected last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

import paper_2309_09061_gb300 as P
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    return P.load()


def _dense_pair(A, n):
    import torch
    dev = torch.device("cuda:0")
    ref = torch.empty((n, n), dtype=torch.float64, device=dev)
    P.h2_to_dense(A, ref)
    got = [torch.full((n, n), float("nan"), dtype=torch.float64, device=dev) for _ in range(2)]
    for g in got:  # two calls in a row through the C-ABI
        P.h2_to_dense_noalloc(A, g)
    torch.cuda.synchronize()
    return ref, got


@pytest.mark.parametrize("kind", ["interp", "product"])
def test_noalloc_matches_to_dense(kind):
    import torch
    n = 1024
    pts = synth.sphere(n, 31)
    A = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    if kind == "product":  # adaptive ranks, separate row and column bases
        Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, 32, 2.0, 3)
        P.h2_mul_add(A, A, Y, 1e-6)
    ref, got = _dense_pair(A, n)
    for g in got:
        err = float(torch.linalg.norm(g - ref) / torch.linalg.norm(ref))
        assert err <= 1e-14, err


def test_noalloc_rejects_too_large():
    import torch
    n = 2100  # n^2 alone exceeds the 4 Mi-double scratch
    A = P.h2_build_interp(synth.sphere(n, 3), P.H2_K_LAPLACE, 64, 2.0, 2)
    out = torch.empty((n, n), dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.H2Error) as e:
        P.h2_to_dense_noalloc(A, out)
    assert e.value.code == -6


def _product_matrix(n=1024):
    pts = synth.sphere(n, 31)
    A = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    Y = P.h2_build_interp(pts, P.H2_K_YUKAWA, 32, 2.0, 3)
    P.h2_mul_add(A, A, Y, 1e-6)
    return A


def test_noalloc_leading_dimension_and_stream():
    """ld = n + 7 on a non-default stream: rows 0..n-1 of every column equal
    h2_to_dense, the padding rows n..ld-1 keep their NaN, two calls in a row."""
    import torch
    n = 1024
    ld = n + 7
    A = _product_matrix(n)
    ref = torch.empty((n, n), dtype=torch.float64, device="cuda:0")
    P.h2_to_dense(A, ref)
    s = torch.cuda.Stream()
    for _ in range(2):
        out = torch.full((n, ld), float("nan"), dtype=torch.float64, device="cuda:0")  # column j = out[j]
        torch.cuda.synchronize()
        P.h2_to_dense_noalloc(A, out, stream=s.cuda_stream, ld=ld)
        torch.cuda.synchronize()
        assert bool(torch.isnan(out[:, n:]).all())
        err = float(torch.linalg.norm(out[:, :n] - ref) / torch.linalg.norm(ref))
        assert err <= 1e-14, err


def test_noalloc_allocates_nothing():
    """Free device memory is the same before and after warmed-up calls: the
    call takes nothing from the driver, the library's pool or torch."""
    import torch
    n = 1024
    A = _product_matrix(n)
    out = torch.empty((n, n), dtype=torch.float64, device="cuda:0")
    P.h2_to_dense_noalloc(A, out)  # warm-up: module load, symbol lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        P.h2_to_dense_noalloc(A, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
