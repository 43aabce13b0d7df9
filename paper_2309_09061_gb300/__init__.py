"""Python binding of the GB300 H^2-matrix product library (libh2mul.so).

Argument marshalling only: every step of the product runs in the library's
CUDA kernels.  The entry points carry the names of the C-ABI in
``include/h2mul.h``: h2_build_interp, h2_mul_add, h2_to_dense, h2_free.
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

from .build import LIB, build

H2_OK = 0
ERRORS = {-1: "H2_ERR_ARG", -2: "H2_ERR_SHAPE", -3: "H2_ERR_OOM", -4: "H2_ERR_NUMERIC",
          -5: "H2_ERR_TIMEOUT", -6: "H2_ERR_UNSUPPORTED", -7: "H2_ERR_CUDA"}
H2_K_LAPLACE, H2_K_YUKAWA, H2_K_POLY2, H2_K_CONST, H2_K_DELTA, H2_K_DLP = 0, 1, 2, 3, 4, 5
H2_FP64, H2_MIXED, H2_TF32X3, H2_TF32, H2_BF16X3, H2_AUTO = 0, 1, 2, 3, 4, 5
H2_TC = H2_TF32X3
PRECISIONS = {"fp64": H2_FP64, "mixed": H2_MIXED, "tf32x3": H2_TF32X3, "tf32": H2_TF32, "bf16x3": H2_BF16X3,
              "auto": H2_AUTO}

EXPORTED = ["h2_build_interp", "h2_build_interp_normals", "h2_mul_add", "h2_to_dense", "h2_info",
            "h2_get_structure", "h2_clone", "h2_plan_structure", "h2_to_dense_noalloc", "h2_matvec", "h2_mul_add_batched", "h2_product_error",
            "h2_recompress", "h2_library_memory", "h2_free", "h2_error_string", "h2_last_error_message",
            "h2_block_norms"]


class H2Error(RuntimeError):
    def __init__(self, code, what, msg=""):
        self.code = code
        super().__init__(f"{what} failed: {ERRORS.get(code, code)} ({msg})")


class Stats(ctypes.Structure):
    _fields_ = [("t_prep_ms", ctypes.c_double), ("t_rows_a_ms", ctypes.c_double),
                ("t_cols_a_ms", ctypes.c_double), ("t_mat_a_ms", ctypes.c_double),
                ("t_rows_b_ms", ctypes.c_double), ("t_cols_b_ms", ctypes.c_double),
                ("t_mat_b_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("product_nodes", ctypes.c_int64),
                ("triples", ctypes.c_int64), ("max_rank_a", ctypes.c_int), ("max_rank_b", ctypes.c_int),
                ("bytes_moved", ctypes.c_double), ("flops", ctypes.c_double),
                ("fam_ms", ctypes.c_double * 12), ("fam_launches", ctypes.c_int64 * 12),
                ("fam_flops", ctypes.c_double * 12), ("fam_bytes", ctypes.c_double * 12)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if k.startswith("fam_") else v
        return d


FAMILIES = ["gemm_fp64", "gemm_fp32", "qr_fp64", "qr_fp32", "pchol", "svd_fp64", "svd_fp32_pre", "norm", "copy", "other",
            "gemm_tc", "gemm_df"]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("stats", ctypes.POINTER(Stats)), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("autotune", ctypes.c_int)]


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator: the
    h2_opts alloc/free callbacks.  A buffer is allocated for the stream the
    library names (torch keeps it in that stream's pool) and returned with
    stream-ordered semantics, as the callbacks' contract asks.  ``live`` and
    ``calls`` count the bytes held and the allocations made through it."""

    def __init__(self):
        import torch
        torch.cuda.init()  # the raw allocator needs an initialised CUDA state
        raw_alloc = torch._C._cuda_cudaCachingAllocator_raw_alloc
        raw_delete = torch._C._cuda_cudaCachingAllocator_raw_delete
        self.live = 0
        self.calls = 0
        self.last_error = ""

        def _alloc(nbytes, stream, ctx):
            try:
                p = raw_alloc(int(nbytes), int(stream or 0))
            except Exception as e:  # out of memory: the library reports H2_ERR_OOM
                self.last_error = f"{type(e).__name__}: {e}"[:300]
                return None
            self.live += int(nbytes)
            self.calls += 1
            return p

        def _free(ptr, nbytes, stream, ctx):
            try:
                raw_delete(int(ptr))
            except Exception:  # interpreter shutdown: torch's allocator may be gone
                return
            self.live -= int(nbytes)

        # the callback objects live as long as this allocator (module-wide singleton,
        # and referenced by every handle made while it was in use)
        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)
        # handles still alive at exit are freed before PyTorch shuts down (atexit
        # runs the handlers registered last first, and torch registered its own on import)
        atexit.register(_free_live)


_allocator = None  # None: not chosen yet; "library" or a TorchAllocator
_autotune = 0


def set_allocator(kind: str = "torch"):
    """Where the library's device memory comes from: "torch" (PyTorch's caching
    allocator through the h2_opts callbacks, the default when PyTorch has CUDA)
    or "library" (the library's own cudaMalloc and stream-ordered pool)."""
    global _allocator
    if kind == "library":
        _allocator = "library"
    elif kind == "torch":
        _allocator = TorchAllocator()
    else:
        raise ValueError(kind)
    return _allocator


def allocator():
    global _allocator
    if _allocator is None:
        try:
            import torch
            _allocator = TorchAllocator() if torch.cuda.is_available() else "library"
        except ImportError:
            _allocator = "library"
    return _allocator


def set_autotune(on: bool = True):
    """Online tuning of launch schedules (h2_opts.autotune) for later calls."""
    global _autotune
    _autotune = 1 if on else 0


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("depth", ctypes.c_int), ("nclusters", ctypes.c_int),
                ("nblocks", ctypes.c_int64), ("nadmissible", ctypes.c_int64), ("ndense", ctypes.c_int64),
                ("leaf_size", ctypes.c_int), ("order", ctypes.c_int), ("eta", ctypes.c_double),
                ("max_row_rank", ctypes.c_int), ("max_col_rank", ctypes.c_int), ("device_bytes", ctypes.c_double)]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libh2mul.so (built in-tree by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libh2mul.so not found at {path}; run paper_2309_09061_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.h2_build_interp.argtypes = [vp, i64, ci, ci, cd, ci, vp, ctypes.POINTER(vp)]
    lib.h2_build_interp_normals.argtypes = [vp, vp, i64, ci, ci, cd, ci, vp, ctypes.POINTER(vp)]
    lib.h2_mul_add.argtypes = [vp, vp, vp, vp]
    lib.h2_to_dense.argtypes = [vp, vp, i64, ci, vp]
    lib.h2_info.argtypes = [vp, vp]
    lib.h2_get_structure.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.h2_clone.argtypes = [vp, vp, ctypes.POINTER(vp)]
    lib.h2_plan_structure.argtypes = [vp, i64, ci, cd, vp, vp]
    lib.h2_to_dense_noalloc.argtypes = [vp, vp, i64, vp]
    lib.h2_matvec.argtypes = [vp, vp, vp, i64, ci, vp]
    lib.h2_mul_add_batched.argtypes = [vp, vp, vp, ci, vp, vp]
    lib.h2_product_error.argtypes = [vp, vp, vp, vp, vp, ci, vp, vp, vp]
    lib.h2_recompress.argtypes = [vp, vp]
    lib.h2_block_norms.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.h2_library_memory.argtypes = [vp, vp, ci]
    lib.h2_library_memory.restype = ci
    lib.h2_free.argtypes = [vp]
    lib.h2_free.restype = None
    lib.h2_error_string.restype = ctypes.c_char_p
    lib.h2_error_string.argtypes = [ci]
    lib.h2_last_error_message.restype = ctypes.c_char_p
    for f in ("h2_build_interp", "h2_build_interp_normals", "h2_mul_add", "h2_to_dense", "h2_info",
              "h2_get_structure", "h2_clone", "h2_plan_structure", "h2_to_dense_noalloc", "h2_matvec",
              "h2_mul_add_batched", "h2_product_error", "h2_recompress", "h2_block_norms"):
        getattr(lib, f).restype = ci
    _lib = lib
    return lib


def _check(code, what):
    if code != H2_OK:
        msg = load().h2_last_error_message().decode(errors="replace")
        if isinstance(_allocator, TorchAllocator) and _allocator.last_error:
            msg += f"; torch allocator: {_allocator.last_error}"
        raise H2Error(code, what, msg)


def _opts(eps=1e-6, precision=H2_FP64, stream=None, stats=None):
    o = Opts()
    o.eps = eps
    o.precision = precision
    o.stream = ctypes.c_void_p(stream or 0)
    if stats is not None:
        o.stats = ctypes.pointer(stats)
    a = allocator()
    if a != "library":
        o.alloc = a.alloc
        o.free = a.free
    o.autotune = _autotune
    return o


_live = weakref.WeakSet()  # handles not yet freed (released at interpreter exit)


def _free_live():
    for A in list(_live):
        A.free()


class H2Matrix:
    """Owning wrapper of an h2_matrix handle.  It keeps the allocator its
    buffers may have come from alive for as long as it lives (h2_free returns
    them through its callbacks)."""

    def __init__(self, handle):
        self.handle = handle
        self._alloc = _allocator
        _live.add(self)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            load().h2_free(self.handle)
            self.handle = None
            _live.discard(self)

    def info(self) -> dict:
        inf = Info()
        _check(load().h2_info(self.handle, ctypes.byref(inf)), "h2_info")
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def structure(self):
        inf = self.info()
        n, nc = inf["n"], inf["nclusters"]
        perm = np.empty(n, np.int64)
        off = np.empty(nc, np.int64)
        size = np.empty(nc, np.int64)
        rr = np.empty(nc, np.int32)
        cr = np.empty(nc, np.int32)
        _check(load().h2_get_structure(self.handle, perm.ctypes.data, off.ctypes.data, size.ctypes.data,
                                       rr.ctypes.data, cr.ctypes.data), "h2_get_structure")
        return perm, off, size, rr, cr


def h2_build_interp(points: np.ndarray, kernel: int, leaf_size: int, eta: float, cheb_order: int,
                    stream: int | None = None, normals: np.ndarray | None = None) -> H2Matrix:
    """Chebyshev H^2-matrix of a kernel; normals (n x 3) are needed for H2_K_DLP
    (h2_build_interp_normals).  points (and normals) are n x 3 float64 arrays on
    the host, or contiguous float64 CUDA tensors (passed as device pointers)."""
    def ptr(a, what):
        if hasattr(a, "is_cuda") and a.is_cuda:
            if a.dtype != __import__("torch").float64 or not a.is_contiguous() or a.dim() != 2 or a.shape[1] != 3:
                raise ValueError(f"{what} must be a contiguous n x 3 float64 tensor")
            return a, a.data_ptr(), a.shape[0]
        h = np.ascontiguousarray(a, dtype=np.float64)
        if h.ndim != 2 or h.shape[1] != 3:
            raise ValueError(f"{what} must be an n x 3 array")
        return h, h.ctypes.data, h.shape[0]
    pts, pp, n = ptr(points, "points")
    h = ctypes.c_void_p()
    o = _opts(stream=stream)
    if normals is None:
        _check(load().h2_build_interp(pp, n, kernel, leaf_size, eta, cheb_order, ctypes.byref(o), ctypes.byref(h)),
               "h2_build_interp")
    else:
        nrm, npp, nn = ptr(normals, "normals")
        if nn != n:
            raise ValueError("normals must be an n x 3 array like points")
        _check(load().h2_build_interp_normals(pp, npp, n, kernel, leaf_size, eta, cheb_order, ctypes.byref(o),
                                              ctypes.byref(h)), "h2_build_interp_normals")
    return H2Matrix(h)


def h2_mul_add(Z: H2Matrix, X: H2Matrix, Y: H2Matrix, eps: float, precision: int = H2_FP64,
               stream: int | None = None) -> dict:
    """Z <- Z + X Y; returns the call's statistics."""
    st = Stats()
    o = _opts(eps, precision, stream, st)
    _check(load().h2_mul_add(Z.handle, X.handle, Y.handle, ctypes.byref(o)), "h2_mul_add")
    return st.as_dict()


def h2_mul_add_batched(Zs, Xs, Ys, eps: float, precision: int = H2_FP64, stream: int | None = None):
    """Z_i <- Z_i + X_i Y_i for independent products, run concurrently;
    returns (statistics summed over the products, per-product codes)."""
    n = len(Zs)
    arr = ctypes.c_void_p * max(n, 1)
    za, xa, ya = arr(*[z.handle for z in Zs]), arr(*[x.handle for x in Xs]), arr(*[y.handle for y in Ys])
    codes = (ctypes.c_int * max(n, 1))()
    st = Stats()
    o = _opts(eps, precision, stream, st)
    rc = load().h2_mul_add_batched(za, xa, ya, n, ctypes.byref(o), codes)
    _check(rc, "h2_mul_add_batched")
    return st.as_dict(), list(codes)[:n]


def h2_to_dense(A: H2Matrix, out=None, stream: int | None = None) -> np.ndarray:
    """Dense n x n expansion in the original point order (host array), or into a
    device buffer when ``out`` is a CUDA tensor (column-major view of its storage)."""
    n = A.info()["n"]
    o = _opts(stream=stream)
    if out is None:
        buf = np.empty((n, n), dtype=np.float64, order="F")
        _check(load().h2_to_dense(A.handle, buf.ctypes.data, n, 0, ctypes.byref(o)), "h2_to_dense")
        return buf
    _check(load().h2_to_dense(A.handle, out.data_ptr(), n, 1, ctypes.byref(o)), "h2_to_dense")
    return out


def h2_clone(A: H2Matrix, stream: int | None = None) -> H2Matrix:
    h = ctypes.c_void_p()
    o = _opts(stream=stream)
    _check(load().h2_clone(A.handle, ctypes.byref(o), ctypes.byref(h)), "h2_clone")
    return H2Matrix(h)


def h2_plan_structure(points: np.ndarray, leaf_size: int, eta: float):
    """Host-only: (perm, counts) of the trees h2_build_interp would build; counts =
    [depth, adm, dense, split blocks, adm, dense, split T^XY nodes, triples]."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    perm = np.empty(pts.shape[0], np.int64)
    counts = np.empty(8, np.int64)
    _check(load().h2_plan_structure(pts.ctypes.data, pts.shape[0], leaf_size, eta, perm.ctypes.data,
                                    counts.ctypes.data), "h2_plan_structure")
    return perm, counts


def h2_to_dense_noalloc(A: H2Matrix, out, stream: int | None = None, ld: int | None = None):
    """Dense expansion into the CUDA tensor ``out`` without device allocation:
    the library's fixed 32 MiB scratch holds all intermediates.  ``out`` holds
    an n x n float64 matrix column-major with leading dimension ld (default n),
    i.e. the storage of an (n, ld) row-major tensor; rows n..ld-1 of each column
    are left untouched.  Calls must not overlap."""
    n = A.info()["n"]
    ld = n if ld is None else int(ld)
    _check(load().h2_to_dense_noalloc(A.handle, out.data_ptr(), ld, ctypes.c_void_p(stream or 0)),
           "h2_to_dense_noalloc")
    return out


def h2_matvec(A: H2Matrix, x, y, trans: bool = False, stream: int | None = None):
    """y = A x or A^* x for CUDA tensors x, y holding n x nvec float64 matrices
    column-major (the storage of an (nvec, n) row-major tensor)."""
    n = A.info()["n"]
    nv = x.numel() // n
    o = _opts(stream=stream)
    _check(load().h2_matvec(A.handle, x.data_ptr(), y.data_ptr(), nv, 1 if trans else 0, ctypes.byref(o)),
           "h2_matvec")
    return y


def h2_recompress(A: H2Matrix, eps: float, precision: int = H2_FP64, stream: int | None = None) -> dict:
    """A <- A with adaptive isometric bases at tolerance eps (in place); returns statistics."""
    st = Stats()
    o = _opts(eps=eps, precision=precision, stream=stream, stats=st)
    _check(load().h2_recompress(A.handle, ctypes.byref(o)), "h2_recompress")
    return st.as_dict()


def h2_product_error(Zr: H2Matrix, Z0: H2Matrix, X: H2Matrix, Y: H2Matrix, x0=None, steps: int = 20,
                     stream: int | None = None):
    """(eps2, norm): relative spectral error ||Zr - (Z0 + X Y)||_2 / ||Z0 + X Y||_2 and
    ||Z0 + X Y||_2 by power iteration (steps steps each) through H^2 matrix-vector
    products; x0 is an optional float64 start vector (original point order)."""
    o = _opts(stream=stream)
    e, nrm = ctypes.c_double(0.0), ctypes.c_double(0.0)
    xp = None
    if x0 is not None:
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        xp = x0.ctypes.data_as(ctypes.c_void_p)
    _check(load().h2_product_error(Zr.handle, Z0.handle, X.handle, Y.handle, xp, int(steps), ctypes.byref(o),
                                   ctypes.byref(e), ctypes.byref(nrm)), "h2_product_error")
    return e.value, nrm.value


def h2_block_norms(A: H2Matrix, precision: int = H2_FP64, eps: float = 1e-6, stream: int | None = None):
    """(t, s, kind, norm) per block of A's block tree: clusters, kind (0 admissible,
    1 dense, 2 split) and the spectral norm of the stored block by the library's
    power iteration in the given precision (h2_block_norms)."""
    nb = int(A.info()["nblocks"])
    t = np.zeros(nb, np.int32)
    s = np.zeros(nb, np.int32)
    kind = np.zeros(nb, np.int32)
    nrm = np.zeros(nb, np.float64)
    o = _opts(eps=eps, precision=precision, stream=stream)
    _check(load().h2_block_norms(A.handle, ctypes.byref(o), t.ctypes.data, s.ctypes.data, kind.ctypes.data,
                                 nrm.ctypes.data), "h2_block_norms")
    return t, s, kind, nrm


def h2_rows(A: H2Matrix, idx):
    """Rows idx of A as an (len(idx), n) float64 CUDA tensor, computed as A^* e_i."""
    import torch
    n = A.info()["n"]
    idx = torch.as_tensor(idx, dtype=torch.int64)
    e = torch.zeros((len(idx), n), dtype=torch.float64, device="cuda")
    e[torch.arange(len(idx)), idx.to("cuda")] = 1.0
    out = torch.empty_like(e)
    h2_matvec(A, e, out, trans=True)
    return out


def h2_library_memory(reset_peak: bool = False):
    """(current, peak) bytes of device memory the library holds from its own
    sources (cudaMalloc and its pool), not from the allocator callbacks."""
    cur, pk = ctypes.c_int64(0), ctypes.c_int64(0)
    load().h2_library_memory(ctypes.byref(cur), ctypes.byref(pk), 1 if reset_peak else 0)
    return cur.value, pk.value


def h2_free(A: H2Matrix) -> None:
    A.free()
