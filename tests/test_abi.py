"""CPU checks of the C-ABI library: it builds, loads, exports every entry
point that include/h2mul.h declares, validates arguments without touching a
device, and its host planner builds the same trees as the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2309_09061_gb300 as P
import synth
from oracle import h2_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "h2mul.h")).read()
    return sorted(set(re.findall(r"H2_API\s+[\w\s\*]*?\b(h2_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(P.EXPORTED) == set(names)


def test_error_strings(lib):
    for code in range(0, -8, -1):
        assert lib.h2_error_string(code)
    assert lib.h2_error_string(-99) == b"unknown error"


def test_argument_validation_without_device(lib):
    h = ctypes.c_void_p()
    pts = np.zeros((4, 3))
    # NULL points, bad sizes, bad kernel, bad order: rejected before any device call
    assert lib.h2_build_interp(None, 4, 0, 2, 2.0, 3, None, ctypes.byref(h)) == -1
    assert lib.h2_build_interp(pts.ctypes.data, 0, 0, 2, 2.0, 3, None, ctypes.byref(h)) == -1
    assert lib.h2_build_interp(pts.ctypes.data, 4, 9, 2, 2.0, 3, None, ctypes.byref(h)) == -1
    assert lib.h2_build_interp(pts.ctypes.data, 4, 0, 2, 2.0, 0, None, ctypes.byref(h)) == -1
    assert lib.h2_build_interp(pts.ctypes.data, 4, 0, 2, -1.0, 3, None, ctypes.byref(h)) == -1
    bad = pts.copy()
    bad[1, 2] = np.nan
    assert lib.h2_build_interp(bad.ctypes.data, 4, 0, 2, 2.0, 3, None, ctypes.byref(h)) == -4
    assert lib.h2_mul_add(None, None, None, None) == -1
    assert lib.h2_to_dense(None, None, 0, 0, None) == -1
    assert lib.h2_info(None, None) == -1
    assert lib.h2_clone(None, None, ctypes.byref(h)) == -1
    assert lib.h2_block_norms(None, None, None, None, None, None) == -1
    lib.h2_free(None)


@pytest.mark.parametrize("geometry,n,leaf,eta", [("sphere", 2048, 32, 2.0), ("cube", 1500, 20, 1.5),
                                                  ("cube_surface", 3000, 64, 2.0), ("sphere", 777, 16, 0.0)])
def test_planner_matches_oracle(lib, geometry, n, leaf, eta):
    pts = synth.make_points(geometry, n, 2309090610)
    perm, counts = P.h2_plan_structure(pts, leaf, eta)
    st = O.build_structure(pts, leaf, eta, 2)
    assert np.array_equal(perm, st.tree.perm)
    kinds = list(st.blocks.kind.values())
    assert counts[0] == st.tree.depth
    assert counts[1:4].tolist() == [kinds.count(O.ADM), kinds.count(O.DENSE), kinds.count(O.SPLIT)]
    X = O.build_interp(st, O.K_CONST) if n <= 800 else None
    if X is not None:
        PT = O.build_product_tree(X, X)
        pk = list(PT.kind.values())
        assert counts[4:7].tolist() == [pk.count(O.ADM), pk.count(O.DENSE), pk.count(O.SPLIT)]
        assert counts[7] == sum(len(v) for v in PT.triples.values())


def test_product_tree_counts_against_oracle(lib):
    pts = synth.sphere(1024, 3)
    perm, counts = P.h2_plan_structure(pts, 16, 2.0)
    st = O.build_structure(pts, 16, 2.0, 1)
    X = O.build_interp(st, O.K_CONST)
    PT = O.build_product_tree(X, X)
    pk = list(PT.kind.values())
    assert counts[4:7].tolist() == [pk.count(O.ADM), pk.count(O.DENSE), pk.count(O.SPLIT)]
    assert counts[7] == sum(len(v) for v in PT.triples.values())


def _c_layout(tmp_path):
    """sizeof/offsetof of the public structs and the enum values, from a C
    program compiled against include/h2mul.h."""
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text('''#include <stddef.h>
#include <stdio.h>
#include "h2mul.h"
int main(void) {
  printf("opts %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(h2_opts), offsetof(h2_opts, eps),
         offsetof(h2_opts, precision), offsetof(h2_opts, stream), offsetof(h2_opts, stats),
         offsetof(h2_opts, alloc), offsetof(h2_opts, free), offsetof(h2_opts, alloc_ctx),
         offsetof(h2_opts, autotune));
  printf("stats %zu\\n", sizeof(h2_stats));
  printf("info %zu\\n", sizeof(h2_info_t));
  printf("prec %d %d %d %d %d %d %d\\n", H2_FP64, H2_MIXED, H2_TF32X3, H2_TC, H2_TF32, H2_BF16X3, H2_AUTO);
  return 0;
}
''')
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no C compiler: " + r.stderr[:200])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    return {ln.split()[0]: [int(x) for x in ln.split()[1:]] for ln in out if ln.strip()}


def test_binding_structs_match_header(tmp_path):
    """The ctypes mirrors of h2_opts, h2_stats and h2_info_t have the C layout,
    and the precision constants are the header's."""
    c = _c_layout(tmp_path)
    O_ = P.Opts
    assert c["opts"] == [ctypes.sizeof(O_)] + [getattr(O_, f).offset for f, _ in O_._fields_]
    assert c["stats"] == [ctypes.sizeof(P.Stats)]
    assert c["info"] == [ctypes.sizeof(P.Info)]
    assert c["prec"] == [P.H2_FP64, P.H2_MIXED, P.H2_TF32X3, P.H2_TC, P.H2_TF32, P.H2_BF16X3, P.H2_AUTO]


def test_precision_and_allocator_validation_without_device(lib):
    """An unknown precision and alloc without free are rejected before any
    device work (H2_ERR_ARG)."""
    o = P.Opts()
    o.eps = 1e-6
    o.precision = 17
    dummy = ctypes.c_void_p(1)
    assert lib.h2_mul_add(dummy, dummy, dummy, ctypes.byref(o)) in (-1, -2)
    o.precision = P.H2_AUTO
    o.alloc = P.ALLOC_FN(lambda n, s, c: None)
    pts = np.random.default_rng(0).random((64, 3))
    h = ctypes.c_void_p()
    # alloc given, free missing: refused (the check runs before the device is touched)
    assert lib.h2_build_interp(pts.ctypes.data, 64, 0, 16, 2.0, 2, ctypes.byref(o), ctypes.byref(h)) == -1


def test_planner_matches_oracle_with_ties(lib):
    """Points on a grid share coordinates along every axis, so the median splits
    are decided by the tie-break on the point index (reading 1); the planner's
    permutation and block counts must still match the oracle's exactly."""
    g = np.arange(10, dtype=np.float64)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3).copy()
    pts = np.ascontiguousarray(np.concatenate([pts, pts[::7]]))  # duplicated points as well
    perm, counts = P.h2_plan_structure(pts, 16, 2.0)
    st = O.build_structure(pts, 16, 2.0, 2)
    assert np.array_equal(perm, st.tree.perm)
    kinds = list(st.blocks.kind.values())
    assert counts[1:4].tolist() == [kinds.count(O.ADM), kinds.count(O.DENSE), kinds.count(O.SPLIT)]
