"""Batched products: independent products of different sizes, orders and
geometries in one call agree with the same products run one by one, and a
small one with the oracle."""
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


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_MIXED])
def test_batched_matches_single(precision):
    eps = 1e-5
    cases = [("sphere", 2048, 3), ("cube_surface", 3000, 4), ("sphere", 4100, 5), ("cube_surface", 2500, 3),
             ("sphere", 1500, 4), ("cube_surface", 5000, 3)]
    Zs, Xs, refs = [], [], []
    for i, (geom, n, m) in enumerate(cases):
        pts = synth.make_points(geom, n, 2309090613 + 1000 * i)
        X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 64, 2.0, m)
        Z1, Z2 = P.h2_clone(X), P.h2_clone(X)
        P.h2_mul_add(Z1, X, X, eps, precision)
        refs.append(P.h2_to_dense(Z1))
        Z1.free()
        Xs.append(X)
        Zs.append(Z2)
    stats, codes = P.h2_mul_add_batched(Zs, Xs, Xs, eps, precision)
    assert codes == [0] * len(cases)
    for Z, r in zip(Zs, refs):
        assert rel(P.h2_to_dense(Z), r) <= 10 * eps


def test_batched_against_oracle_and_errors():
    eps = 1e-5
    pts = synth.cube_surface(1024, 44)
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 32, 2.0, 3)
    Z = P.h2_clone(X)
    _, codes = P.h2_mul_add_batched([Z], [X], [X], eps, P.H2_MIXED)
    assert codes == [0]
    Xo = O.build_interp(O.build_structure(pts, 32, 2.0, 3), O.K_LAPLACE)
    want = O.mul_add(Xo, Xo, Xo, eps).result.to_dense()
    assert rel(P.h2_to_dense(Z), want) <= 10 * eps
    with pytest.raises(P.H2Error) as e:  # a Z may not be an operand of another product
        P.h2_mul_add_batched([Z, X], [X, Z], [X, Z], eps)
    assert e.value.code == -1


_GROUPED = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import paper_2309_09061_gb300 as P, synth
P.build(); P.load()
eps = 1e-5
cases = [("sphere", 2048, 3), ("cube_surface", 3000, 4), ("sphere", 4100, 5), ("cube_surface", 2500, 3),
         ("sphere", 1500, 4), ("cube_surface", 5000, 3)]
Zs, Xs, refs = [], [], []
for i, (geom, n, m) in enumerate(cases):
    X = P.h2_build_interp(synth.make_points(geom, n, 2309090613 + 1000 * i), P.H2_K_LAPLACE, 64, 2.0, m)
    Z1 = P.h2_clone(X)
    P.h2_mul_add(Z1, X, X, eps, {prec})
    refs.append(P.h2_to_dense(Z1))
    Xs.append(X)
    Zs.append(P.h2_clone(X))
st, codes = P.h2_mul_add_batched(Zs, Xs, Xs, eps, {prec})
assert codes == [0] * len(cases), codes
worst = max(float(np.linalg.norm(P.h2_to_dense(Z) - r) / np.linalg.norm(r)) for Z, r in zip(Zs, refs))
print("worst", worst, "launches", st["kernel_launches"])
assert worst <= 0.1 * eps, worst
"""


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_TF32X3])
def test_grouped_launches_match_single(precision):
    """The opt-in grouped launches (H2_BATCH_GROUPING=1, read once per process:
    run in a child process) give each product the result of the product run
    alone, to rounding (the shared launches split K differently)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, H2_BATCH_GROUPING="1")
    p = subprocess.run([sys.executable, "-c", _GROUPED.format(root=root, prec=precision)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]
    assert "worst" in p.stdout


@pytest.mark.parametrize("precision", [P.H2_FP64, P.H2_TF32X3])
def test_products_are_deterministic(precision):
    """The same product computed twice alone, and once inside a batched call
    (whose default runs every product with its own launches), gives the same
    bits: no kernel of the product depends on the order in which its CTAs
    finish (the per-block sums of squares behind the truncation weights are
    added in a fixed order, not with atomics)."""
    eps = 1e-5
    pts = synth.cube_surface(3000, 2309090617)
    X = P.h2_build_interp(pts, P.H2_K_LAPLACE, 64, 2.0, 4)
    outs = []
    for _ in range(2):
        Z = P.h2_clone(X)
        P.h2_mul_add(Z, X, X, eps, precision)
        outs.append(P.h2_to_dense(Z))
        Z.free()
    assert np.array_equal(outs[0], outs[1])
    Y = P.h2_build_interp(synth.sphere(2048, 7), P.H2_K_LAPLACE, 64, 2.0, 3)
    Zs = [P.h2_clone(X), P.h2_clone(Y)]
    _, codes = P.h2_mul_add_batched(Zs, [X, Y], [X, Y], eps, precision)
    assert codes == [0, 0]
    assert np.array_equal(P.h2_to_dense(Zs[0]), outs[0])
    for A in Zs + [X, Y]:
        A.free()
