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
