"""Small seeded problems shared by the oracle pin tests (cached per process)."""
import functools

import numpy as np

import synth
from oracle import h2_oracle as O


@functools.lru_cache(maxsize=None)
def structure(geometry="sphere", n=512, leaf=16, eta=2.0, order=2, seed=11):
    return O.build_structure(synth.make_points(geometry, n, seed), leaf, eta, order)


@functools.lru_cache(maxsize=None)
def product(eps, geometry="sphere", n=512, leaf=16, eta=2.0, order=2, seed=11,
            kx=O.K_LAPLACE, ky=O.K_YUKAWA, kz=O.K_LAPLACE):
    st = structure(geometry, n, leaf, eta, order, seed)
    X, Y, Z = O.build_interp(st, kx), O.build_interp(st, ky), O.build_interp(st, kz)
    res = O.mul_add(Z, X, Y, eps)
    Xd, Yd, Zd = X.to_dense(False), Y.to_dense(False), Z.to_dense(False)
    return st, X, Y, Z, res, Xd, Yd, Zd


def block(M, tree, t, s):
    return M[tree.off[t]:tree.off[t] + tree.size[t], tree.off[s]:tree.off[s] + tree.size[s]]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
