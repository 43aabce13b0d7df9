"""Counter-based SplitMix64 random numbers and the point sets of the workloads.

SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output for a seed is the finaliser applied
to ``seed + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64).  Uniform doubles take the
top 53 bits; normals use the Box-Muller transform.

The paper's experiments (Sec. 7) use Galerkin matrices on a triangulated unit
sphere and cube surface; these generators stand in for them with seeded point
clouds of the same geometry.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 for ``seed`` as uint64."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, 2 * start)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def sphere(n: int, seed: int) -> np.ndarray:
    """n points uniform on the unit sphere (normalised Gaussian triples), n x 3."""
    g = normal01(seed, 3 * n).reshape(n, 3)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def cube(n: int, seed: int) -> np.ndarray:
    """n points uniform in the unit cube [0,1)^3, n x 3."""
    return uniform01(seed, 3 * n).reshape(n, 3)


def cube_surface(n: int, seed: int) -> np.ndarray:
    """n points uniform on the surface of [0,1]^3: a uniform face, then U[0,1)^2 on it."""
    u = uniform01(seed, 3 * n).reshape(n, 3)
    face = np.minimum((u[:, 0] * 6.0).astype(np.int64), 5)
    axis = face % 3
    side = (face // 3).astype(np.float64)
    p = np.empty((n, 3))
    for a in range(3):
        sel = axis == a
        o1, o2 = [b for b in range(3) if b != a]
        p[sel, a] = side[sel]
        p[sel, o1] = u[sel, 1]
        p[sel, o2] = u[sel, 2]
    return p


def cube_surface_normals(p: np.ndarray) -> np.ndarray:
    """Outward unit normals of points on the surface of [0,1]^3 (as drawn by
    cube_surface: exactly one coordinate is 0 or 1): -e_a on the face x_a = 0,
    +e_a on the face x_a = 1."""
    nrm = np.zeros_like(p)
    for i in range(p.shape[0]):
        for a in range(3):
            if p[i, a] == 0.0 or p[i, a] == 1.0:
                nrm[i, a] = 1.0 if p[i, a] == 1.0 else -1.0
                break
    return nrm


def make_points(geometry: str, n: int, seed: int) -> np.ndarray:
    if geometry == "sphere":
        return sphere(n, seed)
    if geometry == "cube":
        return cube(n, seed)
    if geometry == "cube_surface":
        return cube_surface(n, seed)
    raise ValueError(f"unknown geometry {geometry!r}")
