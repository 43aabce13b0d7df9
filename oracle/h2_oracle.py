"""FP64 CPU oracle for the adaptive H^2-matrix product Z <- Z + X Y.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or
runs this module; only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path.

It follows S. Boerm, "Adaptive fast multiplication of H^2-matrices"
(arXiv 2309.09061) step by step, in plain numpy float64, recursively as the
paper's figures are written:

* Sec. 2   cluster tree (Def. "Cluster tree"), block tree (Def. "Block tree"),
           H^2-matrix (Eq. vsw, Def. "Cluster basis", Def. "H^2-matrix"),
           Chebyshev interpolation (Example "Integral operator").
* Sec. 3   induced bases and the semi-uniform products (Eq. semiuniform,
           Eq. semiuniform2).
* Sec. 4   basis weights (Fig. 1), total weights (Fig. 2), cluster basis
           products, compressed induced row basis (Fig. 4); the column basis is
           the same procedure on the adjoint product Y^* X^*.
* Sec. 5   block-relative error control (scaling of the blocks).
* Sec. 6   product block tree T^XY, coarsening to the prescribed block tree:
           total weights (Eq. Zt_condensation), leaf and non-leaf condensed
           matrices (Eq. ct_leaf, Eq. ct_nonleaf), column trees and
           match_column (Fig. 6), build_basis (Fig. 7); the column basis is
           the same procedure on G^*.

Library primitives used as single steps: matrix products, Householder QR
(numpy.linalg.qr, LAPACK geqrf/orgqr) and the SVD (numpy.linalg.svd).

Readings where the paper is silent or garbled are marked "Reading:" at the
place they are used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Kernel functions g(x, y) (Sec. 7 uses 1/(4 pi |x-y|); the workloads add the
# Yukawa-type exp(-|x-y|)/|x-y|).  POLY2, CONST and DELTA exist for the
# closed-form pins: (1 + x.y)^2 is a polynomial of degree 2 per coordinate,
# CONST gives the all-ones matrix, DELTA gives the identity for distinct points.
K_LAPLACE, K_YUKAWA, K_POLY2, K_CONST, K_DELTA = 0, 1, 2, 3, 4
# Double-layer potential of the Laplace kernel (Sec. 7's second operator, as point
# collocation): <n(y), x - y> / (4 pi |x - y|^3), 0 on coinciding points.
K_DLP = 5

TINY = 1e-300


def kernel_matrix(kernel: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """g(x_i, y_j) for point sets x (m x 3) and y (n x 3)."""
    if kernel == K_POLY2:
        return (1.0 + x @ y.T) ** 2
    if kernel == K_CONST:
        return np.ones((x.shape[0], y.shape[0]))
    d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(axis=2))
    if kernel == K_DELTA:
        return (d == 0.0).astype(np.float64)
    zero = d == 0.0
    dd = np.where(zero, 1.0, d)
    if kernel == K_LAPLACE:
        g = 1.0 / (4.0 * math.pi * dd)
    elif kernel == K_YUKAWA:
        g = np.exp(-dd) / dd
    else:
        raise ValueError(kernel)
    # The singular kernels are set to 0 on coinciding points ("diagonal 0").
    return np.where(zero, 0.0, g)


def dlp_matrix(x: np.ndarray, y: np.ndarray, ny: np.ndarray) -> np.ndarray:
    """<n(y_j), x_i - y_j> / (4 pi |x_i - y_j|^3), the normal derivative in y of
    1 / (4 pi |x - y|); 0 on coinciding points."""
    diff = x[:, None, :] - y[None, :, :]
    d = np.sqrt((diff ** 2).sum(axis=2))
    zero = d == 0.0
    dd = np.where(zero, 1.0, d)
    g = (diff * ny[None, :, :]).sum(axis=2) / (4.0 * math.pi * dd ** 3)
    return np.where(zero, 0.0, g)


# --------------------------------------------------------------------------
# Sec. 2: cluster tree
# --------------------------------------------------------------------------

@dataclass
class ClusterTree:
    """Def. "Cluster tree": clusters with index sets, children and boxes.

    Clusters are numbered in creation (pre-)order; ``perm[p]`` is the original
    index at position p, and cluster t owns positions off[t] .. off[t]+size[t].
    """
    perm: np.ndarray
    off: list = field(default_factory=list)
    size: list = field(default_factory=list)
    level: list = field(default_factory=list)
    parent: list = field(default_factory=list)
    children: list = field(default_factory=list)
    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)
    depth: int = 0

    @property
    def nclusters(self):
        return len(self.off)

    def is_leaf(self, t):
        return not self.children[t]

    def indices(self, t):
        return self.perm[self.off[t]:self.off[t] + self.size[t]]

    def by_level(self):
        lv = [[] for _ in range(self.depth + 1)]
        for t in range(self.nclusters):
            lv[self.level[t]].append(t)
        return lv


def tree_depth(n: int, leaf: int) -> int:
    """Reading: every cluster above depth L is split, L the smallest depth with
    ceil(n / 2^L) <= leaf, so that all leaves share one level."""
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    return L


def cluster_box(pts: np.ndarray, pad: float):
    """Tight axis-aligned box of the points; extents below ``pad`` are widened
    symmetrically to ``pad`` (Reading: flat clusters on the cube surface)."""
    lo = pts.min(axis=0).copy()
    hi = pts.max(axis=0).copy()
    for a in range(3):
        if hi[a] - lo[a] < pad:
            c = 0.5 * (lo[a] + hi[a])
            lo[a] = c - 0.5 * pad
            hi[a] = c + 0.5 * pad
    return lo, hi


def build_cluster_tree(points: np.ndarray, leaf: int) -> ClusterTree:
    """Median bisection (Reading of "bisection"): split along the longest box
    axis (ties to the lowest axis), stable order by (coordinate, original
    index), the first floor(#t/2) indices go to the first child."""
    n = points.shape[0]
    L = tree_depth(n, leaf)
    root_ext = points.max(axis=0) - points.min(axis=0) if n else np.zeros(3)
    pad = 1e-8 * max(float(root_ext.max()) if n else 0.0, 1e-300)
    tree = ClusterTree(perm=np.arange(n, dtype=np.int64), depth=L)

    def make(idx, off, level, parent):
        t = len(tree.off)
        tree.off.append(off)
        tree.size.append(len(idx))
        tree.level.append(level)
        tree.parent.append(parent)
        tree.children.append([])
        lo, hi = cluster_box(points[idx], pad)
        tree.lo.append(lo)
        tree.hi.append(hi)
        if level < L:
            raw = points[idx]
            ext = raw.max(axis=0) - raw.min(axis=0)
            axis = int(np.argmax(ext))  # first maximum = lowest axis on ties
            order = np.lexsort((idx, raw[:, axis]))
            idx = idx[order]
            h = len(idx) // 2
            c1 = make(idx[:h], off, level + 1, t)
            c2 = make(idx[h:], off + h, level + 1, t)
            tree.children[t] = [c1, c2]
        else:
            tree.perm[off:off + len(idx)] = idx
        return t

    make(np.arange(n, dtype=np.int64), 0, 0, -1)
    return tree


# --------------------------------------------------------------------------
# Sec. 2: block tree and admissibility
# --------------------------------------------------------------------------

ADM, DENSE, SPLIT = "adm", "dense", "split"


def box_diam(lo, hi):
    return float(np.sqrt(((hi - lo) ** 2).sum()))


def box_dist(lo1, hi1, lo2, hi2):
    gap = np.maximum(0.0, np.maximum(lo1 - hi2, lo2 - hi1))
    return float(np.sqrt((gap ** 2).sum()))


def admissible(rt: ClusterTree, ct: ClusterTree, t: int, s: int, eta: float) -> bool:
    """Standard admissibility max(diam B_t, diam B_s) <= eta dist(B_t, B_s)."""
    dm = max(box_diam(rt.lo[t], rt.hi[t]), box_diam(ct.lo[s], ct.hi[s]))
    return dm <= eta * box_dist(rt.lo[t], rt.hi[t], ct.lo[s], ct.hi[s])


@dataclass
class BlockTree:
    """Def. "Block tree": kind[(t,s)] in {adm, dense, split}; children of a
    split block are chil(t) x chil(s)."""
    rows: ClusterTree
    cols: ClusterTree
    kind: dict
    children: dict

    def row_blocks(self):
        """t -> list of s with (t,s) in the block tree."""
        out = {t: [] for t in range(self.rows.nclusters)}
        for (t, s) in self.kind:
            out[t].append(s)
        for t in out:
            out[t].sort()
        return out

    def col_blocks(self):
        out = {s: [] for s in range(self.cols.nclusters)}
        for (t, s) in self.kind:
            out[s].append(t)
        for s in out:
            out[s].sort()
        return out

    def transpose(self) -> "BlockTree":
        return BlockTree(self.cols, self.rows, {(s, t): k for (t, s), k in self.kind.items()},
                         {(s, t): [(b, a) for (a, b) in ch] for (t, s), ch in self.children.items()})


def build_block_tree(rt: ClusterTree, ct: ClusterTree, eta: float) -> BlockTree:
    kind, children = {}, {}

    def rec(t, s):
        if admissible(rt, ct, t, s, eta):
            kind[(t, s)] = ADM
        elif rt.is_leaf(t) or ct.is_leaf(s):
            kind[(t, s)] = DENSE
        else:
            kind[(t, s)] = SPLIT
            children[(t, s)] = [(a, b) for a in rt.children[t] for b in ct.children[s]]
            for a, b in children[(t, s)]:
                rec(a, b)

    rec(0, 0)
    return BlockTree(rt, ct, kind, children)


# --------------------------------------------------------------------------
# Sec. 2: cluster bases and H^2-matrices
# --------------------------------------------------------------------------

@dataclass
class Basis:
    """Def. "Cluster basis": leaf matrices V_t (#t x k_t) and transfer matrices
    E_t' (k_t' x k_t) with V_t|_{t' x k} = V_t' E_t' (Eq. transfer)."""
    tree: ClusterTree
    rank: dict
    leaf: dict
    transfer: dict

    def expand(self, t: int) -> np.ndarray:
        """The full matrix V_t (#t x k_t) through the transfer matrices."""
        if self.tree.is_leaf(t):
            return self.leaf[t]
        return np.vstack([self.expand(c) @ self.transfer[c] for c in self.tree.children[t]])


@dataclass
class H2Matrix:
    """Def. "H^2-matrix": G|_{t x s} = V_t S_ts W_s^* on admissible leaves
    (Eq. vsw), dense N_ts on inadmissible leaves."""
    blocks: BlockTree
    V: Basis
    W: Basis
    S: dict
    N: dict

    @property
    def rows(self):
        return self.blocks.rows

    @property
    def cols(self):
        return self.blocks.cols

    def transpose(self) -> "H2Matrix":
        return H2Matrix(self.blocks.transpose(), self.W, self.V,
                        {(s, t): m.T for (t, s), m in self.S.items()},
                        {(s, t): m.T for (t, s), m in self.N.items()})

    def matvec(self, x: np.ndarray, trans: bool = False) -> np.ndarray:
        """G x (or G^* x) for x in the original point order (n x nv), by the
        forward transformation x_s = W_s^* x|_s (leaves directly, parents
        through the transfer matrices), the couplings y_t = sum_s S_ts x_s, the
        backward transformation and the dense blocks (Sec. 2: O(nk) work)."""
        A = self.transpose() if trans else self
        x = np.asarray(x, dtype=np.float64)
        one = x.ndim == 1
        X = x[:, None] if one else x
        rt, ct = A.rows, A.cols
        xt = X[ct.perm]
        xh = {}

        def fwd(s):
            if ct.is_leaf(s):
                xh[s] = A.W.leaf[s].T @ xt[ct.off[s]:ct.off[s] + ct.size[s]]
            else:
                acc = np.zeros((A.W.rank[s], X.shape[1]))
                for c in ct.children[s]:
                    fwd(c)
                    acc += A.W.transfer[c].T @ xh[c]
                xh[s] = acc

        fwd(0)
        yh = {t: np.zeros((A.V.rank[t], X.shape[1])) for t in range(rt.nclusters)}
        yt = np.zeros((len(rt.perm), X.shape[1]))
        for (t, s), k in A.blocks.kind.items():
            if k == ADM:
                yh[t] += A.S[(t, s)] @ xh[s]
            elif k == DENSE:
                yt[rt.off[t]:rt.off[t] + rt.size[t]] += A.N[(t, s)] @ xt[ct.off[s]:ct.off[s] + ct.size[s]]

        def bwd(t, acc):
            acc = yh[t] if acc is None else yh[t] + acc
            if rt.is_leaf(t):
                yt[rt.off[t]:rt.off[t] + rt.size[t]] += A.V.leaf[t] @ acc
            else:
                for c in rt.children[t]:
                    bwd(c, A.V.transfer[c] @ acc)

        bwd(0, None)
        out = np.empty_like(yt)
        out[rt.perm] = yt
        return out[:, 0] if one else out

    def rows_of(self, idx) -> np.ndarray:
        """Rows idx of G (len(idx) x n) as G^* applied to unit vectors."""
        E = np.zeros((len(self.cols.perm), len(idx)))
        E[np.asarray(idx), np.arange(len(idx))] = 1.0
        return self.matvec(E, trans=True).T

    def to_dense(self, original_order: bool = True) -> np.ndarray:
        rt, ct = self.rows, self.cols
        G = np.zeros((len(rt.perm), len(ct.perm)))
        for (t, s), k in self.blocks.kind.items():
            r0, r1 = rt.off[t], rt.off[t] + rt.size[t]
            c0, c1 = ct.off[s], ct.off[s] + ct.size[s]
            if k == ADM:
                G[r0:r1, c0:c1] = self.V.expand(t) @ self.S[(t, s)] @ self.W.expand(s).T
            elif k == DENSE:
                G[r0:r1, c0:c1] = self.N[(t, s)]
        if original_order:
            out = np.empty_like(G)
            out[np.ix_(rt.perm, ct.perm)] = G
            return out
        return G


# --------------------------------------------------------------------------
# Example "Integral operator": H^2-matrix by Chebyshev interpolation
# --------------------------------------------------------------------------

def cheb_nodes_1d(a: float, b: float, m: int) -> np.ndarray:
    """First-kind Chebyshev nodes on [a, b] (Reading: first kind, order m)."""
    i = np.arange(m)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * i + 1) * np.pi / (2 * m))


def lagrange_1d(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[p, i] = l_i(x_p) for the Lagrange polynomials of ``nodes``."""
    m = len(nodes)
    out = np.ones((len(x), m))
    for i in range(m):
        for j in range(m):
            if j != i:
                out[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return out


def lagrange_1d_deriv(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[p, i] = l_i'(x_p): the product rule over the factors of l_i."""
    m = len(nodes)
    out = np.zeros((len(x), m))
    for i in range(m):
        for k in range(m):
            if k == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[k]))
            for j in range(m):
                if j != i and j != k:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            out[:, i] += term
    return out


def box_nodes(lo, hi, m):
    """Tensor nodes xi_nu, nu = i_x + m i_y + m^2 i_z, as a (m^3 x 3) array."""
    nx, ny, nz = (cheb_nodes_1d(lo[a], hi[a], m) for a in range(3))
    out = np.empty((m ** 3, 3))
    for iz in range(m):
        for iy in range(m):
            for ix in range(m):
                out[ix + m * iy + m * m * iz] = (nx[ix], ny[iy], nz[iz])
    return out


def lagrange_3d(lo, hi, m, x: np.ndarray) -> np.ndarray:
    """l_{t,nu}(x_p) as a (#x x m^3) matrix."""
    Lx, Ly, Lz = (lagrange_1d(cheb_nodes_1d(lo[a], hi[a], m), x[:, a]) for a in range(3))
    out = np.empty((x.shape[0], m ** 3))
    for iz in range(m):
        for iy in range(m):
            for ix in range(m):
                out[:, ix + m * iy + m * m * iz] = Lx[:, ix] * Ly[:, iy] * Lz[:, iz]
    return out


def lagrange_3d_normal(lo, hi, m, x: np.ndarray, nrm: np.ndarray) -> np.ndarray:
    """grad l_{t,nu}(x_p) . n_p as a (#x x m^3) matrix."""
    L = [lagrange_1d(cheb_nodes_1d(lo[a], hi[a], m), x[:, a]) for a in range(3)]
    D = [lagrange_1d_deriv(cheb_nodes_1d(lo[a], hi[a], m), x[:, a]) for a in range(3)]
    out = np.empty((x.shape[0], m ** 3))
    for iz in range(m):
        for iy in range(m):
            for ix in range(m):
                out[:, ix + m * iy + m * m * iz] = (D[0][:, ix] * L[1][:, iy] * L[2][:, iz] * nrm[:, 0]
                                                    + L[0][:, ix] * D[1][:, iy] * L[2][:, iz] * nrm[:, 1]
                                                    + L[0][:, ix] * L[1][:, iy] * D[2][:, iz] * nrm[:, 2])
    return out


def interp_basis(tree: ClusterTree, points: np.ndarray, m: int) -> Basis:
    """v_{t,i nu} = l_{t,nu}(x_i) on leaves, e_{t',nu' nu} = l_{t,nu}(xi_{t',nu'})."""
    k = m ** 3
    leaf, transfer = {}, {}
    for t in range(tree.nclusters):
        if tree.is_leaf(t):
            leaf[t] = lagrange_3d(tree.lo[t], tree.hi[t], m, points[tree.indices(t)])
        p = tree.parent[t]
        if p >= 0:
            transfer[t] = lagrange_3d(tree.lo[p], tree.hi[p], m, box_nodes(tree.lo[t], tree.hi[t], m))
    return Basis(tree, {t: k for t in range(tree.nclusters)}, leaf, transfer)


# Reading: the interpolation boxes of the double-layer operator.  Clusters of a
# surface are flat (a cube face has zero extent along its normal), and the normal
# derivative of an interpolant across a vanishing extent is ill-conditioned, so
# each box extent is widened symmetrically to at least DLP_FAT times the box's
# largest extent.  Admissibility keeps the bounding boxes.
DLP_FAT = 0.25


def fat_boxes(tree: ClusterTree, rho: float = DLP_FAT):
    """Bounding boxes with every extent widened to >= rho * (largest extent)."""
    lo, hi = [], []
    for t in range(tree.nclusters):
        l, h = np.array(tree.lo[t], dtype=np.float64), np.array(tree.hi[t], dtype=np.float64)
        need = rho * float((h - l).max())
        for a in range(3):
            if h[a] - l[a] < need:
                c = 0.5 * (l[a] + h[a])
                l[a], h[a] = c - 0.5 * need, c + 0.5 * need
        lo.append(l)
        hi.append(h)
    return lo, hi


def interp_basis_boxes(tree: ClusterTree, points: np.ndarray, m: int, lo, hi, normals=None) -> Basis:
    """interp_basis on the given boxes; with normals the leaf entries are
    d/dn(y_j) l_{s,mu}(y_j) (the transfers are the Lagrange ones: differentiation is
    linear and interpolation reproduces the parent's polynomials exactly)."""
    k = m ** 3
    leaf, transfer = {}, {}
    for t in range(tree.nclusters):
        if tree.is_leaf(t):
            idx = tree.indices(t)
            leaf[t] = (lagrange_3d(lo[t], hi[t], m, points[idx]) if normals is None
                       else lagrange_3d_normal(lo[t], hi[t], m, points[idx], normals[idx]))
        p = tree.parent[t]
        if p >= 0:
            transfer[t] = lagrange_3d(lo[p], hi[p], m, box_nodes(lo[t], hi[t], m))
    return Basis(tree, {t: k for t in range(tree.nclusters)}, leaf, transfer)


@dataclass
class Structure:
    """Points, cluster tree and block tree shared by all matrices of a product."""
    points: np.ndarray
    tree: ClusterTree
    blocks: BlockTree
    leaf: int
    eta: float
    order: int


def build_structure(points: np.ndarray, leaf: int, eta: float, order: int) -> Structure:
    tree = build_cluster_tree(points, leaf)
    return Structure(points, tree, build_block_tree(tree, tree, eta), leaf, eta, order)


def build_interp(st: Structure, kernel: int) -> H2Matrix:
    """H^2-matrix of g(x_i, x_j) by tensor Chebyshev interpolation of order m
    (rank m^3): S_ts = g(xi_t, xi_s), dense N_ts = g(x_i, x_j)."""
    tree, m = st.tree, st.order
    V = interp_basis(tree, st.points, m)
    S, N = {}, {}
    for (t, s), k in st.blocks.kind.items():
        if k == ADM:
            S[(t, s)] = kernel_matrix(kernel, box_nodes(tree.lo[t], tree.hi[t], m),
                                      box_nodes(tree.lo[s], tree.hi[s], m))
        elif k == DENSE:
            N[(t, s)] = kernel_matrix(kernel, st.points[tree.indices(t)], st.points[tree.indices(s)])
    return H2Matrix(st.blocks, V, V, S, N)


def build_interp_dlp(st: Structure, normals: np.ndarray) -> H2Matrix:
    """H^2-matrix of the double-layer potential: interpolate 1 / (4 pi |x - y|) in
    both variables on the widened boxes (fat_boxes) and take the normal derivative
    in y, so that V is the Lagrange basis, W the normal-derivative basis and
    S_ts = 1 / (4 pi |xi_t,nu - xi_s,mu|); dense N_ts = <n(x_j), x_i - x_j> /
    (4 pi |x_i - x_j|^3)."""
    tree, m = st.tree, st.order
    lo, hi = fat_boxes(tree)
    V = interp_basis_boxes(tree, st.points, m, lo, hi)
    W = interp_basis_boxes(tree, st.points, m, lo, hi, normals)
    S, N = {}, {}
    for (t, s), k in st.blocks.kind.items():
        if k == ADM:
            S[(t, s)] = kernel_matrix(K_LAPLACE, box_nodes(lo[t], hi[t], m), box_nodes(lo[s], hi[s], m))
        elif k == DENSE:
            js = tree.indices(s)
            N[(t, s)] = dlp_matrix(st.points[tree.indices(t)], st.points[js], normals[js])
    return H2Matrix(st.blocks, V, W, S, N)


# --------------------------------------------------------------------------
# Small helpers: QR, SVD, rank choice, block norms
# --------------------------------------------------------------------------

def qr_r(A: np.ndarray, ncols: int) -> np.ndarray:
    """R factor of a thin Householder QR, min(rows, cols) x cols; 0 x cols if
    A has no rows."""
    if A.shape[0] == 0:
        return np.zeros((0, ncols))
    return np.linalg.qr(A, mode="r")


def spectral_norm(A: np.ndarray) -> float:
    if A.size == 0:
        return 0.0
    return float(np.linalg.norm(A, 2))


def choose_rank(sigma: np.ndarray, eps: float) -> int:
    """Reading of "choose a rank": on the block-scaled matrix keep every
    singular value sigma_i > eps (eps = 0 keeps all positive ones)."""
    return int(np.count_nonzero(sigma > eps))


def left_singular(M: np.ndarray, eps: float) -> np.ndarray:
    """Leading left singular vectors of M with sigma > eps, as a matrix with
    M.shape[0] rows."""
    if M.shape[0] == 0 or M.shape[1] == 0:
        return np.zeros((M.shape[0], 0))
    U, sig, _ = np.linalg.svd(M, full_matrices=False)
    return U[:, :choose_rank(sig, eps)]


def hstack0(blocks, nrows):
    return np.hstack(blocks) if blocks else np.zeros((nrows, 0))


def vstack0(blocks, ncols):
    return np.vstack(blocks) if blocks else np.zeros((0, ncols))


# --------------------------------------------------------------------------
# Sec. 4: basis products, basis weights, total weights
# --------------------------------------------------------------------------

def basis_products(WX: Basis, VY: Basis) -> dict:
    """P_{XY,s} = W_{X,s}^* V_{Y,s} (Sec. 4, "cluster basis products"):
    directly in leaves, Sum_{s'} F_{X,s'}^* P_{s'} E_{Y,s'} in parents."""
    tree = WX.tree
    P = {}

    def rec(s):
        if tree.is_leaf(s):
            P[s] = WX.leaf[s].T @ VY.leaf[s]
        else:
            acc = np.zeros((WX.rank[s], VY.rank[s]))
            for c in tree.children[s]:
                rec(c)
                acc += WX.transfer[c].T @ P[c] @ VY.transfer[c]
            P[s] = acc

    rec(0)
    return P


def basis_weights(W: Basis) -> dict:
    """Fig. 1: R_r with W_r = Q_r R_r, Q_r isometric.  Leaves: thin QR of W_r;
    parents: thin QR of the stacked R_{r'} F_{r'} (Reading: R F as in the
    derivation under Fig. 1, not R F^*)."""
    tree = W.tree
    R = {}

    def rec(r):
        if tree.is_leaf(r):
            R[r] = qr_r(W.leaf[r], W.rank[r])
        else:
            for c in tree.children[r]:
                rec(c)
            R[r] = qr_r(vstack0([R[c] @ W.transfer[c] for c in tree.children[r]], W.rank[r]), W.rank[r])

    rec(0)
    return R


def total_weights(Y: H2Matrix, RW: dict) -> dict:
    """Fig. 2 with the block scaling of Sec. 5: top-down thin QR of
    [Z_{s+} E_{Y,s}^*; R_{Y,r} S_{Y,sr}^* / ||S_{Y,sr} R_{Y,r}^*||_2 ...] over
    the admissible leaves (s, r) (Reading: the garbled "Y_{Y,sr}" of Fig. 2 is
    S_{Y,sr}).  Blocks of norm 0 are left out."""
    tree = Y.rows
    rowb = Y.blocks.row_blocks()
    Zt = {}

    def rec(s, Zp):
        k = Y.V.rank[s]
        rows = []
        if Zp is not None:
            rows.append(Zp @ Y.V.transfer[s].T)
        for r in rowb[s]:
            if Y.blocks.kind[(s, r)] == ADM:
                SR = Y.S[(s, r)] @ RW[r].T
                nrm = spectral_norm(SR)
                if nrm > TINY:
                    rows.append(SR.T / nrm)
        Zt[s] = qr_r(vstack0(rows, k), k)
        for c in tree.children[s]:
            rec(c, Zt[s])

    rec(0, None)
    return Zt


# --------------------------------------------------------------------------
# Sec. 4 / Fig. 4: compressed induced row basis
# --------------------------------------------------------------------------

@dataclass
class InducedRows:
    Q: Basis     # compressed induced row basis (isometric, nested)
    Rbar: dict   # t -> Q_t^* V_{X,t}  (= [R_{X,t}; 0])
    A: dict      # (t, s), s in C_t -> Q_t^* X|_{t x s} V_{Y,s}
    RbarZ: dict = None  # t -> Q_t^* V_{Z,t} when Z's row basis is preserved as well


def same_basis(A: Basis, B: Basis) -> bool:
    """Equal nested bases (ranks, leaf and transfer matrices)."""
    if A is B:
        return True
    if A.rank != B.rank or set(A.leaf) != set(B.leaf) or set(A.transfer) != set(B.transfer):
        return False
    return (all(np.array_equal(A.leaf[t], B.leaf[t]) for t in A.leaf)
            and all(np.array_equal(A.transfer[t], B.transfer[t]) for t in A.transfer))


def induced_rows(X: H2Matrix, Y: H2Matrix, eps: float, VZ: Basis | None = None) -> InducedRows:
    """Fig. 4: compressed induced row basis of XY, preserving range(V_X).
    Reading of "+Z" with Z's own row basis: V_Z is preserved with V_X, the
    preserved block of Eq. (induced_Vtilde) becoming [V_X,t | V_Z,t] (and
    [Rbar_X E_X | Rbar_Z E_Z] above the leaves), so that Z's couplings are
    representable in the new basis through Rbar_Z = Q_t^* V_Z,t."""
    tree = X.rows
    PXY = basis_products(X.W, Y.V)
    RW = basis_weights(Y.W)
    Zt = total_weights(Y, RW)
    rowb = X.blocks.row_blocks()
    C = {t: [s for s in rowb[t] if X.blocks.kind[(t, s)] != ADM] for t in rowb}
    rank, leafm, transfer, Rbar, A, RbarZ = {}, {}, {}, {}, {}, {}

    def compress(VX, blocks):
        """QR of the preserved block, SVD of the remainder (Eq. induced_Vtilde);
        returns the isometric basis matrix and k1."""
        nrow, kx = VX.shape
        k1 = min(nrow, kx)
        QX = np.linalg.qr(VX, mode="complete")[0] if nrow else np.zeros((0, 0))
        M2 = (QX.T @ hstack0(blocks, nrow))[k1:]
        U = left_singular(M2, eps)
        return np.hstack([QX[:, :k1], QX[:, k1:] @ U])

    def rec(t):
        if tree.is_leaf(t):
            VX = X.V.leaf[t]
            VZt = VZ.leaf[t] if VZ is not None else None
            XV = {s: X.N[(t, s)] @ Y.V.leaf[s] for s in C[t]}
            blocks = []
            for s in C[t]:
                nrm = spectral_norm(XV[s])
                if nrm > TINY:
                    blocks.append(XV[s] @ Zt[s].T / nrm)  # Eq. induced_V, Sec. 5 scaling
            Qt = compress(VX if VZt is None else np.hstack([VX, VZt]), blocks)
            leafm[t] = Qt
            rank[t] = Qt.shape[1]
            for s in C[t]:
                A[(t, s)] = Qt.T @ XV[s]
            Rbar[t] = Qt.T @ VX
            if VZt is not None:
                RbarZ[t] = Qt.T @ VZt
        else:
            ch = tree.children[t]
            for c in ch:
                rec(c)
            VXh = np.vstack([Rbar[c] @ X.V.transfer[c] for c in ch])
            VZh = np.vstack([RbarZ[c] @ VZ.transfer[c] for c in ch]) if VZ is not None else None
            Ahat = {}
            for s in C[t]:
                rows = []
                for a in ch:
                    acc = np.zeros((rank[a], Y.V.rank[s]))
                    for b in X.cols.children[s]:
                        if X.blocks.kind[(a, b)] == ADM:
                            Aab = Rbar[a] @ X.S[(a, b)] @ PXY[b]
                        else:
                            Aab = A[(a, b)]
                        acc += Aab @ Y.V.transfer[b]
                    rows.append(acc)
                Ahat[s] = np.vstack(rows)  # Eq. induced_Ahat
            blocks = []
            for s in C[t]:
                nrm = spectral_norm(Ahat[s])
                if nrm > TINY:
                    blocks.append(Ahat[s] @ Zt[s].T / nrm)  # Eq. induced_Vhat, Sec. 5
            Qh = compress(VXh if VZh is None else np.hstack([VXh, VZh]), blocks)
            rank[t] = Qh.shape[1]
            o = 0
            for c in ch:  # Eq. compression_nonleaf: split rows into transfers
                transfer[c] = Qh[o:o + rank[c]]
                o += rank[c]
            for s in C[t]:
                A[(t, s)] = Qh.T @ Ahat[s]
            Rbar[t] = Qh.T @ VXh
            if VZh is not None:
                RbarZ[t] = Qh.T @ VZh

    rec(0)
    return InducedRows(Basis(tree, rank, leafm, transfer), Rbar, A, RbarZ if VZ is not None else None)


# --------------------------------------------------------------------------
# Sec. 6: product block tree T^XY and the intermediate H^2-matrix ("t_mat")
# --------------------------------------------------------------------------

@dataclass
class ProductTree:
    """Product block tree T^XY: kind[(t,r)] in {adm, dense, split}; triples[(t,r)]
    lists the s with (t,s) in T_IJ, (s,r) in T_JK that are not both split."""
    kind: dict
    children: dict
    triples: dict


def build_product_tree(X: H2Matrix, Y: H2Matrix) -> ProductTree:
    """Minimal block tree in which (t,r) is split iff some s has (t,s) and (s,r)
    both non-leaf; a leaf is admissible iff for every s one factor is an
    admissible leaf (Sec. 6, first paragraphs).  Reading: children are
    chil(t) x chil(r) as in Def. "Block tree"."""
    xrow = X.blocks.row_blocks()
    kind, children, triples = {}, {}, {}

    def rec(t, r):
        ss = [s for s in xrow[t] if (s, r) in Y.blocks.kind]
        split = any(X.blocks.kind[(t, s)] == SPLIT and Y.blocks.kind[(s, r)] == SPLIT for s in ss)
        triples[(t, r)] = [s for s in ss if not (X.blocks.kind[(t, s)] == SPLIT and Y.blocks.kind[(s, r)] == SPLIT)]
        if split:
            kind[(t, r)] = SPLIT
            children[(t, r)] = [(a, b) for a in X.rows.children[t] for b in Y.cols.children[r]]
            for a, b in children[(t, r)]:
                rec(a, b)
        else:
            adm = all(X.blocks.kind[(t, s)] == ADM or Y.blocks.kind[(s, r)] == ADM for s in ss)
            kind[(t, r)] = ADM if adm else DENSE

    rec(0, 0)
    return ProductTree(kind, children, triples)


def leaf_block(M: H2Matrix, t: int, s: int) -> np.ndarray:
    """M|_{t x s} for a leaf block (t, s) of M, as a dense matrix."""
    if M.blocks.kind[(t, s)] == DENSE:
        return M.N[(t, s)]
    return M.V.expand(t) @ M.S[(t, s)] @ M.W.expand(s).T


def induced_matrix(X: H2Matrix, Y: H2Matrix, Z: H2Matrix, rowsA: InducedRows, colsA: InducedRows,
                   PT: ProductTree) -> H2Matrix:
    """The product (plus Z) as an H^2-matrix on T^XY in the compressed induced
    bases ("t_mat", Sec. 7).  Reading: every triple (t,s,r) at a node adds its
    projection Q_t^* X_ts Y_sr Q^W_r, namely
        (t,s),(s,r) admissible:  Rbar_t S_X,ts P_s S_Y,sr Rbar^W_r^*
        (t,s) not admissible:    A_ts S_Y,sr Rbar^W_r^*           (Eq. semiuniform)
        (s,r) not admissible:    Rbar_t S_X,ts B_rs^*             (Eq. semiuniform2)
    and couplings of split nodes are moved to the leaves with the new transfer
    matrices.  Dense leaves of T^XY hold the exact leaf-level products plus the
    expansion of what the ancestors pushed down.  Reading of "+Z": Z's row and
    column bases are X's row and Y's column bases, so S_Z enters the node
    (t,r) as Rbar_t S_Z Rbar^W_r^* and N_Z enters the dense leaf; with bases of
    its own, V_Z and W_Z were preserved in phase A and S_Z enters as
    Rbar_Z,t S_Z Rbar^W_Z,r^*."""
    Q, QW = rowsA.Q, colsA.Q
    PXY = basis_products(X.W, Y.V)
    C = {}
    for (t, r), k in PT.kind.items():
        if k == DENSE:
            continue
        acc = np.zeros((Q.rank[t], QW.rank[r]))
        for s in PT.triples[(t, r)]:
            kx, ky = X.blocks.kind[(t, s)], Y.blocks.kind[(s, r)]
            if kx == ADM and ky == ADM:
                acc += rowsA.Rbar[t] @ X.S[(t, s)] @ PXY[s] @ Y.S[(s, r)] @ colsA.Rbar[r].T
            elif ky == ADM:
                acc += rowsA.A[(t, s)] @ Y.S[(s, r)] @ colsA.Rbar[r].T
            elif kx == ADM:
                acc += rowsA.Rbar[t] @ X.S[(t, s)] @ colsA.A[(r, s)].T
            else:
                raise AssertionError("two inadmissible leaves outside a dense T^XY leaf")
        if Z.blocks.kind.get((t, r)) == ADM:
            RZ = rowsA.Rbar if rowsA.RbarZ is None else rowsA.RbarZ
            RWZ = colsA.Rbar if colsA.RbarZ is None else colsA.RbarZ
            acc += RZ[t] @ Z.S[(t, r)] @ RWZ[r].T
        C[(t, r)] = acc
    S, N = {}, {}

    def push(t, r, up):
        """up: coupling pushed down from the ancestors, in Q_t / QW_r."""
        k = PT.kind[(t, r)]
        if k == DENSE:
            D = np.zeros((X.rows.size[t], Y.cols.size[r]))
            for s in PT.triples[(t, r)]:
                D += leaf_block(X, t, s) @ leaf_block(Y, s, r)
            zk = Z.blocks.kind.get((t, r))
            if zk is not None:
                D += leaf_block(Z, t, r)
            if up is not None:
                D += Q.leaf[t] @ up @ QW.leaf[r].T
            N[(t, r)] = D
            return
        cur = C[(t, r)] if up is None else C[(t, r)] + up
        if k == ADM:
            S[(t, r)] = cur
        else:
            for a, b in PT.children[(t, r)]:
                push(a, b, Q.transfer[a] @ cur @ QW.transfer[b].T)

    push(0, 0, None)
    bt = BlockTree(X.rows, Y.cols, dict(PT.kind), dict(PT.children))
    return H2Matrix(bt, Q, QW, S, N)


def check_refinement(G: H2Matrix, coarse: BlockTree):
    """Reading: T^XY refines T_IK (every node of T_IK is a node of T^XY, every
    dense leaf of T_IK is a dense leaf of T^XY)."""
    for b, k in coarse.kind.items():
        if b not in G.blocks.kind:
            raise ValueError(f"T^XY does not refine the target block tree at {b}")
        if k == DENSE and G.blocks.kind[b] != DENSE:
            raise ValueError(f"dense target block {b} is not a dense leaf of T^XY")


# --------------------------------------------------------------------------
# Sec. 6: coarsening (build_basis, Fig. 7) with column trees (Fig. 6)
# --------------------------------------------------------------------------

@dataclass
class CoarseRows:
    Q: Basis    # new adaptive isometric row basis for T_IK
    R: dict     # t -> Q'_t^* Q_t  (basis change from the induced basis)


def coarse_map(G: H2Matrix, coarse: BlockTree) -> dict:
    """(t,r) in T^XY -> the admissible leaf of T_IK that contains it, if any."""
    out = {}

    def rec(t, r, b):
        if b is None and coarse.kind.get((t, r)) == ADM:
            b = (t, r)
        if b is not None:
            out[(t, r)] = b
        for a, c in G.blocks.children.get((t, r), []):
            rec(a, c, b)

    rec(0, 0, None)
    return out


def block_weights(G: H2Matrix, cmap: dict) -> dict:
    """Reading of the block-relative control of the second phase: every part of
    the admissible target block b is scaled by 1/||G|_b||_F, the norm taken
    exactly over the T^XY leaves inside b (isometric bases)."""
    sq = {}
    for (t, r), b in cmap.items():
        k = G.blocks.kind[(t, r)]
        if k == ADM:
            sq[b] = sq.get(b, 0.0) + float((G.S[(t, r)] ** 2).sum())
        elif k == DENSE:
            sq[b] = sq.get(b, 0.0) + float((G.N[(t, r)] ** 2).sum())
    return {b: (1.0 / math.sqrt(v) if v > 0.0 else 0.0) for b, v in sq.items()}


def coarsen_rows(G: H2Matrix, coarse: BlockTree, eps: float) -> CoarseRows:
    """Fig. 7 (build_basis) for the row basis of the coarse block tree."""
    tree, QI, QW = G.rows, G.V, G.W
    cmap = coarse_map(G, coarse)
    wb = block_weights(G, cmap)
    rowb = G.blocks.row_blocks()
    rank, leafm, transfer, R = {}, {}, {}, {}
    A = {}  # (t, r) -> {rho: matrix}: Q'_t^* G|_{t x r} per column-tree leaf rho
    Zt = {}

    def total(t, Zp):
        """Eq. Zt_condensation (Reading: the last block is S_{t,r_m}^*)."""
        rows = [] if Zp is None else [Zp @ QI.transfer[t].T]
        for r in rowb[t]:
            if G.blocks.kind[(t, r)] == ADM:
                rows.append(wb[cmap[(t, r)]] * G.S[(t, r)].T)
        Zt[t] = qr_r(vstack0(rows, QI.rank[t]), QI.rank[t])
        for c in tree.children[t]:
            total(c, Zt[t])

    total(0, None)

    def col_leaves(r, rep):
        """Leaves of the column tree T_(t,r) of a representation, in order."""
        return sorted(rep.keys(), key=lambda c: G.cols.off[c])

    def match(rep: dict, target: dict) -> dict:
        """Fig. 6, match_column: extend a representation {rho: (adm, M)} to the
        finer target partition {rho: adm}.  Admissible leaves split with F^*,
        admissible leaves that are inadmissible in the target expand with W^*."""
        out = {}

        def rec(c, adm, M):
            if c in target:
                if adm and not target[c]:
                    out[c] = (False, M @ QW.leaf[c].T)
                else:
                    out[c] = (adm, M)
                return
            assert adm, "an inadmissible column leaf cannot be split"
            for cc in G.cols.children[c]:
                rec(cc, True, M @ QW.transfer[cc].T)

        for c, (adm, M) in rep.items():
            rec(c, adm, M)
        return out

    def child_rep(a, b):
        """Representation of Q'_a^* G|_{a x b} for a child block (a, b)."""
        k = G.blocks.kind[(a, b)]
        if k == ADM:
            return {b: (True, R[a] @ G.S[(a, b)])}
        return A[(a, b)]

    def build(t):
        if tree.is_leaf(t):
            dense = [r for r in rowb[t] if G.blocks.kind[(t, r)] == DENSE and (t, r) in cmap]
            Ct = hstack0([QI.leaf[t] @ Zt[t].T] + [wb[cmap[(t, r)]] * G.N[(t, r)] for r in dense],
                         tree.size[t])  # Eq. ct_leaf
            Qt = left_singular(Ct, eps)
            leafm[t] = Qt
            rank[t] = Qt.shape[1]
            R[t] = Qt.T @ QI.leaf[t]
            for r in dense:
                A[(t, r)] = {r: (False, Qt.T @ G.N[(t, r)])}
            return
        ch = tree.children[t]
        for c in ch:
            build(c)
        Vh = np.vstack([R[c] @ QI.transfer[c] for c in ch])
        split = [r for r in rowb[t] if G.blocks.kind[(t, r)] == SPLIT and (t, r) in cmap]
        Ahat = {}
        for r in split:
            reps = {a: {} for a in ch}
            for a in ch:
                for b in G.cols.children[r]:
                    reps[a].update(child_rep(a, b))
            target = {}
            for a in ch:  # union of the children's column trees: finest partition
                for c, (adm, _) in reps[a].items():
                    target[c] = target.get(c, True) and adm
            # drop clusters that have a descendant in the target (keep the leaves)
            leaves = {c: adm for c, adm in target.items()
                      if not any(d != c and _is_ancestor(G.cols, c, d) for d in target)}
            rowsb = []
            for a in ch:
                mrep = match(reps[a], leaves)
                rowsb.append([mrep[c][1] for c in col_leaves(r, leaves)])
            order = col_leaves(r, leaves)
            Ahat[r] = (order, [leaves[c] for c in order],
                       [np.vstack([rowsb[i][j] for i in range(len(ch))]) for j in range(len(order))])
        blocks = [Vh @ Zt[t].T]
        for r in split:
            w = wb[cmap[(t, r)]]
            blocks += [w * M for M in Ahat[r][2]]  # Eq. ct_nonleaf
        Qh = left_singular(hstack0(blocks, Vh.shape[0]), eps)
        rank[t] = Qh.shape[1]
        o = 0
        for c in ch:
            transfer[c] = Qh[o:o + rank[c]]
            o += rank[c]
        R[t] = Qh.T @ Vh
        for r in split:
            order, adms, mats = Ahat[r]
            A[(t, r)] = {c: (adm, Qh.T @ M) for c, adm, M in zip(order, adms, mats)}

    build(0)
    return CoarseRows(Basis(tree, rank, leafm, transfer), R)


def _is_ancestor(tree: ClusterTree, a: int, d: int) -> bool:
    while d >= 0:
        if d == a:
            return True
        d = tree.parent[d]
    return False


def final_matrix(G: H2Matrix, coarse: BlockTree, rowsB: CoarseRows, colsB: CoarseRows) -> H2Matrix:
    """The result on T_IK in the new bases ("t_mat" of the final phase):
    S'_tr = Q'_t^* G|_{t x r} Q'^W_r by upward accumulation over the T^XY
    subtree of every admissible target leaf; dense target leaves are the dense
    leaves of T^XY."""
    Qn, Wn = rowsB.Q, colsB.Q

    def up(t, r):
        k = G.blocks.kind[(t, r)]
        if k == ADM:
            return rowsB.R[t] @ G.S[(t, r)] @ colsB.R[r].T
        if k == DENSE:
            return Qn.leaf[t].T @ G.N[(t, r)] @ Wn.leaf[r]
        acc = np.zeros((Qn.rank[t], Wn.rank[r]))
        for a, b in G.blocks.children[(t, r)]:
            acc += Qn.transfer[a].T @ up(a, b) @ Wn.transfer[b]
        return acc

    S, N = {}, {}
    for b, k in coarse.kind.items():
        if k == ADM:
            S[b] = up(*b)
        elif k == DENSE:
            N[b] = G.N[b]
    return H2Matrix(coarse, Qn, Wn, S, N)


# --------------------------------------------------------------------------
# The whole product
# --------------------------------------------------------------------------

@dataclass
class ProductResult:
    result: H2Matrix        # final H^2-matrix on T_IK (Z + XY)
    induced: H2Matrix       # intermediate H^2-matrix on T^XY (phase A)
    rowsA: InducedRows
    colsA: InducedRows
    rowsB: CoarseRows
    colsB: CoarseRows
    product_tree: ProductTree


def mul_add(Z: H2Matrix, X: H2Matrix, Y: H2Matrix, eps: float, eps_induced: float | None = None) -> ProductResult:
    """Z + X Y: compressed induced bases (Sec. 4-5), the H^2-matrix on T^XY,
    coarsening to Z's block tree (Sec. 6).  Reading: both phases use the same
    tolerance unless eps_induced is given (Sec. 7 uses 1e-4 for both).  The
    structures of X, Y and Z must share one cluster tree; when Z's row (column)
    basis differs from X's row (Y's column) basis it is preserved as well."""
    epsA = eps if eps_induced is None else eps_induced
    VZ = None if same_basis(Z.V, X.V) else Z.V
    WZ = None if same_basis(Z.W, Y.W) else Z.W
    rowsA = induced_rows(X, Y, epsA, VZ)
    colsA = induced_rows(Y.transpose(), X.transpose(), epsA, WZ)
    PT = build_product_tree(X, Y)
    G = induced_matrix(X, Y, Z, rowsA, colsA, PT)
    check_refinement(G, Z.blocks)
    rowsB = coarsen_rows(G, Z.blocks, eps)
    colsB = coarsen_rows(G.transpose(), Z.blocks.transpose(), eps)
    F = final_matrix(G, Z.blocks, rowsB, colsB)
    return ProductResult(F, G, rowsA, colsA, rowsB, colsB, PT)


# --------------------------------------------------------------------------
# Sec. 7: the relative spectral error eps_2 of a computed product
# --------------------------------------------------------------------------

def power_norm(apply, apply_t, x0: np.ndarray, steps: int) -> float:
    """Spectral norm of an operator A by power iteration on A^* A (Sec. 7 uses
    20 steps): x is normalised, the estimate is ||A x||, then x <- A^* A x.
    Returns the estimate of the last step (a lower bound of ||A||_2)."""
    x = np.array(x0, dtype=np.float64)
    nx = float(np.linalg.norm(x))
    est = 0.0
    for _ in range(steps):
        if nx == 0.0:
            break
        x = x / nx
        y = apply(x)
        est = float(np.linalg.norm(y))
        if est == 0.0:
            break
        x = apply_t(y)
        nx = float(np.linalg.norm(x))
    return est


def spectral_error(Dr: np.ndarray, D0: np.ndarray, DX: np.ndarray, DY: np.ndarray, x0: np.ndarray,
                   steps: int = 20) -> tuple[float, float]:
    """(eps_2, ||P||_2) with P = D0 + DX DY the exact product and eps_2 =
    ||Dr - P||_2 / ||P||_2, both norms by power_norm from the same start vector
    (Sec. 7).  P is applied as D0 x + DX (DY x), never formed."""
    P = lambda x: D0 @ x + DX @ (DY @ x)
    Pt = lambda y: D0.T @ y + DY.T @ (DX.T @ y)
    p = power_norm(P, Pt, x0, steps)
    e = power_norm(lambda x: Dr @ x - P(x), lambda y: Dr.T @ y - Pt(y), x0, steps)
    return (e / p if p > 0.0 else 0.0), p


# --------------------------------------------------------------------------
# Recompression of an input H^2-matrix (Fig. 1 with the isometric factors, Fig. 7)
# --------------------------------------------------------------------------

def orthogonalize(B: Basis):
    """B_t = Q_t R_t with Q nested and isometric (Fig. 1, keeping the Q factors):
    leaves by a thin QR of B_t, parents by a thin QR of the stacked R_{t'} E_{t'};
    the rows of that Q-hat split into the children's transfer matrices.
    Returns (Q, R) with R[t] of size rank_Q(t) x rank_B(t)."""
    tree = B.tree
    leaf, transfer, rank, R = {}, {}, {}, {}

    def rec(t):
        if tree.is_leaf(t):
            q, r = np.linalg.qr(B.leaf[t])
            leaf[t], R[t], rank[t] = q, r, q.shape[1]
            return
        ch = tree.children[t]
        for c in ch:
            rec(c)
        q, r = np.linalg.qr(np.vstack([R[c] @ B.transfer[c] for c in ch]))
        R[t], rank[t] = r, q.shape[1]
        o = 0
        for c in ch:
            transfer[c] = q[o:o + rank[c]]
            o += rank[c]

    rec(0)
    return Basis(tree, rank, leaf, transfer), R


def recompress(A: H2Matrix, eps: float) -> H2Matrix:
    """Adaptive isometric bases for an input H^2-matrix: orthogonalize both bases,
    move the couplings into them (S' = R_V S R_W^*), then coarsen with the
    matrix's own block tree as the tree of the intermediate matrix (Fig. 7) and
    project (the final couplings of Sec. 6); the block-relative tolerance eps
    is that of the product's second phase."""
    QV, RV = orthogonalize(A.V)
    QW, RW = (QV, RV) if A.W is A.V else orthogonalize(A.W)
    S = {(t, s): RV[t] @ m @ RW[s].T for (t, s), m in A.S.items()}
    G = H2Matrix(A.blocks, QV, QW, S, dict(A.N))
    rowsB = coarsen_rows(G, A.blocks, eps)
    colsB = coarsen_rows(G.transpose(), A.blocks.transpose(), eps)
    return final_matrix(G, A.blocks, rowsB, colsB)
