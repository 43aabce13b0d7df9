// Host planner: cluster tree, block tree and product block tree (Sec. 2, Sec. 6).
// Integer and comparison work only; no product arithmetic happens here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "h2_internal.h"

namespace h2 {

void BlockTree::finish() {
    by_row.assign(nc, {});
    by_col.assign(nc, {});
    for (int i = 0; i < (int)t.size(); ++i) {
        by_row[t[i]].push_back(i);
        by_col[s[i]].push_back(i);
    }
    for (auto& v : by_row) std::sort(v.begin(), v.end(), [&](int a, int b) { return s[a] < s[b]; });
    for (auto& v : by_col) std::sort(v.begin(), v.end(), [&](int a, int b) { return t[a] < t[b]; });
    kids.assign(t.size(), std::array<int, 4>{-1, -1, -1, -1});
    for (size_t b = 0; b < t.size(); ++b)
        if (kind[b] == SPLIT)
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) kids[b][2 * i + j] = find(Tree::child(t[b], i), Tree::child(s[b], j));
}

// Depth L: the smallest depth with ceil(n / 2^L) <= leaf, so that every
// cluster above it splits and all leaves share level L.
static int tree_depth(int64_t n, int leaf) {
    int L = 0;
    while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf) ++L;
    return L;
}

static void box_of(const double* pts, const int64_t* idx, int64_t cnt, double pad, double* lo, double* hi) {
    for (int a = 0; a < 3; ++a) {
        double mn = pts[3 * idx[0] + a], mx = mn;
        for (int64_t i = 1; i < cnt; ++i) {
            double v = pts[3 * idx[i] + a];
            mn = v < mn ? v : mn;
            mx = v > mx ? v : mx;
        }
        if (mx - mn < pad) {  // flat clusters: widen symmetrically
            double c = 0.5 * (mn + mx);
            mn = c - 0.5 * pad;
            mx = c + 0.5 * pad;
        }
        lo[a] = mn;
        hi[a] = mx;
    }
}

static double diam(const double* lo, const double* hi) {
    double d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
    return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

static double dist(const double* lo1, const double* hi1, const double* lo2, const double* hi2) {
    double g[3];
    for (int a = 0; a < 3; ++a) {
        double x = lo1[a] - hi2[a], y = lo2[a] - hi1[a];
        double m = x > y ? x : y;
        g[a] = m > 0.0 ? m : 0.0;
    }
    return std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

std::shared_ptr<Structure> build_structure(const double* pts, int64_t n, int leaf, double eta) {
    auto st = std::make_shared<Structure>();
    st->eta = eta;
    st->points.assign(pts, pts + 3 * n);
    Tree& T = st->tree;
    T.n = n;
    T.leaf_size = leaf;
    T.L = tree_depth(n, leaf);
    if (T.L > 24) throw Error(H2_ERR_ARG, "tree deeper than 24 levels");
    T.nc = (1 << (T.L + 1)) - 1;
    T.perm.resize(n);
    std::iota(T.perm.begin(), T.perm.end(), 0);
    T.off.assign(T.nc, 0);
    T.size.assign(T.nc, 0);
    T.lo.assign(3 * T.nc, 0.0);
    T.hi.assign(3 * T.nc, 0.0);
    double rext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double mn = pts[a], mx = pts[a];
        for (int64_t i = 1; i < n; ++i) {
            mn = std::min(mn, pts[3 * i + a]);
            mx = std::max(mx, pts[3 * i + a]);
        }
        rext = std::max(rext, mx - mn);
    }
    const double pad = 1e-8 * std::max(rext, 1e-300);
    T.off[0] = 0;
    T.size[0] = n;
    std::vector<int8_t> split_axis(T.nc, 0);
    for (int c = 0; c < T.nc; ++c) {
        int64_t* idx = T.perm.data() + T.off[c];
        int64_t cnt = T.size[c];
        box_of(pts, idx, cnt, pad, &T.lo[3 * c], &T.hi[3 * c]);
        if (T.is_leaf(c)) continue;
        // split along the longest raw extent (first maximum), stable in the index
        double ext[3];
        for (int a = 0; a < 3; ++a) {
            double mn = pts[3 * idx[0] + a], mx = mn;
            for (int64_t i = 1; i < cnt; ++i) {
                mn = std::min(mn, pts[3 * idx[i] + a]);
                mx = std::max(mx, pts[3 * idx[i] + a]);
            }
            ext[a] = mx - mn;
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (ext[a] > ext[axis]) axis = a;
        // the first cnt / 2 in (coordinate, index) order go to child 1: a selection,
        // not a sort (only the leaves' order is kept, and it is sorted below)
        int64_t h = cnt / 2;
        split_axis[c] = (int8_t)axis;
        std::nth_element(idx, idx + h, idx + cnt, [&](int64_t p, int64_t q) {
            double vp = pts[3 * p + axis], vq = pts[3 * q + axis];
            return vp < vq || (vp == vq && p < q);
        });
        int c1 = Tree::child(c, 0), c2 = Tree::child(c, 1);
        T.off[c1] = T.off[c];
        T.size[c1] = h;
        T.off[c2] = T.off[c] + h;
        T.size[c2] = cnt - h;
    }
    // a leaf keeps its points in its parent's split order: (coordinate along the
    // parent's split axis, index)
    if (T.L > 0)
        for (int c = Tree::first(T.L); c < T.nc; ++c) {
            int64_t* idx = T.perm.data() + T.off[c];
            const int axis = split_axis[Tree::parent(c)];
            std::sort(idx, idx + T.size[c], [&](int64_t p, int64_t q) {
                double vp = pts[3 * p + axis], vq = pts[3 * q + axis];
                return vp < vq || (vp == vq && p < q);
            });
        }
    for (int c = 0; c < T.nc; ++c)
        if (T.size[c] <= 0) throw Error(H2_ERR_ARG, "empty cluster: fewer points than leaves");
    // block tree with the standard admissibility condition
    BlockTree& B = st->blocks;
    B.nc = T.nc;
    std::vector<std::pair<int, int>> stack{{0, 0}};
    while (!stack.empty()) {
        auto [a, b] = stack.back();
        stack.pop_back();
        double dm = std::max(diam(&T.lo[3 * a], &T.hi[3 * a]), diam(&T.lo[3 * b], &T.hi[3 * b]));
        double ds = dist(&T.lo[3 * a], &T.hi[3 * a], &T.lo[3 * b], &T.hi[3 * b]);
        if (dm <= eta * ds) {
            B.add(a, b, ADM);
        } else if (T.is_leaf(a) || T.is_leaf(b)) {
            B.add(a, b, DENSE);
        } else {
            B.add(a, b, SPLIT);
            for (int i = 1; i >= 0; --i)
                for (int j = 1; j >= 0; --j) stack.push_back({Tree::child(a, i), Tree::child(b, j)});
        }
    }
    B.finish();
    // fingerprint of the structure (points, leaf, eta) for operand checks
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    mix((uint64_t)n);
    mix((uint64_t)leaf);
    uint64_t e;
    std::memcpy(&e, &eta, 8);
    mix(e);
    for (int64_t i = 0; i < 3 * n; ++i) {
        uint64_t v;
        std::memcpy(&v, &pts[i], 8);
        mix(v);
    }
    st->fingerprint = h;
    return st;
}

ProductTree build_product_tree(const BlockTree& X, const BlockTree& Y) {
    ProductTree P;
    P.nodes.nc = X.nc;
    std::vector<std::pair<int, int>> stack{{0, 0}};
    std::vector<int> ss;
    std::vector<std::pair<int, int>> bb;
    std::vector<std::pair<int8_t, int8_t>> kk;
    while (!stack.empty()) {
        auto [t, r] = stack.back();
        stack.pop_back();
        bool split = false;
        bool adm = true;
        ss.clear();
        bb.clear();
        kk.clear();
        for (int bx : X.by_row[t]) {
            int s = X.s[bx];
            int by = Y.find(s, r);
            if (by < 0) continue;
            int8_t kx = X.kind[bx], ky = Y.kind[by];
            if (kx == SPLIT && ky == SPLIT) {
                split = true;
            } else {
                ss.push_back(s);
                bb.push_back({bx, by});
                kk.push_back({kx, ky});
                if (kx != ADM && ky != ADM) adm = false;
            }
        }
        int id = P.nodes.add(t, r, split ? SPLIT : (adm ? ADM : DENSE));
        P.triples.push_back(ss);
        P.tri_blocks.push_back(bb);
        P.tri_kinds.push_back(kk);
        (void)id;
        if (split) {
            for (int i = 1; i >= 0; --i)
                for (int j = 1; j >= 0; --j) stack.push_back({Tree::child(t, i), Tree::child(r, j)});
        }
    }
    P.nodes.finish();
    return P;
}

}  // namespace h2
