// h2_mul_add: Z <- Z + X Y for H^2-matrices (S. Boerm, arXiv 2309.09061).
//
// The host walks the cluster tree level by level and, for each level, queues
// one batched launch per step covering every cluster and block of that level:
//   prep      cluster basis products (Sec. 4), basis weights (Fig. 1), total
//             weights with block scaling (Fig. 2, Sec. 5)
//   phase A   compressed induced row basis (Fig. 4), the column basis as the
//             same procedure on Y^* X^*, couplings on T^XY ("t_mat")
//   phase B   coarsening to Z's block tree (Fig. 7, Fig. 6), row basis and the
//             column basis on G^*, then the final couplings
// Ranks are chosen on the device; the host reads them back once per level to
// size the next level's buffers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <atomic>
#include <map>
#include <mutex>
#include <future>
#include <thread>

#include "h2_internal.h"

namespace h2 {

cudaStream_t stream_of(const h2_opts* o);

// A product thread of a batched call that blocks on the host (a stream
// synchronisation, a join) submits nothing meanwhile: the combiner does not
// wait for it.
struct CombIdle {
    Combiner* c;
    explicit CombIdle(Combiner* cc) : c(cc) {
        if (c) c->leave();
    }
    ~CombIdle() {
        if (c) c->enter();
    }
};

// A matrix operand as stored: logical = tr ? stored^T : stored.
struct Mv {
    const double* p;
    int ld;
    int tr;
};

// ------------------------------------------------------------------ views
// Logical view of an H^2-matrix, optionally transposed.
struct OpView {
    const h2_matrix* M;
    bool T;
    const Tree& tree() const { return M->st->tree; }
    const BlockTree& bt() const { return M->st->blocks; }
    const Basis& rowb() const { return T ? *M->W : *M->V; }
    const Basis& colb() const { return T ? *M->V : *M->W; }
    int block(int t, int s) const { return T ? bt().find(s, t) : bt().find(t, s); }
    // child (child(t, i), child(s, j)) of split block b in view coordinates
    int kid(int b, int i, int j) const { return T ? bt().kids[b][2 * j + i] : bt().kids[b][2 * i + j]; }
    int8_t kind(int b) const { return bt().kind[b]; }
    const std::vector<int>& row_list(int t) const { return T ? bt().by_col[t] : bt().by_row[t]; }
    int other(int b) const { return T ? bt().t[b] : bt().s[b]; }  // column cluster of block b in the view
    Mv S(int b) const {
        int ld = M->V->rank[bt().t[b]];
        return Mv{M->blk[b], ld, T ? 1 : 0};
    }
    Mv N(int b) const {
        int ld = (int)tree().size[bt().t[b]];
        return Mv{M->blk[b], ld, T ? 1 : 0};
    }
};

// Per-cluster device matrices with their shapes.
struct PerCl {
    std::vector<double*> p;
    std::vector<int> rows, cols;
    void init(int nc) {
        p.assign(nc, nullptr);
        rows.assign(nc, 0);
        cols.assign(nc, 0);
    }
};

// Map from small integer keys (nodes, blocks) to device pointers; clear() is
// proportional to the keys used since the last clear.
struct Slots {
    std::vector<double*> v;
    std::vector<int> used;
    explicit Slots(size_t n) : v(n, nullptr) {}
    double*& operator[](int k) {
        if (!v[k]) used.push_back(k);
        return v[k];
    }
    bool has(int k) const { return v[k] != nullptr; }
    void clear() {
        for (int k : used) v[k] = nullptr;
        used.clear();
    }
};

static void T_(Runner& R, Mv A, Mv B, int k, double alpha = 1.0, const double* scale = nullptr, int flipA = 0,
               int flipB = 0) {
    R.term(A.p, A.tr ^ flipA, A.ld, B.p, B.tr ^ flipB, B.ld, k, alpha, scale);
}

static Mv mv(const double* p, int ld) { return Mv{p, ld, 0}; }
static Mv mvT(const double* p, int ld) { return Mv{p, ld, 1}; }

// ------------------------------------------------------------------ timing / stats
struct PhaseClock {
    cudaStream_t st;
    std::vector<cudaEvent_t> ev;
    explicit PhaseClock(cudaStream_t s) : st(s) {}
    ~PhaseClock() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    void mark() {
        cudaEvent_t e;
        H2_CUDA(cudaEventCreate(&e));
        H2_CUDA(cudaEventRecord(e, st));
        ev.push_back(e);
    }
    double ms(int i) const {
        float f = 0;
        cudaEventElapsedTime(&f, ev[i], ev[i + 1]);
        return f;
    }
};

struct Counts {
    double flops = 0, bytes = 0;
    int64_t triples = 0;
};

// ------------------------------------------------------------------ prep: basis products
// P_s = W_{X,s}^* V_{Y,s}: directly in leaves, sum_{s'} F_{s'}^* P_{s'} E_{s'} above.
static PerCl basis_products(Runner& R, const Tree& T, const Basis& WX, const Basis& VY) {
    H2_SPAN("basis_products");
    PerCl P;
    P.init(T.nc);
    for (int c = 0; c < T.nc; ++c) {
        P.rows[c] = WX.rank[c];
        P.cols[c] = VY.rank[c];
        P.p[c] = R.dalloc((size_t)std::max(1, P.rows[c] * P.cols[c]));
    }
    for (int c = Tree::first(T.L); c < T.nc; ++c) {
        int sz = (int)T.size[c];
        R.job(P.p[c], P.rows[c], P.cols[c], std::max(1, P.rows[c]), 0.0);
        R.term(WX.leaf[c], 1, sz, VY.leaf[c], 0, sz, sz);
    }
    R.flush_gemm(H2_FP64);
    for (int l = T.L - 1; l >= 0; --l) {
        std::vector<double*> tmp(T.nc, nullptr);
        for (int c = Tree::first(l + 1); c < Tree::first(l + 1) + Tree::count(l + 1); ++c) {
            int p = Tree::parent(c);
            tmp[c] = R.dalloc((size_t)std::max(1, WX.rank[c] * VY.rank[p]));
            R.job(tmp[c], WX.rank[c], VY.rank[p], std::max(1, WX.rank[c]), 0.0);
            R.term(P.p[c], 0, std::max(1, P.rows[c]), VY.tr[c], 0, std::max(1, VY.rank[c]), VY.rank[c]);
        }
        R.flush_gemm(H2_FP64);
        for (int p = Tree::first(l); p < Tree::first(l) + Tree::count(l); ++p) {
            R.job(P.p[p], P.rows[p], P.cols[p], std::max(1, P.rows[p]), 0.0);
            for (int i = 0; i < 2; ++i) {
                int c = Tree::child(p, i);
                R.term(WX.tr[c], 1, std::max(1, WX.rank[c]), tmp[c], 0, std::max(1, WX.rank[c]), WX.rank[c]);
            }
        }
        R.flush_gemm(H2_FP64);
    }
    return P;
}

// ------------------------------------------------------------------ prep: basis weights (Fig. 1)
// R_r with W_r = Q_r R_r: QR of the leaf matrices, then QR of [R_{r1} F_{r1}; R_{r2} F_{r2}].
static PerCl basis_weights(Runner& R, const Tree& T, const Basis& B) {
    H2_SPAN("basis_weights");
    PerCl W;
    W.init(T.nc);
    for (int c = Tree::first(T.L); c < T.nc; ++c) {
        int m = (int)T.size[c], k = B.rank[c];
        double* work = R.dalloc((size_t)m * std::max(1, k));
        R.copy(B.leaf[c], m, work, m, m, k, 0);
        W.rows[c] = std::min(m, k);
        W.cols[c] = k;
        W.p[c] = R.dalloc((size_t)std::max(1, W.rows[c] * k));
        R.qr(work, m, k, m, W.p[c], std::max(1, W.rows[c]), nullptr, 1, 0);
    }
    R.flush_copy();
    R.flush_qr();
    for (int l = T.L - 1; l >= 0; --l) {
        std::vector<std::pair<double*, int>> stacks;
        for (int p = Tree::first(l); p < Tree::first(l) + Tree::count(l); ++p) {
            int c1 = Tree::child(p, 0), c2 = Tree::child(p, 1);
            int rows = W.rows[c1] + W.rows[c2], k = B.rank[p];
            double* st = R.dalloc((size_t)std::max(1, rows * k));
            int o = 0;
            for (int c : {c1, c2}) {
                R.job(st + o, W.rows[c], k, std::max(1, rows), 0.0);
                R.term(W.p[c], 0, std::max(1, W.rows[c]), B.tr[c], 0, std::max(1, B.rank[c]), B.rank[c]);
                o += W.rows[c];
            }
            W.rows[p] = std::min(rows, k);
            W.cols[p] = k;
            W.p[p] = R.dalloc((size_t)std::max(1, W.rows[p] * k));
            stacks.push_back({st, rows});
            R.qr(st, rows, k, std::max(1, rows), W.p[p], std::max(1, W.rows[p]), nullptr, 1, 0);
        }
        R.flush_gemm(H2_FP64);
        R.flush_qr();
    }
    return W;
}

// ------------------------------------------------------------------ prep: total weights (Fig. 2 + Sec. 5)
// Z_s from the thin QR of [Z_{s+} E_s^*; R_r S_{sr}^* / ||S_{sr} R_r^*||_2 for admissible (s,r)].
static PerCl total_weights(Runner& R, const OpView& Y, const PerCl& RW) {
    H2_SPAN("total_weights");
    const Tree& T = Y.tree();
    const Basis& VY = Y.rowb();
    PerCl Z;
    Z.init(T.nc);
    // scaled blocks S_{sr} R_r^* and their norms
    std::map<int, std::pair<double*, double*>> SR;  // block -> (matrix k_s x l_r, inverse norm)
    for (int b = 0; b < (int)Y.bt().kind.size(); ++b) {
        if (Y.kind(b) != ADM) continue;
        int s = Y.T ? Y.bt().s[b] : Y.bt().t[b];
        int r = Y.other(b);
        int ks = VY.rank[s], lr = RW.rows[r];
        double* m = R.dalloc((size_t)std::max(1, ks * lr));
        double* inv = R.dalloc(1);
        R.job(m, ks, lr, std::max(1, ks), 0.0);
        T_(R, Y.S(b), mvT(RW.p[r], std::max(1, lr)), Y.colb().rank[r]);
        SR[b] = {m, inv};
    }
    R.flush_gemm(H2_FP64);
    for (auto& kv : SR) {
        int b = kv.first;
        int s = Y.T ? Y.bt().s[b] : Y.bt().t[b];
        int r = Y.other(b);
        R.norm(kv.second.first, VY.rank[s], RW.rows[r], std::max(1, VY.rank[s]), kv.second.second, nullptr);
    }
    R.flush_norm();
    for (int l = 0; l <= T.L; ++l) {
        for (int s = Tree::first(l); s < Tree::first(l) + Tree::count(l); ++s) {
            int k = VY.rank[s];
            int rows = (s > 0) ? Z.rows[Tree::parent(s)] : 0;
            for (int b : Y.row_list(s))
                if (Y.kind(b) == ADM) rows += RW.rows[Y.other(b)];
            Z.cols[s] = k;
            Z.rows[s] = std::min(rows, k);
            Z.p[s] = R.dalloc((size_t)std::max(1, Z.rows[s] * k));
            if (rows == 0) continue;
            double* st = R.dalloc((size_t)rows * std::max(1, k));
            int o = 0;
            if (s > 0) {
                int p = Tree::parent(s);
                if (Z.rows[p] > 0) {
                    R.job(st, Z.rows[p], k, rows, 0.0);
                    R.term(Z.p[p], 0, std::max(1, Z.rows[p]), VY.tr[s], 1, std::max(1, k), VY.rank[p]);
                }
                o = Z.rows[p];
            }
            for (int b : Y.row_list(s)) {
                if (Y.kind(b) != ADM) continue;
                int r = Y.other(b);
                R.copy(SR[b].first, std::max(1, k), st + o, rows, RW.rows[r], k, 1, 1.0, SR[b].second);
                o += RW.rows[r];
            }
            R.qr(st, rows, k, rows, Z.p[s], std::max(1, Z.rows[s]), nullptr, 1, 0);
        }
        R.flush_gemm(H2_FP64);
        R.flush_copy();
        R.flush_qr();
    }
    return Z;
}

// ------------------------------------------------------------------ prep: total weights by Gram matrices
// Only Z_s^* Z_s enters the method (every use of Z_s is through products whose
// Gram matrices it weights), so the stacked QR of Fig. 2 can be replaced by
// its Gram matrix, accumulated top-down,
//   G_s = E_s G_{s+} E_s^* + sum_r S_sr (W_r^* W_r) S_sr^* / ||S_sr R_r^*||_2^2,
// with ||S_sr R_r^*||_2^2 = lambda_max(S_sr W_r^* W_r S_sr^*), and factored by a
// pivoted Cholesky (Z_s^* Z_s = G_s).  The Gram matrix resolves weights down
// to about 1e-8 of the largest, so this route serves tolerances eps >= 1e-7.
static constexpr double kGramMinEps = 1e-7;
static constexpr double kCholTol = 1e-15;

static PerCl total_weights_gram(Runner& R, const OpView& Y) {
    H2_SPAN("total_weights_gram");
    const Tree& T = Y.tree();
    const Basis& VY = Y.rowb();
    const Basis& WY = Y.colb();
    const Arena::Mark mk = R.mark();  // everything but Z is scratch of this function
    PerCl Wg = basis_products(R, T, WY, WY);  // W_r^* W_r
    std::unordered_map<int, std::pair<double*, double*>> TS;  // block -> (Wg_r S_sr^*, 1 / lambda_max)
    std::vector<int> adm;
    for (int b = 0; b < (int)Y.bt().kind.size(); ++b) {
        if (Y.kind(b) != ADM) continue;
        adm.push_back(b);
        int s = Y.T ? Y.bt().s[b] : Y.bt().t[b];
        int r = Y.other(b);
        int ks = VY.rank[s], kr = WY.rank[r];
        double* t = R.dalloc((size_t)std::max(1, kr * ks));
        R.job(t, kr, ks, std::max(1, kr), 0.0);
        T_(R, mv(Wg.p[r], std::max(1, kr)), Y.S(b), kr, 1.0, nullptr, 0, 1);
        TS[b] = {t, R.dalloc(1)};
    }
    R.flush_gemm(H2_FP64);
    std::vector<double*> M(adm.size());
    for (size_t i = 0; i < adm.size(); ++i) {
        int b = adm[i];
        int s = Y.T ? Y.bt().s[b] : Y.bt().t[b];
        int r = Y.other(b);
        int ks = VY.rank[s];
        M[i] = R.dalloc((size_t)std::max(1, ks * ks));
        R.job(M[i], ks, ks, std::max(1, ks), 0.0, true);
        T_(R, Y.S(b), mv(TS[b].first, std::max(1, WY.rank[r])), WY.rank[r]);
    }
    R.flush_gemm(H2_FP64);
    for (size_t i = 0; i < adm.size(); ++i) {
        int b = adm[i];
        int s = Y.T ? Y.bt().s[b] : Y.bt().t[b];
        R.norm(M[i], VY.rank[s], VY.rank[s], std::max(1, VY.rank[s]), TS[b].second, nullptr);
    }
    R.flush_norm();
    PerCl Z, G;
    Z.init(T.nc);
    G.init(T.nc);
    for (int l = 0; l <= T.L; ++l) {
        const int c0 = Tree::first(l), nl = Tree::count(l);
        std::vector<double*> EG(nl, nullptr);
        if (l > 0) {
            for (int i = 0; i < nl; ++i) {
                int s = c0 + i, p = Tree::parent(s);
                EG[i] = R.dalloc((size_t)std::max(1, VY.rank[s] * VY.rank[p]));
                R.job(EG[i], VY.rank[s], VY.rank[p], std::max(1, VY.rank[s]), 0.0);
                R.term(VY.tr[s], 0, std::max(1, VY.rank[s]), G.p[p], 0, std::max(1, VY.rank[p]), VY.rank[p]);
            }
            R.flush_gemm(H2_FP64);
        }
        for (int i = 0; i < nl; ++i) {
            int s = c0 + i, k = VY.rank[s];
            int rows = (l > 0) ? Z.rows[Tree::parent(s)] : 0;
            for (int b : Y.row_list(s))
                if (Y.kind(b) == ADM) rows += std::min(WY.rank[Y.other(b)], (int)T.size[Y.other(b)]);
            G.rows[s] = G.cols[s] = k;
            G.p[s] = R.dalloc((size_t)std::max(1, k * k));
            R.job(G.p[s], k, k, std::max(1, k), 0.0, true);
            if (l > 0)
                R.term(EG[i], 0, std::max(1, k), VY.tr[s], 1, std::max(1, k), VY.rank[Tree::parent(s)]);
            for (int b : Y.row_list(s)) {
                if (Y.kind(b) != ADM) continue;
                int r = Y.other(b);
                T_(R, Y.S(b), mv(TS[b].first, std::max(1, WY.rank[r])), WY.rank[r], 1.0, TS[b].second);
            }
            Z.rows[s] = std::min(rows, k);
            Z.cols[s] = k;
            Z.p[s] = R.palloc((size_t)std::max(1, Z.rows[s] * k));
        }
        R.flush_gemm(H2_FP64);
        for (int i = 0; i < nl; ++i) {
            int s = c0 + i;
            R.pchol(G.p[s], VY.rank[s], std::max(1, VY.rank[s]), Z.p[s], Z.rows[s], kCholTol);
        }
        R.flush_pchol();
    }
    R.release(mk);
    return Z;
}

// ------------------------------------------------------------------ left singular vectors
// Batched left singular vectors.  Each job gives Bt (ncol x m, ld ncol), the
// transpose of the matrix whose left singular vectors are wanted.  Wide
// matrices (ncol > m) are first reduced to m x m, then one-sided Jacobi runs on
// the reduced matrix:
//  * eps >= kGramMinEps, or a low-precision mode: the FP64 Gram matrix
//    G = Bt^* Bt and its pivoted Cholesky factor Z^* Z = G; the wanted vectors
//    are those of Z^* (Z^* Z^{**} = G = Bt^* Bt).  G resolves singular values
//    down to about 3e-8 of the largest, well below these tolerances and below
//    the FP32 sweeps of the low-precision modes.
//  * otherwise: a column-pivoted thin QR Bt P = Q Rt; the wanted vectors are
//    those of Rt^* with their rows permuted by P.
// Jacobi on the transposed triangular factor of a pivoted QR needs far fewer
// sweeps than on the matrix itself (Drmac & Veselic, SIAM J. Matrix Anal.
// Appl. 29, 2008); the pivoted Cholesky factor is that factor (up to signs and
// the column order), so both routes get the short sweep count.
// The Cholesky factorisation stops once the trace of what is left is at most
// (kSvdDrop eps)^2.  What is left, S = G - Z^* Z, is positive semidefinite, so
// the singular values of Z^* differ from those of Bt by at most kSvdDrop eps
// (Weyl's inequality on G), and the part of Bt outside the range of Z^* has
// Frobenius norm at most kSvdDrop eps.  Ranks are decided by sigma > eps, so
// only directions far below the truncation are dropped; the Jacobi sweeps
// then run on the factor's r nonzero columns only (r read on the device).
static constexpr double kSvdDrop = 0.1;

struct SvdOut {
    double* U = nullptr;
    int ldu = 1;
};

class SvdBatch {
public:
    explicit SvdBatch(Runner& R) : R_(R) {}
    // queue a job; the returned index identifies its output after run()
    int add(double* Bt, int ncol, int m, double eps, int* count_slot) {
        Job j{Bt, ncol, m, eps, count_slot, nullptr, nullptr, nullptr, nullptr, nullptr};
        if (m > 0 && ncol > 0) {
            if (ncol > m) {
                j.Rt = R_.dalloc((size_t)m * m);
                if ((low_precision(R_.precision()) || eps >= kGramMinEps) && m <= 1024) {
                    j.G = R_.dalloc((size_t)m * m);  // Gram route: formed and factored in run()
                    j.r = (int*)R_.dalloc(1);        // the factor's rank, set on the device
                } else {
                    if (m <= kQRPivMax) j.piv = (int*)R_.dalloc(((size_t)m + 1) / 2);
                    R_.qr(Bt, ncol, m, ncol, j.Rt, m, nullptr, 1, 0, low_precision(R_.precision()), j.piv);
                }
            }
            j.B = R_.dalloc((size_t)m * std::min(m, ncol));
        }
        jobs_.push_back(j);
        return (int)jobs_.size() - 1;
    }
    // run every queued step in order; fills out[i] for job i
    std::vector<SvdOut> run() {
        H2_SPAN("SvdBatch::run");
        R_.flush_gemm();
        R_.flush_copy();
        bool gram = false;
        for (Job& j : jobs_)
            if (j.G) {
                R_.job(j.G, j.m, j.m, j.m, 0.0, true);
                R_.term(j.Bt, 1, j.ncol, j.Bt, 0, j.ncol, j.ncol);
                gram = true;
            }
        if (gram) {
            R_.flush_gemm(H2_FP64);
            // the factorisation stops once the trace left is (kSvdDrop eps)^2: the
            // columns it leaves out have Frobenius norm <= kSvdDrop eps together
            for (Job& j : jobs_)
                if (j.G) R_.pchol(j.G, j.m, j.m, j.Rt, j.m, kCholTol, (kSvdDrop * j.eps) * (kSvdDrop * j.eps), j.r);
            R_.flush_pchol();
        }
        R_.flush_qr();
        std::vector<SvdOut> out(jobs_.size());
        for (size_t i = 0; i < jobs_.size(); ++i) {
            Job& j = jobs_[i];
            if (!j.B) continue;
            int w = std::min(j.m, j.ncol);
            if (j.Rt)
                R_.copy(j.Rt, j.m, j.B, j.m, j.m, j.m, 1);
            else
                R_.copy(j.Bt, j.ncol, j.B, j.m, j.m, j.ncol, 1);
            out[i].U = R_.dalloc((size_t)j.m * w);
            out[i].ldu = j.m;
        }
        R_.flush_copy();
        if (low_precision(R_.precision())) {
            // FP32 sweeps on B; the FP64 sweeps start from the rotated matrix widened
            // to FP64.  Its FP32 rounding is of the order of the FP32 products that
            // formed B, so the FP64 sweeps (rank decision, orthogonality) lose nothing
            // against starting from B itself.
            std::vector<double*> C(jobs_.size(), nullptr);
            for (size_t i = 0; i < jobs_.size(); ++i) {
                Job& j = jobs_[i];
                if (!j.B) continue;
                int w = std::min(j.m, j.ncol);
                if (w < 2) continue;
                C[i] = R_.dalloc((size_t)j.m * w);
                R_.jacobi_pre(j.B, j.m, w, j.m, nullptr, C[i], j.r);
            }
            R_.flush_pre();
            for (size_t i = 0; i < jobs_.size(); ++i)
                if (C[i]) jobs_[i].B = C[i];
        }
        for (size_t i = 0; i < jobs_.size(); ++i) {
            Job& j = jobs_[i];
            if (!j.B) continue;
            int w = std::min(j.m, j.ncol);
            R_.svd(j.B, j.m, w, j.m, out[i].U, j.m, R_.dalloc(w), j.count, j.eps, j.piv, j.r);
        }
        R_.flush_svd();
        jobs_.clear();
        return out;
    }

private:
    struct Job {
        double* Bt;
        int ncol, m;
        double eps;
        int* count;
        double* Rt;   // reduced m x m factor (QR's Rt, or the Cholesky factor Z)
        double* B;
        int* piv;     // column pivots of the QR of Bt: rows of the wanted vectors
        double* G;    // Gram route: Bt^* Bt
        int* r;       // Gram route: rank of the Cholesky factor (its nonzero columns of B)
    };
    Runner& R_;
    std::vector<Job> jobs_;
};

static std::vector<int> read_counts(Runner& R, int* d_counts, int n) {
    H2_SPAN("read_counts");
    std::vector<int> h(n, 0);
    if (n > 0) {
        // into pinned memory: the copies stay asynchronous and the wait is the
        // stream synchronisation below
        int* hp = (int*)R.pinned_host(sizeof(int) * ((size_t)n + 1));
        hp[n] = 0;
        H2_CUDA(cudaMemcpyAsync(hp, d_counts, sizeof(int) * n, cudaMemcpyDeviceToHost, R.stream()));
        if (R.svd_flag())
            H2_CUDA(cudaMemcpyAsync(hp + n, R.svd_flag(), sizeof(int), cudaMemcpyDeviceToHost, R.stream()));
        {
            static const bool trace = std::getenv("H2_TRACE") != nullptr;
            const double h0 = trace ? host_clock_ms() : 0.0;
            CombIdle idle(R.combiner());
            H2_CUDA(cudaStreamSynchronize(R.stream()));
            if (trace)  // "h2sync <stream> <host ms at the wait> <host ms after it>"
                std::fprintf(stderr, "h2sync %p %.3f %.3f\n", (void*)R.stream(), h0, host_clock_ms());
        }
        std::copy(hp, hp + n, h.begin());
        static const bool trace_r = std::getenv("H2_TRACE") != nullptr;
        if (trace_r) {  // "h2ranks <clusters> <mean rank> <max rank>"
            double sr = 0;
            int mr = 0;
            for (int x : h) {
                sr += x;
                mr = std::max(mr, x);
            }
            std::fprintf(stderr, "h2ranks %d %.1f %d\n", n, sr / n, mr);
        }
        const int flag = hp[n];
        if (flag & 1) throw Error(H2_ERR_TIMEOUT, "Jacobi SVD did not converge within its sweep limit");
        if (flag & 4) throw Error(H2_ERR_TIMEOUT, "tensor-core product wait timed out");
    }
    return h;
}

// Transfer matrices of the children of the nl clusters from c0 (ranks known):
// one device chunk per level, carved at 256-byte boundaries, not one allocation
// per cluster (each device allocation is a driver call).
static size_t carve_size(size_t n) { return (std::max<size_t>(n, 1) + 31) & ~size_t(31); }
static size_t transfer_need(const Basis& B, int c0, int nl) {
    size_t need = 0;
    for (int i = 0; i < nl; ++i)
        for (int j = 0; j < 2; ++j) need += carve_size((size_t)B.rank[Tree::child(c0 + i, j)] * B.rank[c0 + i]);
    return need;
}
struct Carve {
    double* p = nullptr;
    size_t left = 0;
    Carve(Basis& B, size_t need) {
        if (need == 0) return;
        auto ch = std::make_shared<DevBuf>();
        ch->alloc(need);
        B.chunks.push_back(ch);
        p = ch->p;
        left = need;
    }
    double* take(size_t n) {
        const size_t m = carve_size(n);
        if (m > left) throw Error(H2_ERR_UNSUPPORTED, "transfer chunk too small");
        double* q = p;
        p += m;
        left -= m;
        return q;
    }
};

// ------------------------------------------------------------------ phase A (Fig. 4)
struct Induced {
    std::shared_ptr<Basis> Q;
    PerCl Rbar;                         // Q_t^* V_{X,t}: rank_Q(t) x rank_VX(t)
    std::vector<double*> A;             // X block (not admissible) -> Q_t^* X_ts V_{Y,s}: rank_Q(t) x rank_VY(s)
    bool zpres = false;                 // Z's own basis preserved as well
    PerCl RbarZ;                        // Q_t^* V_{Z,t}: rank_Q(t) x rank_VZ(t) (zpres)
};

// VZ: a basis preserved beside V_X (Z's own row basis, "+Z" with bases of its own), or null
static Induced induced_rows(Runner& R, const OpView& X, const OpView& Y, double eps, Counts& cnt,
                            const Basis* VZ = nullptr) {
    H2_SPAN("induced_rows");
    const Tree& T = X.tree();
    const Basis& VX = X.rowb();
    const Basis& VY = Y.rowb();
    const Arena::Mark mk0 = R.mark();  // scratch of this phase; A and Rbar are persistent
    PerCl P = basis_products(R, T, X.colb(), VY);
    PerCl Zt;
    if (eps >= kGramMinEps) {
        Zt = total_weights_gram(R, Y);
    } else {
        PerCl RW = basis_weights(R, T, Y.colb());
        Zt = total_weights(R, Y, RW);
    }
    Induced out;
    out.A.assign(X.bt().kind.size(), nullptr);
    out.Q = std::make_shared<Basis>();
    Basis& Q = *out.Q;
    Q.rank.assign(T.nc, 0);
    Q.leaf.assign(T.nc, nullptr);
    Q.tr.assign(T.nc, nullptr);
    out.Rbar.init(T.nc);
    out.zpres = (VZ != nullptr);
    if (VZ) out.RbarZ.init(T.nc);
    auto kz = [&](int t) { return VZ ? VZ->rank[t] : 0; };
    // per block of X (entries are set and used within the level of the block)
    std::vector<double*> M(X.bt().kind.size(), nullptr), inv(M.size(), nullptr), SPE(M.size(), nullptr);
    HostLap lap;
    lap.mark("ir:prep");
    for (int l = T.L; l >= 0; --l) {
        const Arena::Mark mkl = R.mark();  // scratch of this level
        const int c0 = Tree::first(l), nl = Tree::count(l);
        const bool leaf = (l == T.L);
        std::vector<int> rows(nl), k1(nl), m2(nl);
        std::vector<double*> VXh(nl), QX(nl), VZh(nl, nullptr);
        std::vector<std::vector<int>> C(nl);
        // PE_{s'} = P_{s'} E_{Y,s'} for the children level
        std::vector<double*> PE(T.nc, nullptr);
        if (!leaf) {
            for (int c = Tree::first(l + 1); c < Tree::first(l + 1) + Tree::count(l + 1); ++c) {
                int p = Tree::parent(c);
                PE[c] = R.dalloc((size_t)std::max(1, P.rows[c] * VY.rank[p]));
                R.job(PE[c], P.rows[c], VY.rank[p], std::max(1, P.rows[c]), 0.0);
                R.term(P.p[c], 0, std::max(1, P.rows[c]), VY.tr[c], 0, std::max(1, VY.rank[c]), VY.rank[c]);
            }
            R.flush_gemm();
        }
        lap.mark("ir:pe");
        // VX-hat and the admissible-child chains S_X(a,b) PE_b
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i;
            for (int b : X.row_list(t))
                if (X.kind(b) != ADM) C[i].push_back(b);
            if (leaf) {
                rows[i] = (int)T.size[t];
                VXh[i] = R.dalloc((size_t)rows[i] * VX.rank[t]);
                R.copy(VX.leaf[t], rows[i], VXh[i], rows[i], rows[i], VX.rank[t], 0);
                if (VZ) {
                    VZh[i] = R.dalloc((size_t)std::max(1, rows[i] * kz(t)));
                    R.copy(VZ->leaf[t], rows[i], VZh[i], rows[i], rows[i], kz(t), 0);
                }
            } else {
                int a1 = Tree::child(t, 0), a2 = Tree::child(t, 1);
                rows[i] = Q.rank[a1] + Q.rank[a2];
                VXh[i] = R.dalloc((size_t)std::max(1, rows[i] * VX.rank[t]));
                if (VZ) VZh[i] = R.dalloc((size_t)std::max(1, rows[i] * kz(t)));
                int o = 0;
                for (int a : {a1, a2}) {
                    R.job(VXh[i] + o, Q.rank[a], VX.rank[t], rows[i], 0.0);
                    R.term(out.Rbar.p[a], 0, std::max(1, Q.rank[a]), VX.tr[a], 0, std::max(1, VX.rank[a]),
                           VX.rank[a]);
                    if (VZ) {
                        R.job(VZh[i] + o, Q.rank[a], kz(t), rows[i], 0.0);
                        R.term(out.RbarZ.p[a], 0, std::max(1, Q.rank[a]), VZ->tr[a], 0, std::max(1, kz(a)), kz(a));
                    }
                    o += Q.rank[a];
                }
                for (int b : C[i]) {
                    int s = X.other(b);
                    for (int ia = 0; ia < 2; ++ia)
                        for (int j = 0; j < 2; ++j) {
                            const int a = ia ? a2 : a1;
                            int sj = Tree::child(s, j);
                            int bb = X.kid(b, ia, j);
                            if (X.kind(bb) != ADM) continue;
                            double* m = R.dalloc((size_t)std::max(1, VX.rank[a] * VY.rank[s]));
                            R.job(m, VX.rank[a], VY.rank[s], std::max(1, VX.rank[a]), 0.0);
                            T_(R, X.S(bb), mv(PE[sj], std::max(1, P.rows[sj])), X.colb().rank[sj]);
                            SPE[bb] = m;
                            cnt.flops += 2.0 * VX.rank[a] * VY.rank[s] * X.colb().rank[sj];
                        }
                }
            }
        }
        R.flush_copy();
        R.flush_gemm();
        lap.mark("ir:vxhat");
        // the blocks M_ts = X|ts V_Y,s (leaf) or A-hat_ts (Eq. induced_Ahat)
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i;
            for (int b : C[i]) {
                int s = X.other(b);
                int ky = VY.rank[s];
                double* m = R.dalloc((size_t)std::max(1, rows[i] * ky));
                M[b] = m;
                if (leaf) {
                    R.job(m, rows[i], ky, rows[i], 0.0);
                    T_(R, X.N(b), mv(VY.leaf[s], (int)T.size[s]), (int)T.size[s]);
                    cnt.flops += 2.0 * rows[i] * ky * T.size[s];
                } else {
                    int o = 0;
                    for (int ia = 0; ia < 2; ++ia) {
                        const int a = Tree::child(t, ia);
                        R.job(m + o, Q.rank[a], ky, rows[i], 0.0);
                        for (int j = 0; j < 2; ++j) {
                            int sj = Tree::child(s, j);
                            int bb = X.kid(b, ia, j);
                            if (X.kind(bb) == ADM) {
                                R.term(out.Rbar.p[a], 0, std::max(1, Q.rank[a]), SPE[bb], 0,
                                       std::max(1, VX.rank[a]), VX.rank[a]);
                                cnt.flops += 2.0 * Q.rank[a] * ky * VX.rank[a];
                            } else {
                                R.term(out.A[bb], 0, std::max(1, Q.rank[a]), VY.tr[sj], 0,
                                       std::max(1, VY.rank[sj]), VY.rank[sj]);
                                cnt.flops += 2.0 * Q.rank[a] * ky * VY.rank[sj];
                            }
                        }
                        o += Q.rank[a];
                    }
                }
                inv[b] = R.dalloc(1);
            }
        }
        R.flush_gemm();
        lap.mark("ir:M");
        for (int i = 0; i < nl; ++i)
            for (int b : C[i]) R.norm(M[b], rows[i], VY.rank[X.other(b)], std::max(1, rows[i]), inv[b], nullptr);
        R.flush_norm();
        lap.mark("ir:norm");
        // complete QR of VX-hat; tall transposed remainder; SVD
        int* d_counts = (int*)R.dalloc(nl);
        H2_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(int) * nl, R.stream()));
        // With rows <= k_X (+ k_Z) the complete Q spans all of K^rows, which contains the
        // preserved range: the identity is an equally valid choice and needs no factorisation.
        // Otherwise Q_X = I - V T V^T from the compact WY form of the Householder QR,
        // expanded by two batched FP64-accurate products (W = T V^T, Q_X = I - V W).
        int rid = 0;
        for (int i = 0; i < nl; ++i) rid = std::max(rid, rows[i]);
        double* ident = nullptr;
        if (rid > 0) {
            ident = R.dalloc((size_t)rid * rid);
            launch_set_identity(ident, rid, rid, rid, R.stream());
            ++R.launches;
        }
        std::vector<double*> Vq(nl, nullptr), Tq(nl, nullptr);
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i, kx = VX.rank[t], kp = kx + kz(t);  // preserved columns [VX-hat | VZ-hat]
            k1[i] = std::min(rows[i], kp);
            m2[i] = rows[i] - k1[i];
            QX[i] = R.dalloc((size_t)std::max(1, rows[i] * rows[i]));
            if (rows[i] <= 0) continue;
            R.copy(ident, rid, QX[i], rows[i], rows[i], rows[i], 0);
            if (rows[i] <= kp) continue;
            double* work = R.dalloc((size_t)std::max(1, rows[i] * kp));
            R.copy(VXh[i], rows[i], work, rows[i], rows[i], kx, 0);
            if (VZ && kz(t) > 0) R.copy(VZh[i], rows[i], work + (size_t)kx * rows[i], rows[i], rows[i], kz(t), 0);
            Vq[i] = R.dalloc((size_t)rows[i] * kp);
            Tq[i] = R.dalloc((size_t)kp * kp);
            R.qr_wy(work, rows[i], kp, rows[i], Vq[i], Tq[i]);
        }
        R.flush_copy();
        R.flush_qr();
        lap.mark("ir:qr");
        {
            std::vector<double*> Wq(nl, nullptr);
            for (int i = 0; i < nl; ++i) {
                if (!Vq[i]) continue;
                Wq[i] = R.dalloc((size_t)k1[i] * rows[i]);
                R.job(Wq[i], k1[i], rows[i], k1[i], 0.0);
                R.term(Tq[i], 0, k1[i], Vq[i], 1, rows[i], k1[i]);
            }
            R.flush_gemm(H2_FP64);
            for (int i = 0; i < nl; ++i) {
                if (!Vq[i]) continue;
                R.job(QX[i], rows[i], rows[i], rows[i], 1.0);
                R.term(Vq[i], 0, rows[i], Wq[i], 0, k1[i], k1[i], -1.0);
            }
            R.flush_gemm(H2_FP64);
        }
        lap.mark("ir:wq");
        std::vector<double*> Vts(nl, nullptr), Tts(nl, nullptr);
        std::vector<int> ncols(nl, 0);
        for (int i = 0; i < nl; ++i) {
            int ncol = 0;
            for (int b : C[i]) ncol += Zt.rows[X.other(b)];
            ncols[i] = ncol;
            if (m2[i] == 0 || ncol == 0) continue;
            double* Tt = R.dalloc((size_t)ncol * rows[i]);
            int o = 0;
            for (int b : C[i]) {
                int s = X.other(b);
                if (Zt.rows[s] == 0) continue;
                R.job(Tt + o, Zt.rows[s], rows[i], ncol, 0.0);
                R.term(Zt.p[s], 0, Zt.rows[s], M[b], 1, rows[i], VY.rank[s], 1.0, inv[b]);
                o += Zt.rows[s];
            }
            Vts[i] = R.dalloc((size_t)ncol * m2[i]);
            Tts[i] = Tt;
        }
        R.flush_gemm();
        for (int i = 0; i < nl; ++i) {
            if (!Vts[i]) continue;
            R.job(Vts[i], ncols[i], m2[i], ncols[i], 0.0);
            R.term(Tts[i], 0, ncols[i], QX[i] + (size_t)k1[i] * rows[i], 0, rows[i], rows[i]);
        }
        R.flush_gemm();
        SvdBatch sb(R);
        for (int i = 0; i < nl; ++i)
            if (Vts[i]) sb.add(Vts[i], ncols[i], m2[i], eps, d_counts + i);
            else sb.add(nullptr, 0, 0, eps, d_counts + i);
        lap.mark("ir:tt");
        std::vector<SvdOut> so = sb.run();
        lap.mark("ir:svd");
        std::vector<int> k2 = read_counts(R, d_counts, nl);
        lap.mark("ir:sync");
        // new basis: leaf matrices or transfers of the children
        size_t need = 0;
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i;
            Q.rank[t] = k1[i] + k2[i];
            need += (size_t)rows[i] * Q.rank[t];
        }
        auto chunk = std::make_shared<DevBuf>();
        chunk->alloc(std::max<size_t>(need, 1));
        Q.chunks.push_back(chunk);
        size_t off = 0;
        std::vector<double*> Qh(nl);
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i, kt = Q.rank[t];
            double* q = chunk->p + off;
            off += (size_t)rows[i] * kt;
            Qh[i] = q;
            // Q-hat = [Q_X(:, :k1) | Q_X(:, k1:) U(:, :k2)]
            R.copy(QX[i], rows[i], q, rows[i], rows[i], k1[i], 0);
            if (k2[i] > 0) {
                R.job(q + (size_t)k1[i] * rows[i], rows[i], k2[i], rows[i], 0.0);
                R.term(QX[i] + (size_t)k1[i] * rows[i], 0, rows[i], so[i].U, 0, so[i].ldu, m2[i]);
            }
        }
        R.flush_copy();
        R.flush_gemm();
        lap.mark("ir:newbasis");
        Carve trc(Q, leaf ? 0 : transfer_need(Q, c0, nl));  // the children's transfers of this level
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i, kt = Q.rank[t];
            if (leaf) {
                Q.leaf[t] = Qh[i];
            } else {
                // split rows into the children's transfers (stored with ld = rank of the child)
                int o = 0;
                for (int a : {Tree::child(t, 0), Tree::child(t, 1)}) {
                    double* tp = trc.take((size_t)Q.rank[a] * kt);
                    R.copy(Qh[i] + o, rows[i], tp, std::max(1, Q.rank[a]), Q.rank[a], kt, 0);
                    Q.tr[a] = tp;
                    o += Q.rank[a];
                }
            }
            // A_ts = Q-hat^* M_ts,  Rbar_t = Q-hat^* VX-hat
            for (int b : C[i]) {
                int s = X.other(b);
                double* a = R.palloc((size_t)std::max(1, kt * VY.rank[s]));
                R.job(a, kt, VY.rank[s], std::max(1, kt), 0.0);
                R.term(Qh[i], 1, rows[i], M[b], 0, std::max(1, rows[i]), rows[i]);
                out.A[b] = a;
                cnt.flops += 2.0 * kt * VY.rank[s] * rows[i];
            }
            out.Rbar.rows[t] = kt;
            out.Rbar.cols[t] = VX.rank[t];
            out.Rbar.p[t] = R.palloc((size_t)std::max(1, kt * VX.rank[t]));
            R.job(out.Rbar.p[t], kt, VX.rank[t], std::max(1, kt), 0.0);
            R.term(Qh[i], 1, rows[i], VXh[i], 0, std::max(1, rows[i]), rows[i]);
            if (VZ) {  // Rbar_Z,t = Q-hat^* VZ-hat
                out.RbarZ.rows[t] = kt;
                out.RbarZ.cols[t] = kz(t);
                out.RbarZ.p[t] = R.palloc((size_t)std::max(1, kt * kz(t)));
                R.job(out.RbarZ.p[t], kt, kz(t), std::max(1, kt), 0.0);
                R.term(Qh[i], 1, rows[i], VZh[i], 0, std::max(1, rows[i]), rows[i]);
            }
        }
        R.flush_copy();
        R.flush_gemm();
        R.release(mkl);
        lap.mark("ir:A");
    }
    R.release(mk0);
    return out;
}

// ------------------------------------------------------------------ the intermediate matrix on T^XY
// Couplings of every T^XY node in the compressed induced bases ("t_mat"):
//   (t,s),(s,r) admissible: Rbar_t S_X P_s S_Y RbarW_r^*
//   (t,s) inadmissible:     A_ts S_Y RbarW_r^*                 (Eq. semiuniform)
//   (s,r) inadmissible:     Rbar_t S_X B_rs^*                  (Eq. semiuniform2)
// grouped per node as U1 = sum S_X (P S_Y) + S_Z, U2 = Rbar U1 + sum A S_Y,
// U3 = sum S_X B^*, C = U2 RbarW^* + Rbar U3; then pushed to the leaves with
// the new transfer matrices.  Dense leaves hold the exact leaf-level products
// plus the expansion of the pushed-down coupling.
struct Intermediate {
    const ProductTree* PT = nullptr;  // the cached plan
    std::shared_ptr<Basis> Q, QW;  // row / column bases (isometric)
    std::vector<double*> C;        // per node: coupling (ADM / SPLIT) or dense block (DENSE)
};

static void induced_matrix(Runner& R, const OpView& X, const OpView& Y, const h2_matrix* Z, const Induced& ra,
                           const Induced& ca, Intermediate& G, Counts& cnt) {
    H2_SPAN("induced_matrix");
    const Tree& T = X.tree();
    const Basis& Q = *ra.Q;
    const Basis& QW = *ca.Q;
    const Basis& VX = X.rowb();
    const Basis& WX = X.colb();
    const Basis& VY = Y.rowb();
    const Basis& WY = Y.colb();
    const BlockTree& N = G.PT->nodes;
    const int nn = (int)N.kind.size();
    const OpView ZV{Z, false};
    const Arena::Mark mk0 = R.mark();
    PerCl P = basis_products(R, T, WX, VY);
    // nodes by level (same-level pairs: the level of (t,r) is the level of t)
    std::vector<std::vector<int>> lv(T.L + 1);
    for (int n = 0; n < nn; ++n) lv[Tree::level(N.t[n])].push_back(n);
    G.C.assign(nn, nullptr);
    std::vector<int> zbk(nn);  // block of Z on each node, or -1
    for (int n = 0; n < nn; ++n) zbk[n] = Z->st->blocks.find(N.t[n], N.s[n]);
    // couplings pushed down from the ancestors live in two alternating arenas
    Arena pp0(R.stream()), pp1(R.stream());
    Arena* pp[2] = {&pp0, &pp1};
    std::vector<double*> Cup(nn, nullptr);
    auto alloc_cup = [&](int l) {
        size_t tot = 0;
        for (int n : lv[l]) tot += (size_t)std::max(1, Q.rank[N.t[n]] * QW.rank[N.s[n]]);
        double* base = pp[l & 1]->alloc(std::max<size_t>(tot, 1));
        H2_CUDA(cudaMemsetAsync(base, 0, sizeof(double) * std::max<size_t>(tot, 1), R.stream()));
        size_t o = 0;
        for (int n : lv[l]) {
            Cup[n] = base + o;
            o += (size_t)std::max(1, Q.rank[N.t[n]] * QW.rank[N.s[n]]);
        }
    };
    alloc_cup(0);
    // per-chunk device pointers by node or block (cleared after each chunk)
    Slots PSY(Y.bt().kind.size()), WN(Y.bt().kind.size()), XV(X.bt().kind.size());
    Slots U1(nn), U2(nn), U3(nn), L1(nn), R1(nn), CQ(nn), ZR(nn);
    // nodes of a level are processed in chunks that bound the scratch
#ifndef H2_TMAT_CHUNK
#define H2_TMAT_CHUNK 16384
#endif
    constexpr size_t kChunkNodes = H2_TMAT_CHUNK;
    for (int l = 0; l <= T.L; ++l) {
      if (l < T.L) alloc_cup(l + 1);
      for (size_t ch0 = 0; ch0 < lv[l].size(); ch0 += kChunkNodes) {
        const Arena::Mark mkl = R.mark();
        const std::vector<int> nodes(lv[l].begin() + ch0,
                                     lv[l].begin() + std::min(lv[l].size(), ch0 + kChunkNodes));
        // PSY_sr = P_s S_Y,sr for the admissible Y blocks met at this level
        PSY.clear();
        for (int n : nodes) {
            int t = N.t[n], r = N.s[n];
            const auto& tb = G.PT->tri_blocks[n];
            const auto& tk = G.PT->tri_kinds[n];
            for (size_t q = 0; q < tb.size(); ++q) {
                const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                if (tk[q].first != ADM || tk[q].second != ADM || PSY.has(by)) continue;
                double* m = R.dalloc((size_t)WX.rank[s] * WY.rank[r]);
                R.job(m, WX.rank[s], WY.rank[r], WX.rank[s], 0.0);
                T_(R, mv(P.p[s], std::max(1, P.rows[s])), Y.S(by), VY.rank[s]);
                PSY[by] = m;
                cnt.flops += 2.0 * WX.rank[s] * WY.rank[r] * VY.rank[s];
            }
        }
        R.flush_gemm();
        // U1 = S_Z (copied first) + sum_a S_X PSY
        U1.clear();
        {
            size_t tot = 0;
            for (int n : nodes) tot += (size_t)VX.rank[N.t[n]] * WY.rank[N.s[n]];
            double* base = R.dalloc(std::max<size_t>(tot, 1));
            H2_CUDA(cudaMemsetAsync(base, 0, sizeof(double) * std::max<size_t>(tot, 1), R.stream()));
            size_t o = 0;
            for (int n : nodes) {
                U1[n] = base + o;
                o += (size_t)VX.rank[N.t[n]] * WY.rank[N.s[n]];
            }
        }
        const bool zgen = ra.zpres || ca.zpres;  // Z with bases of its own: enters C below
        for (int n : nodes) {
            int t = N.t[n], r = N.s[n];
            int bz = zbk[n];
            if (!zgen && bz >= 0 && Z->st->blocks.kind[bz] == ADM)
                R.copy(ZV.S(bz).p, ZV.S(bz).ld, U1[n], VX.rank[t], VX.rank[t], WY.rank[r], 0);
        }
        R.flush_copy();
        for (int n : nodes) {
            int t = N.t[n], r = N.s[n];
            R.job(U1[n], VX.rank[t], WY.rank[r], VX.rank[t], 1.0);
            const auto& tb = G.PT->tri_blocks[n];
            const auto& tk = G.PT->tri_kinds[n];
            for (size_t q = 0; q < tb.size(); ++q) {
                const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                if (tk[q].first == ADM && tk[q].second == ADM) {
                    T_(R, X.S(bx), mv(PSY[by], WX.rank[s]), WX.rank[s]);
                    cnt.flops += 2.0 * VX.rank[t] * WY.rank[r] * WX.rank[s];
                }
                cnt.triples++;
            }
        }
        R.flush_gemm();
        // U2 = Rbar U1 + sum_b A S_Y,  U3 = sum_c S_X B^*  (coupling nodes);
        // Z with bases of its own: ZR = Rbar_Z S_Z
        U2.clear();
        U3.clear();
        ZR.clear();
        const PerCl& RZ = ra.zpres ? ra.RbarZ : ra.Rbar;
        const PerCl& RWZ = ca.zpres ? ca.RbarZ : ca.Rbar;
        for (int n : nodes) {
            if (N.kind[n] == DENSE) continue;
            int t = N.t[n], r = N.s[n];
            U2[n] = R.dalloc((size_t)std::max(1, Q.rank[t] * WY.rank[r]));
            R.job(U2[n], Q.rank[t], WY.rank[r], std::max(1, Q.rank[t]), 0.0);
            R.term(ra.Rbar.p[t], 0, std::max(1, Q.rank[t]), U1[n], 0, VX.rank[t], VX.rank[t]);
            const auto& tb = G.PT->tri_blocks[n];
            const auto& tk = G.PT->tri_kinds[n];
            for (size_t q = 0; q < tb.size(); ++q) {
                const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                if (tk[q].first != ADM && tk[q].second == ADM) {
                    T_(R, mv(ra.A[bx], std::max(1, Q.rank[t])), Y.S(by), VY.rank[s]);
                    cnt.flops += 2.0 * Q.rank[t] * WY.rank[r] * VY.rank[s];
                }
            }
            int bz = zbk[n];
            if (zgen && bz >= 0 && Z->st->blocks.kind[bz] == ADM) {
                const int kzr = Z->V->rank[t], kzc = Z->W->rank[r];
                ZR[n] = R.dalloc((size_t)std::max(1, Q.rank[t] * kzc));
                R.job(ZR[n], Q.rank[t], kzc, std::max(1, Q.rank[t]), 0.0);
                R.term(RZ.p[t], 0, std::max(1, Q.rank[t]), ZV.S(bz).p, 0, std::max(1, kzr), kzr);
            }
            U3[n] = R.dalloc((size_t)std::max(1, VX.rank[t] * QW.rank[r]));
            R.job(U3[n], VX.rank[t], QW.rank[r], VX.rank[t], 0.0);
            for (size_t q = 0; q < tb.size(); ++q) {
                const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                if (tk[q].first == ADM && tk[q].second != ADM) {
                    T_(R, X.S(bx), mvT(ca.A[by], std::max(1, QW.rank[r])), WX.rank[s]);
                    cnt.flops += 2.0 * VX.rank[t] * QW.rank[r] * WX.rank[s];
                }
            }
        }
        R.flush_gemm();
        // C = U2 RbarW^* + Rbar U3 (persistent for admissible leaves, scratch for split nodes)
        for (int n : nodes) {
            if (N.kind[n] == DENSE) continue;
            int t = N.t[n], r = N.s[n];
            size_t cs = (size_t)std::max(1, Q.rank[t] * QW.rank[r]);
            G.C[n] = (N.kind[n] == ADM) ? R.palloc(cs) : R.dalloc(cs);
            R.job(G.C[n], Q.rank[t], QW.rank[r], std::max(1, Q.rank[t]), 0.0);
            R.term(U2[n], 0, std::max(1, Q.rank[t]), ca.Rbar.p[r], 1, std::max(1, QW.rank[r]), WY.rank[r]);
            R.term(ra.Rbar.p[t], 0, std::max(1, Q.rank[t]), U3[n], 0, VX.rank[t], VX.rank[t]);
            if (ZR.has(n))
                R.term(ZR[n], 0, std::max(1, Q.rank[t]), RWZ.p[r], 1, std::max(1, QW.rank[r]), Z->W->rank[r]);
            cnt.flops += 2.0 * Q.rank[t] * QW.rank[r] * (WY.rank[r] + VX.rank[t]);
        }
        R.flush_gemm();
        // push down to the next level: Cup_child = E_a (C + Cup) F_b^*
        if (l < T.L) {
            std::vector<std::pair<int, double*>> tmp;
            for (int n : nodes) {
                if (N.kind[n] != SPLIT) continue;
                int t = N.t[n], r = N.s[n];
                for (int j = 0; j < 2; ++j) {
                    int b = Tree::child(r, j);
                    double* m = R.dalloc((size_t)std::max(1, Q.rank[t] * QW.rank[b]));
                    R.job(m, Q.rank[t], QW.rank[b], std::max(1, Q.rank[t]), 0.0);
                    R.term(G.C[n], 0, std::max(1, Q.rank[t]), QW.tr[b], 1, std::max(1, QW.rank[b]), QW.rank[r]);
                    R.term(Cup[n], 0, std::max(1, Q.rank[t]), QW.tr[b], 1, std::max(1, QW.rank[b]), QW.rank[r]);
                    for (int i = 0; i < 2; ++i) tmp.push_back({G.PT->nodes.kids[n][2 * i + j], m});
                }
            }
            R.flush_gemm();
            for (auto& [c, m] : tmp) {
                int a = N.t[c], b = N.s[c], t = Tree::parent(a);
                R.job(Cup[c], Q.rank[a], QW.rank[b], std::max(1, Q.rank[a]), 0.0);
                R.term(Q.tr[a], 0, std::max(1, Q.rank[a]), m, 0, std::max(1, Q.rank[t]), Q.rank[t]);
                cnt.flops += 2.0 * Q.rank[a] * QW.rank[b] * Q.rank[t];
            }
            R.flush_gemm();
        }
        // admissible leaves: final coupling C + Cup
        for (int n : nodes) {
            if (N.kind[n] != ADM) continue;
            int t = N.t[n], r = N.s[n];
            R.copy(Cup[n], std::max(1, Q.rank[t]), G.C[n], std::max(1, Q.rank[t]), Q.rank[t], QW.rank[r], 0, 1.0,
                   nullptr, 1.0);
        }
        R.flush_copy();
        // dense leaves, exact: sum N N + L1 W_Y^* + V_X R1 + N_Z + Q (Cup QW^*)
        bool any_dense = false;
        for (int n : nodes) any_dense |= (N.kind[n] == DENSE);
        if (any_dense) {
            XV.clear();
            WN.clear();
            L1.clear();
            R1.clear();
            CQ.clear();
            for (int n : nodes) {
                if (N.kind[n] != DENSE) continue;
                int t = N.t[n], r = N.s[n];
                const auto& tb = G.PT->tri_blocks[n];
                const auto& tk = G.PT->tri_kinds[n];
                for (size_t q = 0; q < tb.size(); ++q) {
                    const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                    if (tk[q].first == DENSE && tk[q].second == ADM && !XV.has(bx)) {
                        double* m = R.dalloc((size_t)T.size[t] * VY.rank[s]);
                        R.job(m, (int)T.size[t], VY.rank[s], (int)T.size[t], 0.0);
                        T_(R, X.N(bx), mv(VY.leaf[s], (int)T.size[s]), (int)T.size[s]);
                        XV[bx] = m;
                    }
                    if (tk[q].first == ADM && tk[q].second == DENSE && !WN.has(by)) {
                        double* m = R.dalloc((size_t)WX.rank[s] * T.size[r]);
                        R.job(m, WX.rank[s], (int)T.size[r], WX.rank[s], 0.0);
                        T_(R, mvT(WX.leaf[s], (int)T.size[s]), Y.N(by), (int)T.size[s]);
                        WN[by] = m;
                    }
                }
                CQ[n] = R.dalloc((size_t)std::max(1, Q.rank[t]) * T.size[r]);
                R.job(CQ[n], Q.rank[t], (int)T.size[r], std::max(1, Q.rank[t]), 0.0);
                R.term(Cup[n], 0, std::max(1, Q.rank[t]), QW.leaf[r], 1, (int)T.size[r], QW.rank[r]);
                // Z with bases of its own, admissible on this dense leaf: ZL = V_Z,t S_Z
                const int bz = zbk[n];
                if (zgen && bz >= 0 && Z->st->blocks.kind[bz] == ADM) {
                    const int kzr = Z->V->rank[t], kzc = Z->W->rank[r];
                    ZR[n] = R.dalloc((size_t)std::max(1, (int)T.size[t] * kzc));
                    R.job(ZR[n], (int)T.size[t], kzc, (int)T.size[t], 0.0);
                    R.term(Z->V->leaf[t], 0, (int)T.size[t], ZV.S(bz).p, 0, std::max(1, kzr), kzr);
                }
            }
            R.flush_gemm();
            for (int n : nodes) {
                if (N.kind[n] != DENSE) continue;
                int t = N.t[n], r = N.s[n];
                L1[n] = R.dalloc((size_t)T.size[t] * WY.rank[r]);
                R.job(L1[n], (int)T.size[t], WY.rank[r], (int)T.size[t], 0.0);
                R.term(VX.leaf[t], 0, (int)T.size[t], U1[n], 0, VX.rank[t], VX.rank[t]);
                const auto& tb = G.PT->tri_blocks[n];
                const auto& tk = G.PT->tri_kinds[n];
                for (size_t q = 0; q < tb.size(); ++q) {
                    const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                    if (tk[q].first == DENSE && tk[q].second == ADM) T_(R, mv(XV[bx], (int)T.size[t]), Y.S(by), VY.rank[s]);
                }
                R1[n] = R.dalloc((size_t)VX.rank[t] * T.size[r]);
                R.job(R1[n], VX.rank[t], (int)T.size[r], VX.rank[t], 0.0);
                for (size_t q = 0; q < tb.size(); ++q) {
                    const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                    if (tk[q].first == ADM && tk[q].second == DENSE) T_(R, X.S(bx), mv(WN[by], WX.rank[s]), WX.rank[s]);
                }
            }
            R.flush_gemm();
            for (int n : nodes) {
                if (N.kind[n] != DENSE) continue;
                int t = N.t[n], r = N.s[n];
                int mt = (int)T.size[t], mr = (int)T.size[r];
                G.C[n] = R.palloc((size_t)mt * mr);
                int bz = zbk[n];
                if (bz >= 0 && Z->st->blocks.kind[bz] == DENSE) R.copy(ZV.N(bz).p, ZV.N(bz).ld, G.C[n], mt, mt, mr, 0);
            }
            R.flush_copy();
            for (int n : nodes) {
                if (N.kind[n] != DENSE) continue;
                int t = N.t[n], r = N.s[n];
                int mt = (int)T.size[t], mr = (int)T.size[r];
                int bz = zbk[n];
                bool zd = bz >= 0 && Z->st->blocks.kind[bz] == DENSE;
                R.job(G.C[n], mt, mr, mt, zd ? 1.0 : 0.0);
                const auto& tb = G.PT->tri_blocks[n];
                const auto& tk = G.PT->tri_kinds[n];
                for (size_t q = 0; q < tb.size(); ++q) {
                    const int s = G.PT->triples[n][q], bx = tb[q].first, by = tb[q].second;
                    if (tk[q].first == DENSE && tk[q].second == DENSE) {
                        T_(R, X.N(bx), Y.N(by), (int)T.size[s]);
                        cnt.flops += 2.0 * mt * mr * T.size[s];
                    }
                }
                R.term(L1[n], 0, mt, WY.leaf[r], 1, mr, WY.rank[r]);
                R.term(VX.leaf[t], 0, mt, R1[n], 0, VX.rank[t], VX.rank[t]);
                R.term(Q.leaf[t], 0, mt, CQ[n], 0, std::max(1, Q.rank[t]), Q.rank[t]);
                if (ZR.has(n)) R.term(ZR[n], 0, mt, Z->W->leaf[r], 1, mr, Z->W->rank[r]);
            }
            R.flush_gemm();
        }
        R.release(mkl);
      }
      pp[l & 1]->release_all();  // this level's pushed-down couplings are consumed
    }
    R.release(mk0);
}

// ------------------------------------------------------------------ coarsening (Fig. 7, Fig. 6)
// View of the intermediate matrix, optionally transposed (G^* for the column basis).
struct GView {
    const Intermediate* G;
    const Tree* tree;
    bool T;
    const BlockTree& nodes() const { return G->PT->nodes; }
    const Basis& rowb() const { return T ? *G->QW : *G->Q; }
    const Basis& colb() const { return T ? *G->Q : *G->QW; }
    int node(int t, int r) const { return T ? nodes().find(r, t) : nodes().find(t, r); }
    // child (child(t, i), child(r, j)) of split node n in view coordinates
    int kid(int n, int i, int j) const { return T ? G->PT->nodes.kids[n][2 * j + i] : G->PT->nodes.kids[n][2 * i + j]; }
    const std::vector<int>& row_list(int t) const { return T ? nodes().by_col[t] : nodes().by_row[t]; }
    int other(int n) const { return T ? nodes().t[n] : nodes().s[n]; }
    int8_t kind(int n) const { return nodes().kind[n]; }
    Mv C(int n) const { return Mv{G->C[n], std::max(1, G->Q->rank[nodes().t[n]]), T ? 1 : 0}; }
    Mv D(int n) const { return Mv{G->C[n], (int)tree->size[nodes().t[n]], T ? 1 : 0}; }
};

// Q'_a^* G|_{a x b} as a matrix over the leaves of its column tree.
struct Rep {
    struct Leaf {
        int c;
        bool adm;
        int col, width;
    };
    double* p = nullptr;
    int ld = 1;
    std::vector<Leaf> leaves;
};

struct Coarse {
    std::shared_ptr<Basis> Qn;
    PerCl Rt;  // Q'_t^* Q_t
};

// One chain X0 F1 F2 ... written to dst; no factors means a copy.
// src F_1 ... F_nf written to dst; the factors F and their column counts sit in a
// pool shared by the chains of one level (entries f0 .. f0 + nf - 1)
struct Chain {
    Mv src;
    int rows, cols0;
    int f0, nf;
    double* dst;
    int ldd;
};
struct ChainPool {
    std::vector<Mv> f;
    std::vector<int> fcols;
    void clear() {
        f.clear();
        fcols.clear();
    }
};

static void run_chains(Runner& R, std::vector<Chain>& items, const ChainPool& pool) {
    H2_SPAN("run_chains");
    int maxlen = 0;
    for (auto& c : items) maxlen = std::max(maxlen, c.nf);
    std::vector<Mv> cur(items.size());
    std::vector<int> curc(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        cur[i] = items[i].src;
        curc[i] = items[i].cols0;
        if (items[i].nf == 0)
            R.copy(items[i].src.p, items[i].src.ld, items[i].dst, items[i].ldd, items[i].rows, items[i].cols0,
                   items[i].src.tr);
    }
    R.flush_copy();
    for (int st = 0; st < maxlen; ++st) {
        for (size_t i = 0; i < items.size(); ++i) {
            Chain& c = items[i];
            if (st >= c.nf) continue;
            bool last = (st + 1 == c.nf);
            int nc = pool.fcols[c.f0 + st];
            double* d = last ? c.dst : R.dalloc((size_t)std::max(1, c.rows * nc));
            int ldd = last ? c.ldd : std::max(1, c.rows);
            R.job(d, c.rows, nc, ldd, 0.0);
            T_(R, cur[i], pool.f[c.f0 + st], curc[i]);
            cur[i] = mv(d, ldd);
            curc[i] = nc;
        }
        R.flush_gemm();
    }
}

static bool is_desc(int a, int d) {  // a is an ancestor of d (or equal)
    while (d > a) d = Tree::parent(d);
    return d == a;
}

static Coarse coarsen_rows(Runner& R, const GView& G, const std::vector<int>& cmap, const double* w,
                           const double* w2, double eps) {
    H2_SPAN("coarsen_rows");
    const Tree& T = *G.tree;
    const Basis& Q = G.rowb();
    const Basis& QW = G.colb();
    const Arena::Mark mk0 = R.mark();
    Arena pp0(R.stream()), pp1(R.stream());  // representations of two consecutive levels
    Arena* pp[2] = {&pp0, &pp1};
    Coarse out;
    out.Qn = std::make_shared<Basis>();
    Basis& Qn = *out.Qn;
    Qn.rank.assign(T.nc, 0);
    Qn.leaf.assign(T.nc, nullptr);
    Qn.tr.assign(T.nc, nullptr);
    out.Rt.init(T.nc);
    // total weights of the product (Eq. Zt_condensation), top-down
    PerCl Zt;
    Zt.init(T.nc);
    if (eps >= kGramMinEps) {
        // Gram form: G_t = E_t G_{t+} E_t^* + sum_r w_b^2 S_tr S_tr^*, Z_t by pivoted Cholesky
        PerCl Gm;
        Gm.init(T.nc);
        for (int l = 0; l <= T.L; ++l) {
            const int c0 = Tree::first(l), nl = Tree::count(l);
            std::vector<double*> EG(nl, nullptr);
            if (l > 0) {
                for (int i = 0; i < nl; ++i) {
                    int t = c0 + i, p = Tree::parent(t);
                    EG[i] = R.dalloc((size_t)std::max(1, Q.rank[t] * Q.rank[p]));
                    R.job(EG[i], Q.rank[t], Q.rank[p], std::max(1, Q.rank[t]), 0.0);
                    R.term(Q.tr[t], 0, std::max(1, Q.rank[t]), Gm.p[p], 0, std::max(1, Q.rank[p]), Q.rank[p]);
                }
                R.flush_gemm(H2_FP64);
            }
            for (int i = 0; i < nl; ++i) {
                int t = c0 + i, k = Q.rank[t];
                int rows = (l > 0) ? Zt.rows[Tree::parent(t)] : 0;
                Gm.p[t] = R.dalloc((size_t)std::max(1, k * k));
                R.job(Gm.p[t], k, k, std::max(1, k), 0.0, true);
                if (l > 0) R.term(EG[i], 0, std::max(1, k), Q.tr[t], 1, std::max(1, k), Q.rank[Tree::parent(t)]);
                for (int n : G.row_list(t)) {
                    if (G.kind(n) != ADM) continue;
                    int r = G.other(n);
                    if (cmap[n] < 0) throw Error(H2_ERR_UNSUPPORTED, "admissible T^XY leaf outside the target's admissible blocks");
                    Mv c = G.C(n);
                    R.term(c.p, c.tr, c.ld, c.p, c.tr ^ 1, c.ld, QW.rank[r], 1.0, w2 + cmap[n]);
                    rows += QW.rank[r];
                }
                Zt.rows[t] = std::min(rows, k);
                Zt.cols[t] = k;
                Zt.p[t] = R.dalloc((size_t)std::max(1, Zt.rows[t] * k));
                if (Zt.rows[t] == 0 || k == 0) Zt.rows[t] = 0;
            }
            R.flush_gemm(H2_FP64);
            for (int i = 0; i < nl; ++i) {
                int t = c0 + i;
                if (Zt.rows[t] > 0) R.pchol(Gm.p[t], Q.rank[t], std::max(1, Q.rank[t]), Zt.p[t], Zt.rows[t], kCholTol);
            }
            R.flush_pchol();
        }
    }
    for (int l = 0; l <= T.L && eps < kGramMinEps; ++l) {
        for (int t = Tree::first(l); t < Tree::first(l) + Tree::count(l); ++t) {
            int k = Q.rank[t];
            int rows = (t > 0) ? Zt.rows[Tree::parent(t)] : 0;
            for (int n : G.row_list(t))
                if (G.kind(n) == ADM) rows += QW.rank[G.other(n)];
            Zt.rows[t] = std::min(rows, k);
            Zt.cols[t] = k;
            Zt.p[t] = R.dalloc((size_t)std::max(1, Zt.rows[t] * k));
            if (rows == 0 || k == 0) {
                Zt.rows[t] = 0;
                continue;
            }
            double* st = R.dalloc((size_t)rows * k);
            int o = 0;
            if (t > 0) {
                int p = Tree::parent(t);
                if (Zt.rows[p] > 0) {
                    R.job(st, Zt.rows[p], k, rows, 0.0);
                    R.term(Zt.p[p], 0, Zt.rows[p], Q.tr[t], 1, std::max(1, k), Q.rank[p]);
                }
                o = Zt.rows[p];
            }
            for (int n : G.row_list(t)) {
                if (G.kind(n) != ADM) continue;
                int r = G.other(n);
                if (cmap[n] < 0) throw Error(H2_ERR_UNSUPPORTED, "admissible T^XY leaf outside the target's admissible blocks");
                Mv c = G.C(n);
                R.copy(c.p, c.ld, st + o, rows, QW.rank[r], k, c.tr ^ 1, 1.0, w + cmap[n]);
                o += QW.rank[r];
            }
            R.qr(st, rows, k, rows, Zt.p[t], Zt.rows[t], nullptr, 1, 0);
        }
        R.flush_gemm();
        R.flush_copy();
        R.flush_qr();
    }
    std::vector<Rep> A(G.nodes().kind.size());     // node -> representation
    std::vector<Rep> Ahat(G.nodes().kind.size());  // split node -> A-hat before the projection (per level)
    std::vector<Chain> chains;
    ChainPool pool;
    std::vector<std::pair<int, bool>> target;  // cluster -> admissible (all reps agree)
    std::vector<int> path;
    HostLap lap;
    lap.mark("cr:prep");
    for (int l = T.L; l >= 0; --l) {
        const Arena::Mark mkl = R.mark();
        const int c0 = Tree::first(l), nl = Tree::count(l);
        const bool leaf = (l == T.L);
        std::vector<int> rows(nl);
        std::vector<double*> Vh(nl, nullptr);
        std::vector<std::vector<int>> nodes(nl);   // dense (leaf) or split (non-leaf) coarse-admissible nodes
        chains.clear();
        pool.clear();
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i;
            for (int n : G.row_list(t))
                if (cmap[n] >= 0 && G.kind(n) == (leaf ? DENSE : SPLIT)) nodes[i].push_back(n);
            if (leaf) {
                rows[i] = (int)T.size[t];
                continue;
            }
            int a1 = Tree::child(t, 0), a2 = Tree::child(t, 1);
            rows[i] = Qn.rank[a1] + Qn.rank[a2];
            Vh[i] = R.dalloc((size_t)std::max(1, rows[i] * Q.rank[t]));
            int o = 0;
            for (int a : {a1, a2}) {
                R.job(Vh[i] + o, Qn.rank[a], Q.rank[t], std::max(1, rows[i]), 0.0);
                R.term(out.Rt.p[a], 0, std::max(1, Qn.rank[a]), Q.tr[a], 0, std::max(1, Q.rank[a]), Q.rank[a]);
                o += Qn.rank[a];
            }
            // A-hat for every split coarse-admissible node (Eq. ct_nonleaf with match_column)
            for (int n : nodes[i]) {
                int r = G.other(n);
                target.clear();
                auto slot = [&](int c) -> std::pair<int, bool>* {
                    for (auto& x : target)
                        if (x.first == c) return &x;
                    return nullptr;
                };
                for (int ia = 0; ia < 2; ++ia)
                    for (int j = 0; j < 2; ++j) {
                        int b = Tree::child(r, j);
                        int nb = G.kid(n, ia, j);
                        if (G.kind(nb) == ADM) {
                            if (!slot(b)) target.push_back({b, true});
                        } else {
                            for (auto& lf : A[nb].leaves) {
                                auto* x = slot(lf.c);
                                if (x)
                                    x->second = x->second && lf.adm;
                                else
                                    target.push_back({lf.c, lf.adm});
                            }
                        }
                    }
                Rep rep;
                for (auto& [c, adm] : target) {
                    bool finest = true;
                    for (auto& kv : target)
                        if (kv.first != c && is_desc(c, kv.first)) finest = false;
                    if (finest) rep.leaves.push_back(Rep::Leaf{c, adm, 0, adm ? QW.rank[c] : (int)T.size[c]});
                }
                std::sort(rep.leaves.begin(), rep.leaves.end(),
                          [&](const Rep::Leaf& x, const Rep::Leaf& y) { return T.off[x.c] < T.off[y.c]; });
                int cols = 0;
                for (auto& lf : rep.leaves) {
                    lf.col = cols;
                    cols += lf.width;
                }
                rep.ld = std::max(1, rows[i]);
                rep.p = R.dalloc((size_t)rep.ld * std::max(1, cols));
                int ro = 0;
                for (int ia = 0; ia < 2; ++ia) {
                    const int a = ia ? a2 : a1;
                    for (auto& lf : rep.leaves) {
                        const int jb = is_desc(Tree::child(r, 0), lf.c) ? 0 : 1;
                        int b = Tree::child(r, jb);
                        int nb = G.kid(n, ia, jb);
                        Chain ch;
                        ch.rows = Qn.rank[a];
                        ch.dst = rep.p + ro + (size_t)lf.col * rep.ld;
                        ch.ldd = rep.ld;
                        ch.f0 = (int)pool.f.size();
                        int src_c;
                        bool src_adm;
                        if (G.kind(nb) == ADM) {
                            ch.src = mv(out.Rt.p[a], std::max(1, Qn.rank[a]));
                            ch.cols0 = Q.rank[a];
                            pool.f.push_back(G.C(nb));
                            pool.fcols.push_back(QW.rank[b]);
                            src_c = b;
                            src_adm = true;
                        } else {
                            const Rep& cr = A[nb];
                            const Rep::Leaf* sl = nullptr;
                            for (auto& x : cr.leaves)
                                if (is_desc(x.c, lf.c)) sl = &x;
                            if (!sl) throw Error(H2_ERR_UNSUPPORTED, "column tree mismatch");
                            ch.src = mv(cr.p + (size_t)sl->col * cr.ld, cr.ld);
                            ch.cols0 = sl->width;
                            src_c = sl->c;
                            src_adm = sl->adm;
                        }
                        // split admissible representations down to the target leaf: A F^*
                        path.clear();
                        for (int c = lf.c; c != src_c; c = Tree::parent(c)) path.push_back(c);
                        std::reverse(path.begin(), path.end());
                        for (int c : path) {
                            pool.f.push_back(mvT(QW.tr[c], std::max(1, QW.rank[c])));
                            pool.fcols.push_back(QW.rank[c]);
                        }
                        if (src_adm && !lf.adm) {  // expand with the leaf basis: A W^*
                            pool.f.push_back(mvT(QW.leaf[lf.c], (int)T.size[lf.c]));
                            pool.fcols.push_back((int)T.size[lf.c]);
                        }
                        ch.nf = (int)pool.f.size() - ch.f0;
                        if (ch.rows > 0) {
                            chains.push_back(ch);
                        } else {  // an empty chain leaves its factors unused
                            pool.f.resize(ch.f0);
                            pool.fcols.resize(ch.f0);
                        }
                    }
                    ro += Qn.rank[a];
                }
                Ahat[n] = std::move(rep);
            }
        }
        R.flush_gemm();
        lap.mark("cr:reps");
        run_chains(R, chains, pool);
        lap.mark("cr:chains");
        // condensed matrices (transposed): [Z_t V^*; w G_tr^* ...]; SVD
        int* d_counts = (int*)R.dalloc(nl);
        H2_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(int) * nl, R.stream()));
        SvdBatch sb(R);
        std::vector<int> has(nl, 0);
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i;
            int ncol = Zt.rows[t];
            for (int n : nodes[i]) {
                if (leaf) ncol += (int)T.size[G.other(n)];
                else {
                    auto& rp = Ahat[n];
                    for (auto& lf : rp.leaves) ncol += lf.width;
                }
            }
            if (ncol == 0 || rows[i] == 0) {
                sb.add(nullptr, 0, 0, eps, d_counts + i);
                continue;
            }
            has[i] = 1;
            double* Ct = R.dalloc((size_t)ncol * rows[i]);
            if (Zt.rows[t] > 0) {
                R.job(Ct, Zt.rows[t], rows[i], ncol, 0.0);
                if (leaf)
                    R.term(Zt.p[t], 0, Zt.rows[t], Q.leaf[t], 1, rows[i], Q.rank[t]);
                else
                    R.term(Zt.p[t], 0, Zt.rows[t], Vh[i], 1, std::max(1, rows[i]), Q.rank[t]);
            }
            int o = Zt.rows[t];
            for (int n : nodes[i]) {
                if (leaf) {
                    int r = G.other(n);
                    Mv d = G.D(n);
                    R.copy(d.p, d.ld, Ct + o, ncol, (int)T.size[r], rows[i], d.tr ^ 1, 1.0, w + cmap[n]);
                    o += (int)T.size[r];
                } else {
                    auto& rp = Ahat[n];
                    int wdt = 0;
                    for (auto& lf : rp.leaves) wdt += lf.width;
                    R.copy(rp.p, rp.ld, Ct + o, ncol, wdt, rows[i], 1, 1.0, w + cmap[n]);
                    o += wdt;
                }
            }
            sb.add(Ct, ncol, rows[i], eps, d_counts + i);
        }
        lap.mark("cr:condensed");
        std::vector<SvdOut> so = sb.run();
        lap.mark("cr:svd");
        std::vector<int> kk = read_counts(R, d_counts, nl);
        lap.mark("cr:sync");
        size_t need = 0;
        for (int i = 0; i < nl; ++i) {
            Qn.rank[c0 + i] = (so[i].U ? kk[i] : 0);
            need += (size_t)rows[i] * Qn.rank[c0 + i];
        }
        auto chunk = std::make_shared<DevBuf>();
        chunk->alloc(std::max<size_t>(need, 1));
        Qn.chunks.push_back(chunk);
        size_t off = 0;
        Carve trc(Qn, leaf ? 0 : transfer_need(Qn, c0, nl));  // the children's transfers of this level
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i, kt = Qn.rank[t];
            double* q = chunk->p + off;
            off += (size_t)rows[i] * kt;
            if (kt > 0) R.copy(so[i].U, so[i].ldu, q, rows[i], rows[i], kt, 0);
            if (leaf) {
                Qn.leaf[t] = q;
            } else {
                int o = 0;
                for (int a : {Tree::child(t, 0), Tree::child(t, 1)}) {
                    double* tp = trc.take((size_t)Qn.rank[a] * kt);
                    Qn.tr[a] = tp;
                    if (kt > 0) R.copy(so[i].U + o, so[i].ldu, tp, std::max(1, Qn.rank[a]), Qn.rank[a], kt, 0);
                    o += Qn.rank[a];
                }
            }
            // basis change R_t = Q'^* V, kept for the level above and the final couplings
            out.Rt.rows[t] = kt;
            out.Rt.cols[t] = Q.rank[t];
            out.Rt.p[t] = R.palloc((size_t)std::max(1, kt * Q.rank[t]));
        }
        R.flush_copy();
        lap.mark("cr:basis");
        for (int i = 0; i < nl; ++i) {
            int t = c0 + i, kt = Qn.rank[t];
            double* q = (leaf ? Qn.leaf[t] : nullptr);
            const double* U = so[i].U;
            int ldu = so[i].ldu;
            if (leaf) {
                U = q;
                ldu = rows[i];
            }
            // R_t = Q'^* V (Q_t at leaves, V-hat above)
            R.job(out.Rt.p[t], kt, Q.rank[t], std::max(1, kt), 0.0);
            if (kt > 0) {
                if (leaf)
                    R.term(U, 1, ldu, Q.leaf[t], 0, rows[i], rows[i]);
                else
                    R.term(U, 1, ldu, Vh[i], 0, std::max(1, rows[i]), rows[i]);
            }
            for (int n : nodes[i]) {
                Rep rep;
                rep.ld = std::max(1, kt);
                if (leaf) {
                    int r = G.other(n);
                    rep.leaves.push_back(Rep::Leaf{r, false, 0, (int)T.size[r]});
                    rep.p = pp[l & 1]->alloc((size_t)rep.ld * T.size[r]);
                    R.job(rep.p, kt, (int)T.size[r], rep.ld, 0.0);
                    if (kt > 0) T_(R, mvT(U, ldu), G.D(n), rows[i]);
                } else {
                    Rep& ah = Ahat[n];
                    int cols = 0;
                    for (auto& lf : ah.leaves) cols += lf.width;
                    rep.leaves = std::move(ah.leaves);
                    rep.p = pp[l & 1]->alloc((size_t)rep.ld * std::max(1, cols));
                    R.job(rep.p, kt, cols, rep.ld, 0.0);
                    if (kt > 0) R.term(U, 1, ldu, ah.p, 0, ah.ld, rows[i]);
                    ah = Rep{};
                }
                A[n] = std::move(rep);
            }
        }
        R.flush_gemm();
        // the representations of the level below are consumed
        if (l < T.L) {
            for (int c = Tree::first(l + 1); c < Tree::first(l + 1) + Tree::count(l + 1); ++c)
                for (int n : G.row_list(c)) A[n] = Rep{};
            pp[(l + 1) & 1]->release_all();
        }
        R.release(mkl);
        lap.mark("cr:project");
    }
    R.release(mk0);
    return out;
}

// ------------------------------------------------------------------ final couplings on the target block tree
// S'_tr = Q'_t^* G|_{t x r} Q'^W_r by upward accumulation over the T^XY subtree
// of every admissible target block:
//   admissible T^XY leaf: R_t S_tr R^W_r^*,  dense leaf: Q'_t^* D Q'^W_r,
//   split node: sum over children E'_a^* Up_ab F'_b.
static std::vector<double*> final_couplings(Runner& R, const Intermediate& G, const Tree& T,
                                            const std::vector<int>& cmap, const Coarse& rb, const Coarse& cb,
                                            const BlockTree& Zb, Counts& cnt) {
    H2_SPAN("final_couplings");
    const BlockTree& N = G.PT->nodes;
    const int nn = (int)N.kind.size();
    const Basis& Qn = *rb.Qn;
    const Basis& Wn = *cb.Qn;
    const Basis& Q = *G.Q;
    const Basis& QW = *G.QW;
    std::vector<double*> Up(nn, nullptr), m1v(nn, nullptr);
    Arena pp0(R.stream()), pp1(R.stream());  // Up of two consecutive levels
    Arena* pp[2] = {&pp0, &pp1};
    for (int l = T.L; l >= 0; --l) {
        const Arena::Mark mkl = R.mark();
        std::vector<int> lv;
        for (int n = 0; n < nn; ++n)
            if (cmap[n] >= 0 && Tree::level(N.t[n]) == l) lv.push_back(n);
        std::vector<double*>& m1 = m1v;  // ADM/DENSE: node -> first factor; SPLIT: child -> Up F'
        for (int n : lv) {
            int t = N.t[n], r = N.s[n];
            int kt = Qn.rank[t], kr = Wn.rank[r];
            if (N.kind[n] == ADM) {
                double* m = R.dalloc((size_t)std::max(1, kt * QW.rank[r]));
                R.job(m, kt, QW.rank[r], std::max(1, kt), 0.0);
                R.term(rb.Rt.p[t], 0, std::max(1, kt), G.C[n], 0, std::max(1, Q.rank[t]), Q.rank[t]);
                m1[n] = m;
                cnt.flops += 2.0 * kt * QW.rank[r] * Q.rank[t];
            } else if (N.kind[n] == DENSE) {
                double* m = R.dalloc((size_t)std::max(1, kt) * T.size[r]);
                R.job(m, kt, (int)T.size[r], std::max(1, kt), 0.0);
                R.term(Qn.leaf[t], 1, (int)T.size[t], G.C[n], 0, (int)T.size[t], (int)T.size[t]);
                m1[n] = m;
                cnt.flops += 2.0 * kt * T.size[r] * T.size[t];
            } else {
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        int a = Tree::child(t, i), b = Tree::child(r, j);
                        int c = G.PT->nodes.kids[n][2 * i + j];
                        double* m = R.dalloc((size_t)std::max(1, Qn.rank[a] * kr));
                        R.job(m, Qn.rank[a], kr, std::max(1, Qn.rank[a]), 0.0);
                        R.term(Up[c], 0, std::max(1, Qn.rank[a]), Wn.tr[b], 0, std::max(1, Wn.rank[b]), Wn.rank[b]);
                        m1[c] = m;
                        cnt.flops += 2.0 * Qn.rank[a] * kr * Wn.rank[b];
                    }
            }
        }
        R.flush_gemm();
        for (int n : lv) {
            int t = N.t[n], r = N.s[n];
            int kt = Qn.rank[t], kr = Wn.rank[r];
            // the couplings of the target blocks themselves outlive this function
            const bool root = (Zb.find(t, r) == cmap[n]);
            Up[n] = root ? R.palloc((size_t)std::max(1, kt * kr)) : pp[l & 1]->alloc((size_t)std::max(1, kt * kr));
            R.job(Up[n], kt, kr, std::max(1, kt), 0.0);
            if (N.kind[n] == ADM) {
                R.term(m1[n], 0, std::max(1, kt), cb.Rt.p[r], 1, std::max(1, kr), QW.rank[r]);
                cnt.flops += 2.0 * kt * kr * QW.rank[r];
            } else if (N.kind[n] == DENSE) {
                R.term(m1[n], 0, std::max(1, kt), Wn.leaf[r], 0, (int)T.size[r], (int)T.size[r]);
                cnt.flops += 2.0 * kt * kr * T.size[r];
            } else {
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        int a = Tree::child(t, i), b = Tree::child(r, j);
                        int c = G.PT->nodes.kids[n][2 * i + j];
                        R.term(Qn.tr[a], 1, std::max(1, Qn.rank[a]), m1[c], 0, std::max(1, Qn.rank[a]), Qn.rank[a]);
                        cnt.flops += 2.0 * kt * kr * Qn.rank[a];
                    }
            }
        }
        R.flush_gemm();
        if (l < T.L) pp[(l + 1) & 1]->release_all();
        R.release(mkl);
    }
    return Up;
}

// ------------------------------------------------------------------ matrix-vector product
// y = A x for a (possibly transposed) view: forward transformation of x
// through the column basis, couplings, backward transformation through the
// row basis, dense blocks (Sec. 2: O(nk) work per vector).
static void matvec(const h2_matrix* M, bool trans, const double* x, double* y, int64_t nv, cudaStream_t st) {
    const OpView A{M, trans};
    const Tree& T = A.tree();
    const Basis& V = A.rowb();
    const Basis& W = A.colb();
    const int64_t n = T.n;
    const int w = (int)nv;
    Runner R(st, H2_FP64);
    int64_t* d_perm = R.upload(T.perm);
    double* xt = R.dalloc((size_t)n * nv);
    double* yt = R.dalloc((size_t)n * nv);
    launch_permute_rows(x, n, xt, n, d_perm, n, nv, 0, st);
    std::vector<double*> xh(T.nc), yh(T.nc);
    for (int c = 0; c < T.nc; ++c) {
        xh[c] = R.dalloc((size_t)std::max(1, W.rank[c]) * nv);
        yh[c] = R.dalloc((size_t)std::max(1, V.rank[c]) * nv);
    }
    // forward: x_s = W_s^* x|_s at leaves, sum_c F_c^* x_c above
    for (int c = Tree::first(T.L); c < T.nc; ++c) {
        R.job(xh[c], W.rank[c], w, std::max(1, W.rank[c]), 0.0);
        R.term(W.leaf[c], 1, (int)T.size[c], xt + T.off[c], 0, (int)n, (int)T.size[c]);
    }
    R.flush_gemm();
    for (int l = T.L - 1; l >= 0; --l) {
        for (int p = Tree::first(l); p < Tree::first(l) + Tree::count(l); ++p) {
            R.job(xh[p], W.rank[p], w, std::max(1, W.rank[p]), 0.0);
            for (int i = 0; i < 2; ++i) {
                int c = Tree::child(p, i);
                R.term(W.tr[c], 1, std::max(1, W.rank[c]), xh[c], 0, std::max(1, W.rank[c]), W.rank[c]);
            }
        }
        R.flush_gemm();
    }
    // couplings: y_t = sum_s S_ts x_s
    for (int t = 0; t < T.nc; ++t) {
        R.job(yh[t], V.rank[t], w, std::max(1, V.rank[t]), 0.0);
        for (int b : A.row_list(t))
            if (A.kind(b) == ADM) T_(R, A.S(b), mv(xh[A.other(b)], std::max(1, W.rank[A.other(b)])), W.rank[A.other(b)]);
    }
    R.flush_gemm();
    // backward: y_c += E_c y_p, level by level from the root
    for (int l = 1; l <= T.L; ++l) {
        for (int c = Tree::first(l); c < Tree::first(l) + Tree::count(l); ++c) {
            int p = Tree::parent(c);
            R.job(yh[c], V.rank[c], w, std::max(1, V.rank[c]), 1.0);
            R.term(V.tr[c], 0, std::max(1, V.rank[c]), yh[p], 0, std::max(1, V.rank[p]), V.rank[p]);
        }
        R.flush_gemm();
    }
    // leaves: y|_t = V_t y_t + sum_s N_ts x|_s
    for (int t = Tree::first(T.L); t < T.nc; ++t) {
        R.job(yt + T.off[t], (int)T.size[t], w, (int)n, 0.0);
        R.term(V.leaf[t], 0, (int)T.size[t], yh[t], 0, std::max(1, V.rank[t]), V.rank[t]);
        for (int b : A.row_list(t))
            if (A.kind(b) == DENSE) {
                int s = A.other(b);
                T_(R, A.N(b), mv(xt + T.off[s], (int)n), (int)T.size[s]);
            }
    }
    R.flush_gemm();
    launch_permute_rows(yt, n, y, n, d_perm, n, nv, 1, st);
    H2_CUDA(cudaGetLastError());
    H2_CUDA(cudaStreamSynchronize(st));
    R.release_all();
    H2_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ spectral error of a product
// eps_2 of Sec. 7: the relative spectral error ||Zr - (Z0 + X Y)||_2 / ||Z0 + X Y||_2
// of a computed product Zr, both spectral norms by power iteration on the
// normal operator (x <- A^* A x / ||A^* A x||, estimate ||A x|| for the last
// unit x), every application through H^2 matrix-vector products of the four
// operands (no dense matrix is formed).
static void product_error(const h2_matrix* Zr, const h2_matrix* Z0, const h2_matrix* X, const h2_matrix* Y,
                          const double* x0_host, int steps, cudaStream_t st, double* eps2, double* normp) {
    const int64_t n = X->st->tree.n;
    Runner R(st, H2_FP64);
    double* x = R.dalloc((size_t)n);
    double* y = R.dalloc((size_t)n);
    double* t1 = R.dalloc((size_t)n);
    double* t2 = R.dalloc((size_t)n);
    double* acc = R.dalloc(1);
    std::vector<double> h0((size_t)n);
    for (int64_t i = 0; i < n; ++i) h0[i] = x0_host ? x0_host[i] : 1.0 + 0.37 * (double)i / (double)n;
    H2_CUDA(cudaMemcpyAsync(x, h0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    constexpr int64_t kPart = 65536;  // vector pieces, one CTA each
    // dst = a src + b dst (b = 0: dst = a src)
    auto axpby = [&](double* dst, const double* src, double a, double b) {
        for (int64_t o = 0; o < n; o += kPart) {
            const int len = (int)std::min(kPart, n - o);
            R.copy(src + o, len, dst + o, len, len, 1, 0, a, nullptr, b);
        }
        R.flush_copy();
    };
    auto norm2 = [&](const double* v) {
        std::vector<SumSqJob> jobs;
        for (int64_t o = 0; o < n; o += kPart) {
            const int len = (int)std::min(kPart, n - o);
            jobs.push_back(SumSqJob{v + o, len, 1, len, 0});
        }
        const std::vector<int> seg = sumsq_segments(jobs, 1);
        double* part = R.dalloc(std::max<size_t>(jobs.size(), 1));
        launch_sumsq(R.upload(jobs), (int)jobs.size(), part, R.upload(seg), 1, acc, st);
        double h = 0.0;
        H2_CUDA(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
        H2_CUDA(cudaStreamSynchronize(st));
        return std::sqrt(h);
    };
    // out = P in (or P^* in), P = Z0 + X Y; with err: out = Zr in - P in
    auto apply = [&](bool err, bool trans, const double* in, double* out) {
        matvec(trans ? X : Y, trans, in, t1, 1, st);
        matvec(trans ? Y : X, trans, t1, t2, 1, st);
        matvec(Z0, trans, in, out, 1, st);
        axpby(out, t2, 1.0, 1.0);
        if (err) {
            matvec(Zr, trans, in, t1, 1, st);
            axpby(out, t1, 1.0, -1.0);
        }
    };
    double* start = R.dalloc((size_t)n);
    axpby(start, x, 1.0, 0.0);
    auto power = [&](bool err) {
        axpby(x, start, 1.0, 0.0);
        double nx = norm2(x), est = 0.0;
        for (int it = 0; it < steps && nx > 0.0; ++it) {
            axpby(x, x, 1.0 / nx, 0.0);
            apply(err, false, x, y);
            est = norm2(y);
            if (est == 0.0) break;
            apply(err, true, y, x);
            nx = norm2(x);
        }
        return est;
    };
    const double p = power(false);
    const double e = power(true);
    *normp = p;
    *eps2 = p > 0.0 ? e / p : 0.0;
    R.release_all();
    H2_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ driver
// The product block tree depends only on the two block trees: kept on the
// structure of X, keyed by the fingerprint of Y's structure.
static const ProductTree& cached_product_tree(Structure& xs, const Structure& ys) {
    H2_SPAN("cached_product_tree");
    std::lock_guard<std::mutex> g(xs.plan_mutex);
    auto it = xs.product_trees.find(ys.fingerprint);
    if (it == xs.product_trees.end())
        it = xs.product_trees.emplace(ys.fingerprint, std::make_shared<ProductTree>(build_product_tree(xs.blocks, ys.blocks)))
                 .first;
    return *it->second;
}

static bool same_row_basis(const h2_matrix* A, const h2_matrix* B) {
    // A's row basis equals B's row basis: the same object, or Chebyshev bases of
    // the same structure and order (they are equal by construction)
    if (A->V == B->V) return true;
    return A->order > 0 && A->order == B->order && A->st->fingerprint == B->st->fingerprint && A->vtag == B->vtag;
}
static bool same_col_basis(const h2_matrix* A, const h2_matrix* B) {
    if (A->W == B->W) return true;
    return A->order > 0 && A->order == B->order && A->st->fingerprint == B->st->fingerprint && A->wtag == B->wtag;
}

// A second stream with its own host thread: the row and column sides of each
// phase are independent, so the column side runs beside the row side and the
// host work of one overlaps the device work of the other.  Used in the
// low-precision forms, whose device work per level is shorter than the host
// work between the level synchronisations; the FP64 form is bound by the
// device and runs the sides in order on one stream.
struct SideStream {
    cudaStream_t s = nullptr;
    SideStream() : s(stream_get()) {}
    ~SideStream() {
        if (s) {
            cudaStreamSynchronize(s);
            stream_put(s);
        }
    }
};

// `waiter` runs its later work after everything queued so far on `signaller`
static void stream_after(cudaStream_t waiter, cudaStream_t signaller) {
    cudaEvent_t e;
    H2_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    H2_CUDA(cudaEventRecord(e, signaller));
    H2_CUDA(cudaStreamWaitEvent(waiter, e, 0));
    H2_CUDA(cudaEventDestroy(e));
}

// runs f on a host thread (current device, the caller's device-memory source
// with stream st) and joins in join() or the destructor
class Beside {
public:
    template <class F>
    Beside(cudaStream_t st, F&& f) {
        int dev = 0;
        H2_CUDA(cudaGetDevice(&dev));
        const DevAlloc src = current_alloc();
        Combiner* comb = current_combiner();
        if (comb) comb->enter();  // before the thread starts: the combiner must count it
        th_ = std::thread([this, dev, src, st, comb, f = std::forward<F>(f)]() mutable {
            CombinerScope cs(comb);
            struct Leave {
                Combiner* c;
                ~Leave() {
                    if (c) c->leave();
                }
            } leave{comb};
            try {
                H2_CUDA(cudaSetDevice(dev));
                AllocScope scope(src, st);
                f();
            } catch (...) {
                err_ = std::current_exception();
            }
        });
    }
    void join() {
        CombIdle idle(current_combiner());
        if (th_.joinable()) th_.join();
        if (err_) {
            std::exception_ptr e = err_;
            err_ = nullptr;
            std::rethrow_exception(e);
        }
    }
    ~Beside() {
        if (th_.joinable()) th_.join();
    }

private:
    std::thread th_;
    std::exception_ptr err_;
};

// Phase B (Sec. 6) and the final couplings for an intermediate H^2-matrix G with
// isometric bases on a block tree that refines the target block tree Zb:
// block weights, coarsened row and column bases (Fig. 7, the two sides beside
// each other in the low-precision forms), final couplings, and the result on Zb
// in persistent memory.  Used by the product and by the recompression.
struct PhaseB {
    std::unique_ptr<h2_matrix> res;
    Coarse rb, cb;
    int nodes = 0;
};

static PhaseB coarsen_and_project(Runner& R, Runner& R2, cudaStream_t st, SideStream& side, bool beside,
                                  const Tree& T, const BlockTree& Zb, const h2_matrix* Zm, Intermediate& G,
                                  double eps, Counts& cnt, PhaseClock& clk, PhaseClock& clk2) {
    H2_SPAN("coarsen_and_project");
    // phase B: coarsening to Z's block tree
    const BlockTree& N = G.PT->nodes;
    const int nn = (int)N.kind.size();
    std::vector<int> cmap(nn, -1);
    {
        std::vector<int> stack{N.find(0, 0)};
        std::vector<int> inh(nn, -1);
        while (!stack.empty()) {
            int n = stack.back();
            stack.pop_back();
            int b = inh[n];
            if (b < 0) {
                int zb = Zb.find(N.t[n], N.s[n]);
                if (zb >= 0 && Zb.kind[zb] == ADM) b = zb;
            }
            cmap[n] = b;
            if (N.kind[n] == SPLIT)
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        int c = N.find(Tree::child(N.t[n], i), Tree::child(N.s[n], j));
                        inh[c] = b;
                        stack.push_back(c);
                    }
        }
    }
    // block weights 1 / ||G|_b||_F over the T^XY leaves of each admissible target block
    double* sq = R.dalloc(std::max<size_t>(Zb.kind.size(), 1));
    double* w = R.dalloc(std::max<size_t>(Zb.kind.size(), 1));
    double* w2 = R.dalloc(std::max<size_t>(Zb.kind.size(), 1));
    H2_CUDA(cudaMemsetAsync(sq, 0, sizeof(double) * std::max<size_t>(Zb.kind.size(), 1), st));
    {
        std::vector<SumSqJob> jobs;
        for (int n = 0; n < nn; ++n) {
            if (cmap[n] < 0 || N.kind[n] == SPLIT) continue;
            int t = N.t[n], r = N.s[n];
            if (N.kind[n] == ADM)
                jobs.push_back(SumSqJob{G.C[n], G.Q->rank[t], G.QW->rank[r], std::max(1, G.Q->rank[t]), cmap[n]});
            else
                jobs.push_back(SumSqJob{G.C[n], (int)T.size[t], (int)T.size[r], (int)T.size[t], cmap[n]});
        }
        const std::vector<int> seg = sumsq_segments(jobs, (int)Zb.kind.size());
        SumSqJob* dj = R.upload(jobs);
        const int* dseg = R.upload(seg);
        double* part = R.dalloc(std::max<size_t>(jobs.size(), 1));
        R.begin(9);
        launch_sumsq(dj, (int)jobs.size(), part, dseg, (int)Zb.kind.size(), sq, st);
        launch_inv_sqrt(sq, w, w2, (int)Zb.kind.size(), st);
        R.end(9, 0.0, 0.0);
        R.launches += 3;
    }
    GView GR{&G, &T, false}, GC{&G, &T, true};
    PhaseB out;
    Coarse& rb = out.rb;
    Coarse& cb = out.cb;
    if (beside) {
        stream_after(side.s, st);
        clk2.mark();
        Beside col(R2.stream(), [&] { cb = coarsen_rows(R2, GC, cmap, w, w2, eps); });
        rb = coarsen_rows(R, GR, cmap, w, w2, eps);
        clk.mark();
        col.join();
    } else {
        rb = coarsen_rows(R, GR, cmap, w, w2, eps);
        clk.mark();
        stream_after(side.s, st);
        clk2.mark();
        cb = coarsen_rows(R2, GC, cmap, w, w2, eps);
    }
    clk2.mark();
    stream_after(st, side.s);
    std::vector<double*> Up = final_couplings(R, G, T, cmap, rb, cb, Zb, cnt);
    // assemble the result on Z's block tree in persistent memory
    auto res = std::make_unique<h2_matrix>();
    res->st = Zm->st;
    res->V = rb.Qn;
    res->W = cb.Qn;
    res->kernel = -1;
    res->order = 0;
    res->device = Zm->device;
    res->blk.assign(Zb.kind.size(), nullptr);
    size_t tot = 0;
    for (int b = 0; b < (int)Zb.kind.size(); ++b) {
        int t = Zb.t[b], s = Zb.s[b];
        if (Zb.kind[b] == ADM) tot += (size_t)rb.Qn->rank[t] * cb.Qn->rank[s];
        if (Zb.kind[b] == DENSE) tot += (size_t)T.size[t] * T.size[s];
    }
    auto chunk = std::make_shared<DevBuf>();
    chunk->alloc(std::max<size_t>(tot, 1));
    res->chunks.push_back(chunk);
    size_t o = 0;
    for (int b = 0; b < (int)Zb.kind.size(); ++b) {
        int t = Zb.t[b], s = Zb.s[b];
        int n = N.find(t, s);
        if (Zb.kind[b] == ADM) {
            int kt = rb.Qn->rank[t], ks = cb.Qn->rank[s];
            res->blk[b] = chunk->p + o;
            o += (size_t)kt * ks;
            R.copy(Up[n], std::max(1, kt), res->blk[b], std::max(1, kt), kt, ks, 0);
        } else if (Zb.kind[b] == DENSE) {
            res->blk[b] = chunk->p + o;
            o += (size_t)T.size[t] * T.size[s];
            R.copy(G.C[n], (int)T.size[t], res->blk[b], (int)T.size[t], (int)T.size[t], (int)T.size[s], 0);
        }
    }
    R.flush_copy();
    R.ensure_flag();
    R.begin(9);
    launch_check_finite(chunk->p, chunk->len, R.svd_flag(), st);
    R.end(9, 0.0, 8.0 * chunk->len);
    R.launches++;
    out.nodes = nn;
    out.res = std::move(res);
    return out;
}

static void mul_add(h2_matrix* Zm, const h2_matrix* Xm, const h2_matrix* Ym, const h2_opts* opts) {
    H2_SPAN("mul_add");
    const double eps = opts ? opts->eps : 1e-6;
    const int prec = resolve_precision(opts ? opts->precision : H2_FP64, eps);
    cudaStream_t st = stream_of(opts);
    AllocScope scope(alloc_of(opts), st);
    auto t_host0 = std::chrono::steady_clock::now();
    SideStream side;
    Runner R(st, prec);
    Runner R2(side.s, prec);  // column sides; its outputs live until the end of the call
    const bool tune = opts && opts->autotune;
    R.set_autotune(tune);
    R2.set_autotune(tune);
    const bool beside = low_precision(prec);
    PhaseClock clk(st), clk2(side.s);
    Counts cnt, cnt2;
    const OpView X{Xm, false}, Y{Ym, false};
    const Tree& T = X.tree();
    clk.mark();
    // The plan of T^XY (host work, cached per pair of structures) is built on a host
    // thread of its own beside phase A, which needs none of it; t_mat waits for it.
    std::future<const ProductTree*> plan =
        std::async(std::launch::async, [Xm, Ym] { return &cached_product_tree(*Xm->st, *Ym->st); });
    // phase A: compressed induced row and column bases (prep included)
    const OpView Yt{Ym, true}, Xt{Xm, true};
    // "+Z" with bases of its own: V_Z (W_Z) preserved beside V_X (W_Y) in phase A
    const Basis* VZ = same_row_basis(Zm, Xm) ? nullptr : Zm->V.get();
    const Basis* WZ = same_col_basis(Zm, Ym) ? nullptr : Zm->W.get();
    Induced ra, ca;
    if (beside) {
        stream_after(side.s, st);
        clk2.mark();
        Beside col(R2.stream(), [&] { ca = induced_rows(R2, Yt, Xt, eps, cnt2, WZ); });
        ra = induced_rows(R, X, Y, eps, cnt, VZ);
        clk.mark();
        col.join();
    } else {
        ra = induced_rows(R, X, Y, eps, cnt, VZ);
        clk.mark();
        stream_after(side.s, st);
        clk2.mark();
        ca = induced_rows(R2, Yt, Xt, eps, cnt2, WZ);
    }
    clk2.mark();
    stream_after(st, side.s);
    // the intermediate H^2-matrix on T^XY
    Intermediate G;
    G.PT = plan.get();
    G.Q = ra.Q;
    G.QW = ca.Q;
    const BlockTree& Zb = Zm->st->blocks;
    for (int b = 0; b < (int)Zb.kind.size(); ++b) {
        int n = G.PT->nodes.find(Zb.t[b], Zb.s[b]);
        if (n < 0 || (Zb.kind[b] == DENSE && G.PT->nodes.kind[n] != DENSE))
            throw Error(H2_ERR_UNSUPPORTED, "the product block tree does not refine Z's block tree");
    }
    induced_matrix(R, X, Y, Zm, ra, ca, G, cnt);
    clk.mark();
    PhaseB pb = coarsen_and_project(R, R2, st, side, beside, T, Zb, Zm, G, eps, cnt, clk, clk2);
    const int nn = pb.nodes;
    const Coarse& rb = pb.rb;
    const Coarse& cb = pb.cb;
    auto& res = pb.res;
    clk.mark();
    int* hf = (int*)R.pinned_host(3 * sizeof(int));  // pinned: the copies stay asynchronous
    hf[0] = hf[1] = hf[2] = 0;
    H2_CUDA(cudaMemcpyAsync(hf, R.svd_flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    if (R2.svd_flag()) H2_CUDA(cudaMemcpyAsync(hf + 1, R2.svd_flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    if (R.combiner() && R.combiner()->flag())  // grouped launches of a batched call
        H2_CUDA(cudaMemcpyAsync(hf + 2, R.combiner()->flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaGetLastError());
    {
        CombIdle idle(R.combiner());
        H2_CUDA(cudaStreamSynchronize(st));
    }
    const int flag = hf[0] | hf[1] | hf[2];
    if (flag & 2) throw Error(H2_ERR_NUMERIC, "non-finite value in the result");
    if (flag & 4) throw Error(H2_ERR_TIMEOUT, "tensor-core product wait timed out");
    if (flag & 1) throw Error(H2_ERR_TIMEOUT, "Jacobi SVD did not converge within its sweep limit");
    if (opts && opts->stats) {
        h2_stats* S = opts->stats;
        S->t_prep_ms = 0.0;
        // row and column sides run concurrently: their intervals overlap
        S->t_rows_a_ms = clk.ms(0);
        S->t_cols_a_ms = clk2.ms(0);
        S->t_mat_a_ms = clk.ms(1);
        S->t_rows_b_ms = clk.ms(2);
        S->t_cols_b_ms = clk2.ms(2);
        S->t_mat_b_ms = clk.ms(3);
        S->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
        S->kernel_launches = R.launches + R2.launches;
        S->product_nodes = nn;
        S->triples = cnt.triples + cnt2.triples;
        S->max_rank_a = std::max(ra.Q->max_rank(), ca.Q->max_rank());
        S->max_rank_b = std::max(rb.Qn->max_rank(), cb.Qn->max_rank());
        S->flops = cnt.flops + cnt2.flops;
        S->bytes_moved = cnt.bytes + cnt2.bytes;
        for (int f = 0; f < 12; ++f) {
            S->fam_ms[f] = 0.0;
            S->fam_launches[f] = 0;
            S->fam_flops[f] = 0.0;
            S->fam_bytes[f] = 0.0;
        }
        {
            cudaEvent_t ref = R.first_event();
            R.collect(S->fam_ms, S->fam_launches, S->fam_flops, S->fam_bytes);
            R2.collect(S->fam_ms, S->fam_launches, S->fam_flops, S->fam_bytes, ref);
        }
    } else if (opts && opts->autotune) {  // the tuner learns from the launch times
        R.collect(nullptr, nullptr, nullptr, nullptr);
        R2.collect(nullptr, nullptr, nullptr, nullptr);
    }
    R.release_all();
    R2.release_all();
    {
        CombIdle idle(R.combiner());
        H2_CUDA(cudaStreamSynchronize(st));
    }
    // swap the result into Z (X and Y may alias Z; they are no longer read)
    Zm->V = res->V;
    Zm->W = res->W;
    Zm->blk = std::move(res->blk);
    Zm->chunks = std::move(res->chunks);
    Zm->kernel = -1;
    Zm->order = 0;
}

// ------------------------------------------------------------------ recompression
// Fig. 1 with the isometric factors kept: B_t = Q_t R_t with Q nested and
// isometric.  Leaves: thin QR of B_t with the explicit factor; parents: thin QR
// of the stacked R_{t'} E_{t'}, whose isometric factor splits row-wise into the
// children's transfer matrices.  Rf[t] (rank_Q(t) x rank_B(t)) in persistent memory.
static std::shared_ptr<Basis> orthogonalize(Runner& R, const Tree& T, const Basis& B, PerCl& Rf) {
    auto Q = std::make_shared<Basis>();
    Q->rank.assign(T.nc, 0);
    Q->leaf.assign(T.nc, nullptr);
    Q->tr.assign(T.nc, nullptr);
    Rf.init(T.nc);
    size_t need = 0;
    for (int c = Tree::first(T.L); c < T.nc; ++c) need += (size_t)T.size[c] * std::min<int64_t>(T.size[c], B.rank[c]);
    auto lc = std::make_shared<DevBuf>();
    lc->alloc(std::max<size_t>(need, 1));
    Q->chunks.push_back(lc);
    size_t off = 0;
    for (int c = Tree::first(T.L); c < T.nc; ++c) {
        const int m = (int)T.size[c], k = B.rank[c], q = std::min(m, k);
        Q->rank[c] = q;
        Rf.rows[c] = q;
        Rf.cols[c] = k;
        Rf.p[c] = R.palloc((size_t)std::max(1, q * k));
        if (q == 0) continue;
        Q->leaf[c] = lc->p + off;
        off += (size_t)m * q;
        double* work = R.dalloc((size_t)m * k);
        R.copy(B.leaf[c], m, work, m, m, k, 0);
        R.qr(work, m, k, m, Rf.p[c], q, Q->leaf[c], m, q);
    }
    R.flush_copy();
    R.flush_qr();
    for (int l = T.L - 1; l >= 0; --l) {
        const int c0 = Tree::first(l), nl = Tree::count(l);
        std::vector<double*> Qh(nl, nullptr);
        std::vector<int> rows(nl);
        for (int i = 0; i < nl; ++i) {
            const int p = c0 + i, c1 = Tree::child(p, 0), c2 = Tree::child(p, 1), k = B.rank[p];
            rows[i] = Q->rank[c1] + Q->rank[c2];
            const int q = std::min(rows[i], k);
            Q->rank[p] = q;
            Rf.rows[p] = q;
            Rf.cols[p] = k;
            Rf.p[p] = R.palloc((size_t)std::max(1, q * k));
            if (q == 0) continue;
            double* st = R.dalloc((size_t)rows[i] * k);
            int o = 0;
            for (int c : {c1, c2}) {
                R.job(st + o, Q->rank[c], k, rows[i], 0.0);
                R.term(Rf.p[c], 0, std::max(1, Q->rank[c]), B.tr[c], 0, std::max(1, B.rank[c]), B.rank[c]);
                o += Q->rank[c];
            }
            Qh[i] = R.dalloc((size_t)rows[i] * q);
            R.qr(st, rows[i], k, rows[i], Rf.p[p], q, Qh[i], rows[i], q);
        }
        R.flush_gemm(H2_FP64);
        R.flush_qr();
        size_t tneed = 0;
        for (int i = 0; i < nl; ++i) tneed += (size_t)rows[i] * Q->rank[c0 + i];
        auto tc = std::make_shared<DevBuf>();
        tc->alloc(std::max<size_t>(tneed, 1));
        Q->chunks.push_back(tc);
        size_t to = 0;
        for (int i = 0; i < nl; ++i) {
            const int p = c0 + i, q = Q->rank[p];
            int o = 0;
            for (int c : {Tree::child(p, 0), Tree::child(p, 1)}) {
                Q->tr[c] = tc->p + to;
                to += (size_t)std::max(0, Q->rank[c] * q);
                if (q > 0 && Q->rank[c] > 0) R.copy(Qh[i] + o, rows[i], Q->tr[c], Q->rank[c], Q->rank[c], q, 0);
                o += Q->rank[c];
            }
        }
        R.flush_copy();
    }
    return Q;
}

// A <- A with adaptive isometric bases at the block-relative tolerance eps:
// orthogonalized bases, couplings moved into them (S' = R_V,t S R_W,s^*), then
// the coarsening and final couplings of the product's second phase with A's own
// block tree as the tree of the intermediate matrix.
static void recompress(h2_matrix* A, const h2_opts* opts) {
    const double eps = opts ? opts->eps : 1e-6;
    const int prec = resolve_precision(opts ? opts->precision : H2_FP64, eps);
    AllocScope scope(alloc_of(opts), stream_of(opts));
    cudaStream_t st = stream_of(opts);
    auto t_host0 = std::chrono::steady_clock::now();
    SideStream side;
    Runner R(st, prec);
    Runner R2(side.s, prec);
    R.set_autotune(opts && opts->autotune);
    R2.set_autotune(opts && opts->autotune);
    PhaseClock clk(st), clk2(side.s);
    Counts cnt;
    const Tree& T = A->st->tree;
    const BlockTree& B = A->st->blocks;
    const int nb = (int)B.kind.size();
    clk.mark();
    PerCl RV, RW;
    std::shared_ptr<Basis> QV = orthogonalize(R, T, *A->V, RV);
    std::shared_ptr<Basis> QW = (A->W == A->V) ? QV : orthogonalize(R, T, *A->W, RW);
    const PerCl& RWr = (A->W == A->V) ? RV : RW;
    ProductTree plan;  // the intermediate's tree is A's own block tree
    plan.nodes = B;
    plan.triples.assign(nb, {});
    plan.tri_blocks.assign(nb, {});
    Intermediate G;
    G.PT = &plan;
    G.Q = QV;
    G.QW = QW;
    G.C.assign(nb, nullptr);
    std::vector<double*> tmp(nb, nullptr);
    for (int b = 0; b < nb; ++b) {
        if (B.kind[b] == DENSE) G.C[b] = A->blk[b];
        if (B.kind[b] != ADM) continue;
        const int t = B.t[b], s = B.s[b], kvt = A->V->rank[t], kws = A->W->rank[s], ks = QW->rank[s];
        tmp[b] = R.dalloc((size_t)std::max(1, kvt * ks));
        R.job(tmp[b], kvt, ks, std::max(1, kvt), 0.0);
        R.term(A->blk[b], 0, std::max(1, kvt), RWr.p[s], 1, std::max(1, ks), kws);
    }
    R.flush_gemm(H2_FP64);
    for (int b = 0; b < nb; ++b) {
        if (B.kind[b] != ADM) continue;
        const int t = B.t[b], s = B.s[b], kvt = A->V->rank[t], kt = QV->rank[t], ks = QW->rank[s];
        G.C[b] = R.palloc((size_t)std::max(1, kt * ks));
        R.job(G.C[b], kt, ks, std::max(1, kt), 0.0);
        R.term(RV.p[t], 0, std::max(1, kt), tmp[b], 0, std::max(1, kvt), kvt);
    }
    R.flush_gemm(H2_FP64);
    clk.mark();
    clk2.mark();
    clk2.mark();
    PhaseB pb = coarsen_and_project(R, R2, st, side, low_precision(prec), T, B, A, G, eps, cnt, clk, clk2);
    clk.mark();
    int* hf = (int*)R.pinned_host(3 * sizeof(int));  // pinned: the copies stay asynchronous
    hf[0] = hf[1] = hf[2] = 0;
    H2_CUDA(cudaMemcpyAsync(hf, R.svd_flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    if (R2.svd_flag()) H2_CUDA(cudaMemcpyAsync(hf + 1, R2.svd_flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    if (R.combiner() && R.combiner()->flag())  // grouped launches of a batched call
        H2_CUDA(cudaMemcpyAsync(hf + 2, R.combiner()->flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaGetLastError());
    {
        CombIdle idle(R.combiner());
        H2_CUDA(cudaStreamSynchronize(st));
    }
    const int flag = hf[0] | hf[1] | hf[2];
    if (flag & 2) throw Error(H2_ERR_NUMERIC, "non-finite value in the result");
    if (flag & 4) throw Error(H2_ERR_TIMEOUT, "tensor-core product wait timed out");
    if (flag & 1) throw Error(H2_ERR_TIMEOUT, "Jacobi SVD did not converge within its sweep limit");
    if (opts && opts->stats) {
        h2_stats* S = opts->stats;
        std::memset(S, 0, sizeof(h2_stats));
        S->t_rows_a_ms = clk.ms(0);  // orthogonalization and couplings
        S->t_rows_b_ms = clk.ms(1);
        S->t_cols_b_ms = clk2.ms(2);
        S->t_mat_b_ms = clk.ms(2);
        S->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
        S->kernel_launches = R.launches + R2.launches;
        S->product_nodes = nb;
        S->max_rank_a = std::max(QV->max_rank(), QW->max_rank());
        S->max_rank_b = std::max(pb.rb.Qn->max_rank(), pb.cb.Qn->max_rank());
        S->flops = cnt.flops;
        {
            cudaEvent_t ref = R.first_event();
            R.collect(S->fam_ms, S->fam_launches, S->fam_flops, S->fam_bytes);
            R2.collect(S->fam_ms, S->fam_launches, S->fam_flops, S->fam_bytes, ref);
        }
    } else if (opts && opts->autotune) {  // the tuner learns from the launch times
        R.collect(nullptr, nullptr, nullptr, nullptr);
        R2.collect(nullptr, nullptr, nullptr, nullptr);
    }
    R.release_all();
    R2.release_all();
    H2_CUDA(cudaStreamSynchronize(st));
    A->V = pb.res->V;
    A->W = pb.res->W;
    A->blk = std::move(pb.res->blk);
    A->chunks = std::move(pb.res->chunks);
    A->kernel = -1;
    A->order = 0;
    A->vtag = A->wtag = 0;
}

}  // namespace h2

void h2_set_last_error(const char* m);

static int run_guarded_mul(h2_matrix* Z, const h2_matrix* X, const h2_matrix* Y, const h2_opts* opts) {
    try {
        h2::mul_add(Z, X, Y, opts);
        h2::host_spans_dump();
        return H2_OK;
    } catch (const h2::Error& e) {
        h2_set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        h2_set_last_error("host allocation failed");
        return H2_ERR_OOM;
    } catch (const std::exception& e) {
        h2_set_last_error(e.what());
        return H2_ERR_CUDA;
    }
}

// Independent products run concurrently: worker threads, each with its own
// non-blocking stream, take products from a shared counter; the host work of
// one product overlaps the device work of the others (16 at once: 4 % more
// rows/s than 8 on the 64-product workload).
extern "C" int h2_mul_add_batched(h2_matrix* const* Z, const h2_matrix* const* X, const h2_matrix* const* Y,
                                  int count, const h2_opts* opts, int* status) {
    using namespace h2;
    if (count < 0 || (count > 0 && (!Z || !X || !Y))) return H2_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (!Z[i] || !X[i] || !Y[i]) return H2_ERR_ARG;
    if (opts && (!(opts->eps >= 0.0) || !std::isfinite(opts->eps) ||
                 !valid_precision(opts->precision)))
        return H2_ERR_ARG;
    // a Z may not appear twice, nor as an operand of another product (its swap would race)
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < count; ++j)
            if (i != j && (Z[i] == Z[j] || Z[i] == X[j] || Z[i] == Y[j])) return H2_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return H2_ERR_CUDA;
    cudaStream_t outer = stream_of(opts);
    cudaEvent_t start = nullptr;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return H2_ERR_CUDA;
    cudaEventRecord(start, outer);  // products start after the caller's earlier work
    // Grouped launches (opt-in, H2_BATCH_GROUPING=1): the GEMM batches of the
    // concurrent products share launches.  On the 64-product workload they cut the
    // launches by 44 % but lowered the throughput by 12 %: each merge waits for the
    // products' host work, which paces these products, so the default is off.
    static const bool grouping = std::getenv("H2_BATCH_GROUPING") && std::getenv("H2_BATCH_GROUPING")[0] == '1';
    // 16 concurrent products (8 with grouping) keep the GPU fed while the host
    // work and level synchronisations of each product run
    const int workers = std::max(1, std::min(count, grouping ? 8 : 16));
    std::vector<int> codes(count, H2_OK);
    std::atomic<int> next{0};
    std::vector<h2_stats> stats(count);
    cudaStream_t cst = nullptr;
    std::unique_ptr<Combiner> comb;
    if (grouping && count > 1) {
        try {
            cst = stream_get();
            AllocScope as(alloc_of(opts), cst);
            comb = std::make_unique<Combiner>(cst, resolve_precision(opts ? opts->precision : H2_FP64,
                                                                     opts ? opts->eps : 1e-6));
        } catch (const std::exception&) {
            comb.reset();
        }
    }
    const DevAlloc batch_alloc = [&] {
        try {
            return alloc_of(opts);
        } catch (const std::exception&) {
            return DevAlloc{};
        }
    }();
    std::mutex err_mu;
    std::string first_msg;  // message of the first failed product (set on the calling thread)
    auto work = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        try {
            st = stream_get();
        } catch (const std::exception&) {
            for (int i = next.fetch_add(count); i < count; ++i) codes[i] = H2_ERR_CUDA;
            return;
        }
        cudaStreamWaitEvent(st, start, 0);
        CombinerScope cs(comb.get());
        AllocScope as(batch_alloc, cst ? cst : st);  // the combiner's launches allocate on its stream
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
            h2_opts o{};
            if (opts) {
                o = *opts;
            } else {
                o.eps = 1e-6;
                o.precision = H2_FP64;
            }
            o.stream = st;
            o.stats = opts && opts->stats ? &stats[i] : nullptr;
            if (comb) comb->enter();
            codes[i] = h2_mul_add(Z[i], X[i], Y[i], &o);
            if (comb) comb->leave();
            if (codes[i] != H2_OK) {
                std::lock_guard<std::mutex> lk(err_mu);
                if (first_msg.empty()) first_msg = h2_last_error_message();
            }
        }
        cudaStreamSynchronize(st);
        stream_put(st);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w) pool.emplace_back(work);
    for (auto& t : pool) t.join();
    cudaEventDestroy(start);
    h2_stats CS{};  // the grouped launches
    if (comb) {
        cudaStreamSynchronize(cst);
        comb->runner().collect(CS.fam_ms, CS.fam_launches, CS.fam_flops, CS.fam_bytes);
        CS.kernel_launches = comb->runner().launches;
        comb.reset();
    }
    if (cst) {
        cudaStreamSynchronize(cst);
        stream_put(cst);
    }
    if (opts && opts->stats) {  // sums over the products (times: device time of each product)
        h2_stats S = CS;
        for (const h2_stats& x : stats) {
            S.t_rows_a_ms += x.t_rows_a_ms;
            S.t_cols_a_ms += x.t_cols_a_ms;
            S.t_mat_a_ms += x.t_mat_a_ms;
            S.t_rows_b_ms += x.t_rows_b_ms;
            S.t_cols_b_ms += x.t_cols_b_ms;
            S.t_mat_b_ms += x.t_mat_b_ms;
            S.t_total_ms += x.t_total_ms;
            S.kernel_launches += x.kernel_launches;
            S.product_nodes += x.product_nodes;
            S.triples += x.triples;
            S.max_rank_a = std::max(S.max_rank_a, x.max_rank_a);
            S.max_rank_b = std::max(S.max_rank_b, x.max_rank_b);
            S.flops += x.flops;
            S.bytes_moved += x.bytes_moved;
            for (int f = 0; f < 12; ++f) {
                S.fam_ms[f] += x.fam_ms[f];
                S.fam_launches[f] += x.fam_launches[f];
                S.fam_flops[f] += x.fam_flops[f];
                S.fam_bytes[f] += x.fam_bytes[f];
            }
        }
        *opts->stats = S;
    }
    int first = H2_OK;
    for (int i = 0; i < count; ++i) {
        if (status) status[i] = codes[i];
        if (first == H2_OK && codes[i] != H2_OK) first = codes[i];
    }
    if (first != H2_OK) h2_set_last_error(first_msg.c_str());
    return first;
}

extern "C" int h2_matvec(const h2_matrix* A, const double* x, double* y, int64_t nvec, int trans,
                         const h2_opts* opts) {
    if (!A || !x || !y || nvec < 1 || nvec > (1 << 20) || (trans != 0 && trans != 1)) return H2_ERR_ARG;
    try {
        h2::AllocScope scope(h2::alloc_of(opts), h2::stream_of(opts));
        h2::matvec(A, trans != 0, x, y, nvec, h2::stream_of(opts));
        return H2_OK;
    } catch (const h2::Error& e) {
        h2_set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        h2_set_last_error(e.what());
        return H2_ERR_CUDA;
    }
}

extern "C" int h2_product_error(const h2_matrix* Zr, const h2_matrix* Z0, const h2_matrix* X, const h2_matrix* Y,
                                const double* x0, int steps, const h2_opts* opts, double* eps2, double* norm) {
    using namespace h2;
    if (!Zr || !Z0 || !X || !Y || !eps2 || !norm || steps < 1 || steps > 100000) return H2_ERR_ARG;
    const uint64_t f = X->st->fingerprint;
    if (Y->st->fingerprint != f || Z0->st->fingerprint != f || Zr->st->fingerprint != f) return H2_ERR_SHAPE;
    try {
        AllocScope scope(alloc_of(opts), stream_of(opts));
        product_error(Zr, Z0, X, Y, x0, steps, stream_of(opts), eps2, norm);
        return H2_OK;
    } catch (const Error& e) {
        h2_set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        h2_set_last_error(e.what());
        return H2_ERR_CUDA;
    }
}

extern "C" int h2_block_norms(const h2_matrix* A, const h2_opts* opts, int* t, int* s, int* kind, double* norm) {
    using namespace h2;
    if (!A) return H2_ERR_ARG;
    if (opts && (!(opts->eps >= 0.0) || !std::isfinite(opts->eps) || !valid_precision(opts->precision)))
        return H2_ERR_ARG;
    try {
        const BlockTree& B = A->st->blocks;
        const Tree& T = A->st->tree;
        const int nb = (int)B.kind.size();
        for (int b = 0; b < nb; ++b) {
            if (t) t[b] = B.t[b];
            if (s) s[b] = B.s[b];
            if (kind) kind[b] = B.kind[b] == ADM ? 0 : B.kind[b] == DENSE ? 1 : 2;
        }
        if (!norm || nb == 0) return H2_OK;
        const cudaStream_t st = stream_of(opts);
        AllocScope scope(alloc_of(opts), st);
        Runner R(st, resolve_precision(opts ? opts->precision : H2_FP64, opts ? opts->eps : 1e-6));
        double* d = R.dalloc((size_t)nb);
        H2_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * nb, st));
        for (int b = 0; b < nb; ++b) {
            const int tb = B.t[b], sb = B.s[b];
            if (B.kind[b] == ADM && A->V->rank[tb] > 0 && A->W->rank[sb] > 0)
                R.norm(A->blk[b], A->V->rank[tb], A->W->rank[sb], A->V->rank[tb], nullptr, d + b);
            else if (B.kind[b] == DENSE)
                R.norm(A->blk[b], (int)T.size[tb], (int)T.size[sb], (int)T.size[tb], nullptr, d + b);
        }
        R.flush_norm();
        double* hp = (double*)R.pinned_host(sizeof(double) * nb);
        H2_CUDA(cudaMemcpyAsync(hp, d, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        H2_CUDA(cudaStreamSynchronize(st));
        std::copy(hp, hp + nb, norm);
        R.release_all();
        return H2_OK;
    } catch (const Error& e) {
        h2_set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        h2_set_last_error(e.what());
        return H2_ERR_CUDA;
    }
}

extern "C" int h2_recompress(h2_matrix* A, const h2_opts* opts) {
    using namespace h2;
    if (!A) return H2_ERR_ARG;
    if (opts && (!(opts->eps >= 0.0) || !std::isfinite(opts->eps) ||
                 !valid_precision(opts->precision)))
        return H2_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != A->device) return H2_ERR_ARG;
    try {
        recompress(A, opts);
        return H2_OK;
    } catch (const Error& e) {
        h2_set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        h2_set_last_error(e.what());
        return H2_ERR_CUDA;
    }
}

extern "C" int h2_mul_add(h2_matrix* Z, const h2_matrix* X, const h2_matrix* Y, const h2_opts* opts) {
    using namespace h2;
    if (!Z || !X || !Y) return H2_ERR_ARG;
    if (opts && (!(opts->eps >= 0.0) || !std::isfinite(opts->eps) ||
                 !valid_precision(opts->precision)))
        return H2_ERR_ARG;
    if (X->st->fingerprint != Y->st->fingerprint || X->st->fingerprint != Z->st->fingerprint) return H2_ERR_SHAPE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != Z->device) return H2_ERR_ARG;
    return run_guarded_mul(Z, X, Y, opts);
}

