// Internal declarations of the H^2 product library: host structures (cluster
// tree, block trees, product block tree), device storage of a handle, and the
// descriptors of the batched device operations.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <array>
#include <condition_variable>
#include <vector>

#include "../../include/h2mul.h"

namespace h2 {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& what) : std::runtime_error(what), code(c) {}
};

#define H2_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw ::h2::Error(e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

// ---------------------------------------------------------------- trees
// Complete binary cluster tree, numbered level by level: cluster c has
// children 2c+1, 2c+2; level l holds clusters 2^l-1 .. 2^(l+1)-2.
struct Tree {
    int64_t n = 0;
    int L = 0;
    int nc = 0;
    int leaf_size = 0;
    std::vector<int64_t> perm;       // tree position -> original index
    std::vector<int64_t> off, size;  // per cluster
    std::vector<double> lo, hi;      // per cluster, 3 each (padded boxes)
    static int first(int l) { return (1 << l) - 1; }
    static int count(int l) { return 1 << l; }
    static int parent(int c) { return (c - 1) / 2; }
    static int child(int c, int i) { return 2 * c + 1 + i; }
    static int level(int c) {
        int l = 0;
        while (((1 << (l + 1)) - 1) <= c) ++l;
        return l;
    }
    bool is_leaf(int c) const { return c >= first(L); }
};

enum Kind : int8_t { ADM = 0, DENSE = 1, SPLIT = 2 };

// A block tree over (rows x cols) of the same cluster tree (Def. "Block tree").
struct BlockTree {
    int nc = 0;
    std::vector<int> t, s;
    std::vector<int8_t> kind;
    std::unordered_map<int64_t, int> id;     // t * nc + s -> block index
    std::vector<std::vector<int>> by_row;    // t -> blocks of row t, by increasing s
    std::vector<std::vector<int>> by_col;    // s -> blocks of column s, by increasing t
    std::vector<std::array<int, 4>> kids;    // SPLIT block: block (child(t,i), child(s,j)) at 2 i + j
    int find(int a, int b) const {
        auto it = id.find((int64_t)a * nc + b);
        return it == id.end() ? -1 : it->second;
    }
    int add(int a, int b, int8_t k) {
        int i = (int)t.size();
        t.push_back(a);
        s.push_back(b);
        kind.push_back(k);
        id[(int64_t)a * nc + b] = i;
        return i;
    }
    void finish();  // fills by_row / by_col / kids
    int64_t count(int8_t k) const {
        int64_t c = 0;
        for (auto x : kind) c += (x == k);
        return c;
    }
};

// Product block tree T^XY (Sec. 6) with its triples: for node (t,r), the s with
// (t,s) in T_IJ, (s,r) in T_JK, not both split.
struct ProductTree {
    BlockTree nodes;                       // kind ADM / DENSE / SPLIT
    std::vector<std::vector<int>> triples; // per node: list of s
    std::vector<std::vector<std::pair<int, int>>> tri_blocks;  // per node and triple: blocks (t,s) of X, (s,r) of Y
    std::vector<std::vector<std::pair<int8_t, int8_t>>> tri_kinds;  // per node and triple: kinds of the two blocks
};
ProductTree build_product_tree(const BlockTree& X, const BlockTree& Y);

// Shared structure of matrices built from one point set, with the cached
// product block trees of products with other structures.
struct Structure {
    Tree tree;
    BlockTree blocks;
    double eta = 0;
    std::vector<double> points;  // n x 3, original order
    uint64_t fingerprint = 0;
    std::mutex plan_mutex;
    std::unordered_map<uint64_t, std::shared_ptr<ProductTree>> product_trees;
};

std::shared_ptr<Structure> build_structure(const double* pts, int64_t n, int leaf, double eta);

// ---------------------------------------------------------------- device memory
// Source of device memory: the caller's callbacks (h2_opts alloc/free/alloc_ctx)
// or, when alloc is null, the library itself.
struct DevAlloc {
    h2_alloc_fn alloc = nullptr;
    h2_free_fn free = nullptr;
    void* ctx = nullptr;
    bool external() const { return alloc != nullptr; }
};
DevAlloc alloc_of(const h2_opts* o);  // throws H2_ERR_ARG for alloc without free
// The device-memory source and stream of the API call running on this thread;
// every device buffer a call makes comes from it.  Set for the duration of a
// call (and in its helper threads) by AllocScope.
struct AllocScope {
    AllocScope(const DevAlloc& a, cudaStream_t st);
    ~AllocScope();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;

private:
    DevAlloc prev_a_;
    cudaStream_t prev_s_;
};
const DevAlloc& current_alloc();
cudaStream_t current_alloc_stream();
// one buffer of `bytes` from the current source, for work on `st`
void* dev_get(const DevAlloc& a, size_t bytes, cudaStream_t st, bool pooled);
void dev_put(const DevAlloc& a, void* p, size_t bytes, cudaStream_t st, bool pooled);

// ---------------------------------------------------------------- device storage
// A device buffer of a handle; it remembers where its memory came from.
struct DevBuf {
    double* p = nullptr;
    size_t len = 0;  // doubles
    DevAlloc src;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { reset(); }
    void alloc(size_t n);
    void reset();
};

// A cluster basis: leaf matrices (size x rank, column-major) and transfer
// matrices (rank x rank(parent)), one device pointer per cluster into chunks
// owned by the basis (ranks are only known level by level).
struct Basis {
    std::vector<int> rank;
    std::vector<double*> leaf;  // nullptr for non-leaves
    std::vector<double*> tr;    // nullptr for the root
    std::vector<std::shared_ptr<DevBuf>> chunks;
    int max_rank() const {
        int m = 0;
        for (int r : rank) m = r > m ? r : m;
        return m;
    }
    double bytes() const {
        double b = 0;
        for (auto& c : chunks) b += 8.0 * c->len;
        return b;
    }
};

}  // namespace h2

struct h2_matrix {
    std::shared_ptr<h2::Structure> st;
    std::shared_ptr<h2::Basis> V, W;      // W may alias V
    std::vector<double*> blk;             // per block: S (ADM, rank x rank) or N (DENSE, size x size); null for SPLIT
    std::vector<std::shared_ptr<h2::DevBuf>> chunks;
    int kernel = -1;
    int order = 0;                        // Chebyshev order of the bases, 0 for product results
    int device = 0;
    uint64_t vtag = 0;                    // Chebyshev row basis: 0 on the bounding boxes, else the
                                          // widened interpolation boxes of the double-layer kernel
    uint64_t wtag = 0;                    // Chebyshev column basis: 0 Lagrange, else a hash of the
                                          // normals of a normal-derivative basis
};

namespace h2 {

// Host clock in ms since the first call (trace output only).
double host_clock_ms();

// With H2_TRACE set, the host time of a named scope is summed per thread;
// host_spans_dump() prints the sums ("h2span <thread> <name> <ms> <count>")
// and clears them.  Without it a span costs one test.
struct HostSpan {
    explicit HostSpan(const char* name);
    ~HostSpan();
    HostSpan(const HostSpan&) = delete;
    HostSpan& operator=(const HostSpan&) = delete;

private:
    const char* name_;
    double t0_ = 0.0;
};
void host_spans_dump();
// Successive laps of a scope: mark(name) adds the host time since the previous
// mark (or construction) to span `name` (with H2_TRACE set).
struct HostLap {
    HostLap();
    void mark(const char* name);

private:
    double t_ = 0.0;
};
#define H2_SPAN_CAT2(a, b) a##b
#define H2_SPAN_CAT(a, b) H2_SPAN_CAT2(a, b)
#define H2_SPAN(name) ::h2::HostSpan H2_SPAN_CAT(h2_span_, __LINE__)(name)

// Non-blocking streams kept for the life of the process and handed out per
// call on the current device.  PyTorch's caching allocator keeps freed blocks
// per stream, so a stream created per call would never reuse the blocks that
// earlier calls freed on theirs.  stream_get throws H2_ERR_CUDA when no stream
// can be created; a stream is returned with stream_put once its work is done.
cudaStream_t stream_get();
void stream_put(cudaStream_t s);

// ---------------------------------------------------------------- batched ops
// One term op(A) op(B) of a product sum; op transposes when the flag is set.
// The effective factor is alpha * (*scale) when scale is not null.
struct GTerm {
    const double* A;
    const double* B;
    const double* scale;
    double alpha;
    int k, lda, ldb;
    int ta, tb;
};
// C (m x n, ldc) = beta C + sum of terms [t0, t0 + nt).
struct GJob {
    double* C;
    int m, n, ldc;
    int t0, nt;
    double beta;
    int sym;  // C is symmetric (m == n): only tiles with i0 <= j0 are launched, and
              // the off-diagonal ones also write their transpose
};
struct GTile {
    int job, i0, j0;
};

// Householder QR of A (m x n, in place, lda).  R (min(m,n) x n, ldr) receives
// the triangular factor (zeros below the diagonal); Q (m x q, ldq) the first q
// columns of the orthogonal factor when Q is not null.
struct QRJob {
    double* A;
    double* R;
    double* Q;
    double* tau;  // workspace, min(m,n) entries
    float* A32;   // when set: FP32 workspace (m x n, ld m); A is only read and the
                  // factorisation runs in FP32 (R written in FP64, Q not formed)
    int m, n, lda, ldr, ldq, q;
    int* piv;     // when set (n <= kQRPivMax): column pivoting, A P = Q R with
                  // column j of A P = column piv[j] of A
    double* V;    // when set (FP64, no pivoting, min(m,n) <= kQRPivMax): instead of Q,
    double* T;    // the compact WY form H_0 ... H_{p-1} = I - V T V^T: V (m x p, ld m)
                  // the Householder vectors with unit diagonal and zeros above it,
                  // T (p x p, ld p) upper triangular
};

// widest matrix the column-pivoted QR takes (its norms live in shared memory)
constexpr int kQRPivMax = 2048;

// One-sided Jacobi SVD of B (m x n, in place).  U (m x n, ldu) receives the
// left singular vectors sorted by decreasing singular value, sigma the values,
// *count the number of values above eps, *flag nonzero if the sweep limit was
// reached without convergence.
struct SVDJob {
    double* B;
    double* U;
    double* sigma;
    int* count;
    int* flag;
    double* flops;  // optional accumulator: executed sweep flops (12 m per pair)
    int m, n, ldb, ldu;
    double eps;
    const int* rowperm;  // when set: row i of the singular vectors goes to row rowperm[i] of U
    const int* ncols;    // when set: only the first min(n, *ncols) columns of B are nonzero
};

// FP32 preconditioning of a one-sided Jacobi SVD: sweeps on an FP32 copy W of
// B (m x n) accumulate the right rotations in V; V64 (n x n) receives them.
struct PreJob {
    const double* B;
    float* W;
    float* V;       // accumulated rotations (n x n), or null: not accumulated
    double* V64;    // when set: V in FP64
    double* W64;    // when set: the rotated W in FP64 (m x n, ld m)
    double* flops;  // optional accumulator: executed sweep flops
    int m, n, ldb;
    const int* ncols;  // when set: only the first min(n, *ncols) columns of B are nonzero
};

// Pivoted Cholesky of a symmetric positive semidefinite G (k x k, FP64): Z
// (k x k, ld k) receives a factor with Z^* Z = G up to the pivots below
// rel_tol * max(diag G), which are dropped (their rows of Z stay zero).  With
// abs_tol > 0 it also stops once the trace of the remaining Schur complement
// is at most abs_tol: then G - Z^* Z is positive semidefinite with trace <=
// abs_tol.  *rank (when set) receives the number of pivots taken.
struct CholJob {
    const double* G;
    double* W;  // workspace k x k
    double* Z;  // zrows x k, ld zrows; at most zrows pivots are taken
    int k, ldg, zrows;
    double rel_tol;
    double abs_tol;
    int* rank;
};

// Spectral norm of A (m x n) by power iteration; writes 1/||A|| (0 if the norm
// is below tiny) to *inv and ||A|| to *nrm.
struct NormJob {
    const double* A;
    double* inv;
    double* nrm;
    int m, n, lda;
};

// dst (rows x cols) = beta * dst + alpha * (*scale) * op(src), op = transpose if trans.
struct CopyJob {
    const double* src;
    double* dst;
    const double* scale;
    double alpha, beta;
    int rows, cols, lds, ldd, trans;
};

// C = beta C + sum over `slices` partial products W_s (m x n each, ld m,
// contiguous) of a split-K job.
struct SliceSum {
    double* C;
    const double* W;
    int m, n, ldc, slices;
    double beta;
};

// Kernel launchers (h2_kernels.cu); job arrays are device pointers.
void launch_gemm(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int precision,
                 cudaStream_t st);
void launch_slice_sum(const SliceSum* jobs, int njobs, int max_n, cudaStream_t st);
int device_sm_count();
// tcgen05 variant (mode H2_TF32X3, H2_TF32 or H2_BF16X3): tiles of 128 x 64;
// *err |= 4 if a wait timed out
void launch_gemm_tc(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int mode, int* err,
                    cudaStream_t st);
// output tile edge of the batched GEMM in FP32 (H2_MIXED) and double-float; FP64 uses 32
constexpr int kF32Tile = 64;
// launch_gemm precision tag (not an API value): FP64-accurate products in
// double-float FP32 arithmetic, used for the FP64 products of H2_MIXED and H2_TC
constexpr int kGemmDF = 100;
constexpr int kTcTileM = 128, kTcTileN = 64;
// precision modes that run the factorisation-side steps in FP32 as well
inline bool low_precision(int precision) { return precision != H2_FP64; }
inline bool valid_precision(int p) { return p >= H2_FP64 && p <= H2_AUTO; }
// the FP32-class products run on the tensor cores
inline bool tc_precision(int p) { return p == H2_TF32X3 || p == H2_TF32 || p == H2_BF16X3; }
// H2_AUTO by tolerance: one TF32 product (operand rounding 2^-12, products off
// by about 5e-4) only from eps = 1e-3 up, BF16 pieces (about 2^-17, single
// blocks off by up to 3e-5) down to 1e-4, three-term TF32 products (about FP32
// accuracy) below that, and FP64
// where a Gram matrix in FP32-class arithmetic could no longer resolve the
// singular values the tolerance keeps
inline int resolve_precision(int p, double eps) {
    if (p != H2_AUTO) return p;
    if (eps >= 1e-3) return H2_TF32;
    if (eps >= 1e-4) return H2_BF16X3;
    if (eps >= 1e-7) return H2_TF32X3;
    return H2_FP64;
}
void launch_qr(const QRJob* jobs, int njobs, cudaStream_t st);
void launch_qr32(const QRJob* jobs, int njobs, cudaStream_t st);
// clusters: a level with fewer matrices than SMs may spread each matrix over a
// thread-block cluster (worth it when no other stream's kernels compete for the SMs)
void launch_svd(const SVDJob* jobs, int njobs, int max_n, cudaStream_t st, bool clusters = true);
// max_mn: largest m n of the jobs; max_mnv: largest (m + n) n (W and V together)
void launch_jacobi_pre(const PreJob* jobs, int njobs, size_t max_mn, size_t max_mnv, cudaStream_t st,
                       bool clusters = true);
void launch_pchol(const CholJob* jobs, int njobs, int max_k, cudaStream_t st);
void launch_norm(const NormJob* jobs, int njobs, int precision, cudaStream_t st);
void launch_copy(const CopyJob* jobs, int njobs, cudaStream_t st);
// Stream-ordered pull of up to 4 buffers from mapped pinned host memory into
// device memory (16-byte words; both sides 16-byte aligned), as one kernel.
struct PullSeg {
    const void* src;  // device-visible address of the pinned source
    void* dst;
    size_t bytes;     // rounded up to 16 by the kernel: both buffers must hold it
};
struct PullBatch {
    PullSeg seg[4];
    int n;
};
void launch_pull(const PullBatch& b, cudaStream_t st);
// nrm (n x 3, original order) non-null: the normal-derivative basis
// grad l_nu(x_i) . n_i instead of l_nu(x_i)
void launch_interp_leaf(const double* pts, const double* nrm, const int64_t* perm, const int64_t* off,
                        const int64_t* size, const double* lo, const double* hi, double* const* leafp, int first_leaf,
                        int nleaves, int m, int64_t max_size, cudaStream_t st);
void launch_interp_transfer(const double* lo, const double* hi, double* const* trp, int nc, int m, cudaStream_t st);
void launch_interp_coupling(const double* lo, const double* hi, const int* bt, const int* bs, double* const* bp,
                            int nblocks, int m, int kernel, cudaStream_t st);
void launch_interp_dense(const double* pts, const double* nrm, const int64_t* perm, const int64_t* off,
                         const int64_t* size, const int* bt, const int* bs, double* const* bp, int nblocks, int kernel,
                         cudaStream_t st);
void launch_scatter_dense(const double* src, int64_t n, const int64_t* perm, double* out, int64_t ld,
                          cudaStream_t st);
void launch_set_identity(double* A, int m, int n, int lda, cudaStream_t st);
// rows of an n x nv matrix: gather dst[i] = src[perm[i]] (scatter = 0) or
// scatter dst[perm[i]] = src[i] (scatter = 1)
void launch_permute_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* perm, int64_t n,
                         int64_t nv, int scatter, cudaStream_t st);
void launch_check_finite(const double* A, size_t len, int* flag, cudaStream_t st);
// Sum of squares of the entries of A (rows x cols, lda), added to out[slot].
struct SumSqJob {
    const double* A;
    int rows, cols, lda, slot;
};
// out[b] = sum of the jobs' sums of squares over jobs seg[b] .. seg[b+1]-1, added
// in job order (the jobs sorted by slot; seg has nslots + 1 entries, on the
// device), so that the result does not depend on the order in which CTAs finish;
// part: njobs doubles of scratch
void launch_sumsq(const SumSqJob* jobs, int njobs, double* part, const int* seg, int nslots, double* out,
                  cudaStream_t st);
// sorts the jobs by slot (stable) and returns the nslots + 1 segment offsets
std::vector<int> sumsq_segments(std::vector<SumSqJob>& jobs, int nslots);
// w[i] = 1 / sqrt(v[i]) (0 where v[i] == 0), i < n
void launch_inv_sqrt(const double* v, double* w, double* w2, int n, cudaStream_t st);

// Stream-ordered bump allocator over chunks of the library's memory pool.
// mark()/release() return everything allocated after a mark (stream order
// makes the reuse safe: later work on the stream runs after earlier work).
class Arena {
public:
    explicit Arena(cudaStream_t st) : st_(st) {}
    ~Arena() { release_all(); }
    Arena(const Arena&) = delete;
    Arena& operator=(const Arena&) = delete;
    double* alloc(size_t n);
    struct Mark {
        size_t nchunks;
        char* cur;
        size_t left;
    };
    Mark mark() const { return Mark{chunks_.size(), cur_, left_}; }
    void release(const Mark& m);
    void release_all();

private:
    struct Chunk {
        void* p;
        size_t bytes;
        DevAlloc src;
    };
    cudaStream_t st_;
    std::vector<Chunk> chunks_;
    std::vector<Chunk> spare_;  // released chunks, reused by later allocations of the call
    char* cur_ = nullptr;
    size_t left_ = 0;
};

// Online tuner of GEMM launch schedules (h2_opts.autotune), process-wide.  A
// batch is keyed by its kernel family and the logarithms of its tile count and
// of its K chunks per tile.  The candidates of a key run in turn until each
// has been timed (the times arrive when a call collects its launch events);
// from then on the cheapest, in device milliseconds per GFLOP, runs.
// Candidates: for the FP32-class products the mode's kernel or the other one
// (CUDA-core FP32 against the tensor-core mode, at least as accurate), each
// with split-K by the default rule or off; for the others split-K by the
// default rule, off, or over 2 or 4 slices.
class Tuner {
public:
    static constexpr int kCand = 4;
    static Tuner& get();
    int pick(uint64_t key, int ncand);
    void report(uint64_t key, int cand, double ms_per_gflop);
    // choices made so far (for tests and traces): key -> best candidate or -1
    std::vector<std::pair<uint64_t, int>> table();

private:
    struct Entry {
        double cost[kCand] = {};
        int timed[kCand] = {};
        int issued[kCand] = {};
        int best = -1;
        int ncand = 0;
    };
    std::mutex mu_;
    std::unordered_map<uint64_t, Entry> map_;
};

class Combiner;
// The combiner of the batched call running on this thread (null outside
// h2_mul_add_batched with H2_BATCH_GROUPING=1); Runners built while it is set
// hand it their GEMM batches.
Combiner* current_combiner();
struct CombinerScope {
    explicit CombinerScope(Combiner* c);
    ~CombinerScope();
    CombinerScope(const CombinerScope&) = delete;
    CombinerScope& operator=(const CombinerScope&) = delete;

private:
    Combiner* prev_;
};

// Host-side driver of batched ops: collects jobs, uploads, launches.
class Runner {
public:
    explicit Runner(cudaStream_t st, int precision)
        : st_(st), prec_(precision), scratch_(st), persist_(st), comb_(current_combiner()) {}
    void set_autotune(bool on) { tune_ = on; }
    Combiner* combiner() const { return comb_; }
    ~Runner();
    cudaStream_t stream() const { return st_; }
    int precision() const { return prec_; }
    int64_t launches = 0;

    // GEMM: start a job, add terms, the job is closed by the next job/flush.
    void job(double* C, int m, int n, int ldc, double beta, bool sym = false);
    void term(const double* A, int ta, int lda, const double* B, int tb, int ldb, int k, double alpha = 1.0,
              const double* scale = nullptr);
    void flush_gemm(int precision_override = -1);
    // force: 0 the default rule (when the batch would not fill the GPU), 1 never,
    // S >= 2 every job with enough K into S slices
    void split_k(int pr, int tile, std::vector<SliceSum>& sums, int64_t ntiles = -1, int force = 0);
    void qr(double* A, int m, int n, int lda, double* R, int ldr, double* Q, int ldq, int q, bool fp32 = false,
            int* piv = nullptr);
    // FP64 QR of A (m x n, in place) returning the compact WY form of its Q:
    // Q = I - V T V^T with V (m x p) and T (p x p), p = min(m, n)
    void qr_wy(double* A, int m, int n, int lda, double* V, double* T);
    void flush_qr();
    // ncols (device, optional): only the first min(n, *ncols) columns of B are
    // nonzero; the sweeps and the outputs cover those columns only
    void svd(double* B, int m, int n, int ldb, double* U, int ldu, double* sigma, int* count, double eps,
             const int* rowperm = nullptr, const int* ncols = nullptr);
    void flush_svd();
    void jacobi_pre(const double* B, int m, int n, int ldb, double* V64, double* W64 = nullptr,
                    const int* ncols = nullptr);
    void flush_pre();
    void pchol(const double* G, int k, int ldg, double* Z, int zrows, double rel_tol, double abs_tol = 0.0,
               int* rank = nullptr);
    void flush_pchol();
    void norm(const double* A, int m, int n, int lda, double* inv, double* nrm);
    void flush_norm();
    void copy(const double* src, int lds, double* dst, int ldd, int rows, int cols, int trans, double alpha = 1.0,
              const double* scale = nullptr, double beta = 0.0);
    void flush_copy();
    void flush_all();
    int* svd_flag() const { return d_flag_; }
    void ensure_flag();

    // per-family device time: events around every launch (collected after a sync)
    void begin(int fam);
    void end(int fam, double flops, double bytes, int64_t units = 0);
    void collect(double* ms, int64_t* launches, double* flops, double* bytes, cudaEvent_t ref = nullptr);
    cudaEvent_t first_event() const { return marks_.empty() ? nullptr : marks_.front().a; }

    // device scratch from the stream-ordered pool
    double* dalloc(size_t n) { return scratch_.alloc(n); }
    // device memory that lives until the end of the call (release_all)
    double* palloc(size_t n) { return persist_.alloc(n); }
    Arena::Mark mark() const { return scratch_.mark(); }
    void release(const Arena::Mark& m) { scratch_.release(m); }
    template <class T>
    T* upload(const std::vector<T>& v);
    void release_all();  // frees every allocation of this runner (stream ordered)
    // returns the pinned staging chunks of the uploads issued so far to the
    // process-wide pool (each is reused once the pulls queued so far are done)
    void recycle_staging() { release_pinned(); }
    // host memory in this runner's pinned staging, for device-to-host reads on
    // its stream (a read into pageable memory blocks the calling thread inside
    // the copy call, and other host threads' CUDA calls with it); valid until
    // the staging is recycled
    void* pinned_host(size_t bytes);

private:
    cudaStream_t st_;
    int prec_;
    std::vector<GTerm> terms_;
    std::vector<GJob> jobs_;
    std::vector<GTile> tiles_;
    // accumulated while the batch is built: algorithmic flops and bytes, and
    // its tiles at 32 x 32 and 64 x 64
    double pend_flops_ = 0.0, pend_bytes_ = 0.0;
    int64_t pend_tiles32_ = 0, pend_tiles64_ = 0;
    std::vector<QRJob> qrs_;
    std::vector<SVDJob> svds_;
    std::vector<PreJob> pres_;
    std::vector<CholJob> chols_;
    std::vector<QRJob> qrs32_;
    int svd_maxn_ = 0;
    std::vector<NormJob> norms_;
    std::vector<CopyJob> copies_;
    Arena scratch_;
    Arena persist_;
    int* d_flag_ = nullptr;
    struct Mark {
        int fam;
        cudaEvent_t a, b;
        double flops, bytes;
        double* dflops;  // device-side flop count of the launch, read at collect()
        int64_t units;   // CTAs of the launch (tiles for the products)
        uint64_t tkey = 0;  // autotuned batch: its key and candidate
        int tcand = -1;
        double host_ms = 0.0;  // host clock at the launch (trace only)
    };
    bool tune_ = false;
    Combiner* comb_ = nullptr;
    double* dev_counter();
    std::vector<Mark> marks_;
    std::vector<cudaEvent_t> pool_;
    cudaEvent_t cur_ = nullptr;
    double cur_host_ = 0.0;
    cudaEvent_t get_event();
public:
    // Uploads are staged in mapped pinned host memory and pulled into device
    // memory by a kernel on the Runner's stream (k_pull).  A copy-engine copy
    // could queue behind the copies of another stream, and those behind that
    // stream's kernels; a pageable source could make the copy wait for the
    // stream.  Chunks return to a process-wide pool on release, with an event
    // that marks the end of their last pull.
    struct Pinned {
        char* p;
        char* dp;  // the same memory as seen by the device (mapped)
        size_t size;
        cudaEvent_t done;
    };

private:
    std::vector<Pinned> pinned_;
    size_t pinned_used_ = 0;
    const void* stage(const void* src, size_t bytes);  // returns the device-visible copy
    char* carve_pinned(size_t bytes, char** dev);
    template <class A, class B, class C>
    void upload3(const std::vector<A>& a, A*& da, const std::vector<B>& b, B*& db, const std::vector<C>& c, C*& dc);
    void release_pinned();
};

// Grouped launches across the products of h2_mul_add_batched (opt-in:
// H2_BATCH_GROUPING=1 in the environment).  The products run on their own host
// threads and streams; when one of them flushes a GEMM batch it hands the batch
// to the combiner and waits.  Once every thread that is running product code
// has handed over a batch, or 100 microseconds after a batch was handed over,
// the thread whose wait ends first takes all waiting
// batches, concatenates those of the same kernel (same effective precision)
// into one job list, and launches each list once on the combiner's stream,
// after events of the submitting streams; each submitting stream then waits for
// the launch's event.  One launch per kernel serves every product at that step
// of its level sweep (the products' levels and shapes differ; the segmented
// batched kernels take any mix of jobs).
class Combiner {
public:
    Combiner(cudaStream_t st, int precision);
    ~Combiner();
    void enter();  // a thread starts running product code (it may submit)
    void leave();
    // hands over a GEMM batch of precision tag pr (the jobs' term indices refer
    // to `terms`); returns once the launch holding it is queued and `from` waits
    // for it
    void submit(int pr, std::vector<GTerm>& terms, std::vector<GJob>& jobs, cudaStream_t from);
    Runner& runner() { return R_; }
    int* flag() { return R_.svd_flag(); }
    std::mutex& stats_mutex() { return smu_; }

private:
    struct Sub {
        int pr;
        std::vector<GTerm> terms;
        std::vector<GJob> jobs;
        cudaStream_t st;
        cudaEvent_t ready;
        bool done = false;
        std::string error;
    };
    void launch(std::vector<Sub*>& subs);
    cudaEvent_t event();
    std::mutex mu_, smu_;
    std::condition_variable cv_;
    std::vector<Sub*> pending_;
    int active_ = 0;
    bool leading_ = false;
    Runner R_;
    std::vector<cudaEvent_t> events_;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace h2
