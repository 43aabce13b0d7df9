// h2_to_dense_noalloc: the dense expansion of h2_to_dense without any device
// allocation.  All scratch (job descriptors, expanded cluster bases, the
// matrix in tree order) comes from one file-scope device array.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "h2_internal.h"

namespace h2 {

// Fixed scratch shared by every call on a device: 4 Mi doubles (32 MiB),
// allocated when the library is loaded and held until the process exits.
constexpr size_t kNoAllocScratchDoubles = (size_t)4 << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is not a device address).  The lookup
// is serialised, so concurrent first calls from several threads are safe.  A
// device reset (cudaDeviceReset) invalidates the cached address: a process
// that resets a device must not call h2_to_dense_noalloc on it afterwards.
static double* noalloc_scratch_ptr(int dev) {
    static double* ptrs[64] = {};
    static std::mutex mu;
    if (dev < 0 || dev >= 64) throw Error(H2_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) throw Error(H2_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        ptrs[dev] = (double*)p;
    }
    return ptrs[dev];
}

// Bump allocation inside the fixed scratch.  A dry arena (base null) only
// counts: the expansion first runs dry, issuing no device work, so that a
// matrix whose buffers and descriptor arrays do not fit is rejected before
// anything is queued.
class FixedArena {
public:
    FixedArena(double* base, size_t cap) : base_(base), cap_(cap) {}
    bool dry() const { return base_ == nullptr; }
    size_t used() const { return used_; }
    double* take(size_t n) {
        size_t aligned = (std::max<size_t>(n, 1) + 31) & ~(size_t)31;  // 256-byte steps
        if (!dry() && used_ + aligned > cap_)
            throw Error(H2_ERR_UNSUPPORTED, "matrix too large for the fixed scratch of h2_to_dense_noalloc");
        double* p = dry() ? nullptr : base_ + used_;
        used_ += aligned;
        return p;
    }
    template <class T>
    T* put(const std::vector<T>& v, cudaStream_t st) {
        T* d = (T*)take((v.size() * sizeof(T) + 7) / 8);
        if (!dry() && !v.empty())
            H2_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
        return d;
    }

private:
    double* base_;
    size_t cap_, used_ = 0;
};

// Batched products C = sum op(A) op(B) in FP64 through the library's GEMM kernel.
struct GemmList {
    std::vector<GTerm> terms;
    std::vector<GJob> jobs;
    void job(double* C, int m, int n, int ldc) { jobs.push_back(GJob{C, m, n, ldc, (int)terms.size(), 0, 0.0}); }
    void term(const double* A, int ta, int lda, const double* B, int tb, int ldb, int k) {
        if (k <= 0) return;
        terms.push_back(GTerm{A, B, nullptr, 1.0, k, lda, ldb, ta, tb});
        jobs.back().nt++;
    }
    void run(FixedArena& ar, cudaStream_t st) {
        if (jobs.empty()) return;
        std::vector<GTile> tiles;
        for (int j = 0; j < (int)jobs.size(); ++j)
            for (int i0 = 0; i0 < jobs[j].m; i0 += 32)
                for (int j0 = 0; j0 < jobs[j].n; j0 += 32) tiles.push_back(GTile{j, i0, j0});
        GTerm* dt = ar.put(terms, st);
        GJob* dj = ar.put(jobs, st);
        GTile* dti = ar.put(tiles, st);
        if (!ar.dry()) launch_gemm(dt, dj, dti, (int)tiles.size(), H2_FP64, st);
        terms.clear();
        jobs.clear();
    }
};

// The expansion into `ar`; with a dry arena it only measures the scratch it needs.
static void to_dense_noalloc(const h2_matrix* A, double* out, int64_t ld, cudaStream_t st, FixedArena& ar) {
    const Tree& T = A->st->tree;
    const BlockTree& B = A->st->blocks;
    const int64_t n = T.n;
    // expanded bases: rows of the cluster x rank, level by level from the leaves
    auto expand = [&](const Basis& b) {
        std::vector<double*> ex(T.nc, nullptr);
        for (int c = 0; c < T.nc; ++c) ex[c] = ar.take((size_t)T.size[c] * std::max(1, b.rank[c]));
        std::vector<CopyJob> cp;
        for (int c = Tree::first(T.L); c < T.nc; ++c)
            if (b.rank[c] > 0)
                cp.push_back(CopyJob{b.leaf[c], ex[c], nullptr, 1.0, 0.0, (int)T.size[c], b.rank[c], (int)T.size[c],
                                     (int)T.size[c], 0});
        if (!cp.empty()) {
            CopyJob* d = ar.put(cp, st);
            if (!ar.dry()) launch_copy(d, (int)cp.size(), st);
        }
        GemmList g;
        for (int l = T.L - 1; l >= 0; --l) {
            for (int c = Tree::first(l); c < Tree::first(l) + Tree::count(l); ++c)
                for (int i = 0; i < 2; ++i) {
                    int ch = Tree::child(c, i);
                    g.job(ex[c] + (T.off[ch] - T.off[c]), (int)T.size[ch], b.rank[c], (int)T.size[c]);
                    g.term(ex[ch], 0, (int)T.size[ch], b.tr[ch], 0, std::max(1, b.rank[ch]), b.rank[ch]);
                }
            g.run(ar, st);
        }
        return ex;
    };
    auto ev = expand(*A->V);
    auto ew = (A->W == A->V) ? ev : expand(*A->W);
    // the matrix in tree order; cleared because the scratch keeps the last call's contents
    double* dense = ar.take((size_t)n * n);
    if (!ar.dry()) H2_CUDA(cudaMemsetAsync(dense, 0, sizeof(double) * n * n, st));
    GemmList g;
    std::vector<CopyJob> cp;
    std::vector<double*> tmp(B.kind.size(), nullptr);
    for (int b = 0; b < (int)B.kind.size(); ++b) {
        int t = B.t[b], s = B.s[b];
        if (B.kind[b] == ADM) {
            tmp[b] = ar.take((size_t)T.size[t] * std::max(1, A->W->rank[s]));
            g.job(tmp[b], (int)T.size[t], A->W->rank[s], (int)T.size[t]);
            g.term(ev[t], 0, (int)T.size[t], A->blk[b], 0, std::max(1, A->V->rank[t]), A->V->rank[t]);
        } else if (B.kind[b] == DENSE) {
            cp.push_back(CopyJob{A->blk[b], dense + T.off[t] + T.off[s] * n, nullptr, 1.0, 0.0, (int)T.size[t],
                                 (int)T.size[s], (int)T.size[t], (int)n, 0});
        }
    }
    g.run(ar, st);
    if (!cp.empty()) {
        CopyJob* d = ar.put(cp, st);
        if (!ar.dry()) launch_copy(d, (int)cp.size(), st);
    }
    for (int b = 0; b < (int)B.kind.size(); ++b) {
        int t = B.t[b], s = B.s[b];
        if (B.kind[b] != ADM) continue;
        g.job(dense + T.off[t] + T.off[s] * n, (int)T.size[t], (int)T.size[s], (int)n);
        g.term(tmp[b], 0, (int)T.size[t], ew[s], 1, (int)T.size[s], A->W->rank[s]);
    }
    g.run(ar, st);
    int64_t* d_perm = ar.put(T.perm, st);
    if (ar.dry()) return;
    launch_scatter_dense(dense, n, d_perm, out, ld, st);
    H2_CUDA(cudaGetLastError());
    H2_CUDA(cudaStreamSynchronize(st));
}

static void to_dense_noalloc(const h2_matrix* A, double* out, int64_t ld, cudaStream_t st) {
    int dev = 0;
    H2_CUDA(cudaGetDevice(&dev));
    FixedArena probe(nullptr, 0);  // every buffer and descriptor array, measured on the host
    to_dense_noalloc(A, out, ld, st, probe);
    if (probe.used() > kNoAllocScratchDoubles)
        throw Error(H2_ERR_UNSUPPORTED, "matrix too large for the fixed scratch of h2_to_dense_noalloc");
    FixedArena ar(noalloc_scratch_ptr(dev), kNoAllocScratchDoubles);
    to_dense_noalloc(A, out, ld, st, ar);
}

}  // namespace h2

void h2_set_last_error(const char* m);

extern "C" int h2_to_dense_noalloc(const h2_matrix* A, double* out, int64_t ld, void* stream) {
    if (!A || !out || ld < A->st->tree.n) return H2_ERR_ARG;
    try {
        h2::to_dense_noalloc(A, out, ld, (cudaStream_t)stream);
        return H2_OK;
    } catch (const h2::Error& e) {
        h2_set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        h2_set_last_error(e.what());
        return H2_ERR_CUDA;
    }
}
