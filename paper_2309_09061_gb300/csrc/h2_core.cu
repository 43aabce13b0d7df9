// Runtime of the H^2 library: device buffers, the batched-op runner, and the
// entry points h2_build_interp, h2_to_dense, h2_info, h2_get_structure,
// h2_free, h2_error_string.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <exception>
#include <functional>
#include <atomic>
#include <condition_variable>
#include <map>
#include <mutex>

#include "h2_internal.h"

namespace h2 {

// ---------------------------------------------------------------- memory
static cudaMemPool_t lib_pool(int dev) {
    static cudaMemPool_t pools[64] = {};
    static std::mutex mu;
    if (dev < 0 || dev >= 64) throw Error(H2_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> g(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        H2_CUDA(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t thr = UINT64_MAX;
        H2_CUDA(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &thr));
    }
    return pools[dev];
}

// With H2_TRACE set, host calls that may block print "h2wait <call> <ms> <bytes>"
// when they take longer than 0.2 ms.
struct HostWait {
    const char* what;
    size_t bytes;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    HostWait(const char* w, size_t b) : what(w), bytes(b) {}
    ~HostWait() {
        static const bool trace = std::getenv("H2_TRACE") != nullptr;
        if (!trace) return;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > 0.2) std::fprintf(stderr, "h2wait %s %.3f %zu\n", what, ms, bytes);
    }
};

double host_clock_ms() {
    static const auto t0 = std::chrono::steady_clock::now();
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

namespace {
bool trace_on() {
    static const bool on = std::getenv("H2_TRACE") != nullptr;
    return on;
}
struct SpanSum {
    double ms = 0.0;
    int64_t n = 0;
};
std::mutex g_span_mu;
std::map<std::pair<int, std::string>, SpanSum> g_spans;
std::atomic<int> g_span_threads{0};
thread_local int tl_span_thread = -1;
}  // namespace

HostSpan::HostSpan(const char* name) : name_(trace_on() ? name : nullptr) {
    if (name_) t0_ = host_clock_ms();
}

HostSpan::~HostSpan() {
    if (!name_) return;
    const double ms = host_clock_ms() - t0_;
    if (tl_span_thread < 0) tl_span_thread = g_span_threads.fetch_add(1);
    std::lock_guard<std::mutex> lk(g_span_mu);
    SpanSum& a = g_spans[{tl_span_thread, name_}];
    a.ms += ms;
    a.n += 1;
}

HostLap::HostLap() {
    if (trace_on()) t_ = host_clock_ms();
}

void HostLap::mark(const char* name) {
    if (!trace_on()) return;
    const double now = host_clock_ms();
    if (tl_span_thread < 0) tl_span_thread = g_span_threads.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(g_span_mu);
        SpanSum& a = g_spans[{tl_span_thread, name}];
        a.ms += now - t_;
        a.n += 1;
    }
    t_ = now;
}

void host_spans_dump() {
    if (!trace_on()) return;
    std::lock_guard<std::mutex> lk(g_span_mu);
    for (const auto& kv : g_spans)
        std::fprintf(stderr, "h2span %d %s %.3f %lld\n", kv.first.first, kv.first.second.c_str(), kv.second.ms,
                     (long long)kv.second.n);
    g_spans.clear();
}

namespace {
std::mutex g_stream_mu;
std::vector<std::pair<int, cudaStream_t>> g_streams;  // (device, stream) not in use
}  // namespace

cudaStream_t stream_get() {
    int dev = 0;
    H2_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_stream_mu);
        for (size_t i = 0; i < g_streams.size(); ++i)
            if (g_streams[i].first == dev) {
                cudaStream_t s = g_streams[i].second;
                g_streams.erase(g_streams.begin() + (long)i);
                return s;
            }
    }
    cudaStream_t s = nullptr;
    H2_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    return s;
}

void stream_put(cudaStream_t s) {
    if (!s) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_stream_mu);
    g_streams.emplace_back(dev, s);
}

// ---------------------------------------------------------------- memory sources
namespace {
thread_local DevAlloc tl_alloc;
thread_local cudaStream_t tl_alloc_stream = nullptr;
// device memory the library holds from its own sources (not from callbacks)
std::atomic<int64_t> g_own_bytes{0}, g_own_peak{0};
void own_add(int64_t b) {
    const int64_t now = g_own_bytes.fetch_add(b) + b;
    int64_t pk = g_own_peak.load();
    while (now > pk && !g_own_peak.compare_exchange_weak(pk, now)) {
    }
}
}  // namespace

DevAlloc alloc_of(const h2_opts* o) {
    DevAlloc a;
    if (!o || !o->alloc) return a;
    if (!o->free) throw Error(H2_ERR_ARG, "h2_opts.alloc given without h2_opts.free");
    a.alloc = o->alloc;
    a.free = o->free;
    a.ctx = o->alloc_ctx;
    return a;
}

AllocScope::AllocScope(const DevAlloc& a, cudaStream_t st) : prev_a_(tl_alloc), prev_s_(tl_alloc_stream) {
    tl_alloc = a;
    tl_alloc_stream = st;
}
AllocScope::~AllocScope() {
    tl_alloc = prev_a_;
    tl_alloc_stream = prev_s_;
}
const DevAlloc& current_alloc() { return tl_alloc; }
cudaStream_t current_alloc_stream() { return tl_alloc_stream; }

// pooled: scratch from the library's stream-ordered pool; otherwise cudaMalloc
// (the buffers of handles, returned to the driver when they are freed)
void* dev_get(const DevAlloc& a, size_t bytes, cudaStream_t st, bool pooled) {
    H2_SPAN("dev_get");
    void* p = nullptr;
    if (a.external()) {
        HostWait hw("alloc_callback", bytes);
        p = a.alloc(bytes, (void*)st, a.ctx);
        if (!p) throw Error(H2_ERR_OOM, "the caller's allocator returned NULL");
        if (((uintptr_t)p & 255u) != 0) {
            a.free(p, bytes, (void*)st, a.ctx);
            throw Error(H2_ERR_ARG, "the caller's allocator returned memory aligned to less than 256 bytes");
        }
        return p;
    }
    if (pooled) {
        int dev = 0;
        H2_CUDA(cudaGetDevice(&dev));
        HostWait hw("pool_alloc", bytes);
        H2_CUDA(cudaMallocFromPoolAsync(&p, bytes, lib_pool(dev), st));
    } else {
        HostWait hw("cudaMalloc", bytes);
        H2_CUDA(cudaMalloc(&p, bytes));
    }
    own_add((int64_t)bytes);
    return p;
}

void dev_put(const DevAlloc& a, void* p, size_t bytes, cudaStream_t st, bool pooled) {
    if (!p) return;
    if (a.external()) {
        a.free(p, bytes, (void*)st, a.ctx);
        return;
    }
    if (pooled) {
        cudaFreeAsync(p, st);
    } else {
        HostWait hw("cudaFree", bytes);
        cudaFree(p);
    }
    own_add(-(int64_t)bytes);
}

void DevBuf::alloc(size_t n) {
    H2_SPAN("DevBuf::alloc");
    reset();
    if (n == 0) return;
    src = current_alloc();
    st = current_alloc_stream();
    p = (double*)dev_get(src, n * sizeof(double), st, false);
    len = n;
}

void DevBuf::reset() {
    if (p) dev_put(src, p, len * sizeof(double), st, false);
    p = nullptr;
    len = 0;
}

// ---------------------------------------------------------------- runner
Runner::~Runner() {
    // on an error path work may still be queued (on this or another stream) that
    // reads buffers about to be returned: wait for it before freeing them
    if (std::uncaught_exceptions() > 0) cudaDeviceSynchronize();
    release_all();
    for (auto& m : marks_) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : pool_) cudaEventDestroy(e);
}

cudaEvent_t Runner::get_event() {
    if (!pool_.empty()) {
        cudaEvent_t e = pool_.back();
        pool_.pop_back();
        return e;
    }
    cudaEvent_t e;
    H2_CUDA(cudaEventCreate(&e));
    return e;
}

double* Runner::dev_counter() {
    double* c = palloc(1);
    H2_CUDA(cudaMemsetAsync(c, 0, sizeof(double), st_));
    return c;
}

void Runner::begin(int fam) {
    (void)fam;
    static const bool trace = std::getenv("H2_TRACE") != nullptr;
    if (trace) cur_host_ = host_clock_ms();
    cur_ = get_event();
    H2_CUDA(cudaEventRecord(cur_, st_));
}

void Runner::end(int fam, double flops, double bytes, int64_t units) {
    // a refused launch (an invalid configuration) fails here, not silently: its
    // outputs would keep whatever the scratch held
    H2_CUDA(cudaGetLastError());
    cudaEvent_t b = get_event();
    H2_CUDA(cudaEventRecord(b, st_));
    marks_.push_back(Mark{fam, cur_, b, flops, bytes, nullptr, units});
    marks_.back().host_ms = cur_host_;
    cur_ = nullptr;
}

// With H2_TRACE set in the environment, every launch is also printed to
// stderr as "h2trace <family> <units> <GFLOP> <MB> <ms> <start ms> <stream>
// <host ms>" in launch order (start relative to ref, else to the first launch
// collected here; host ms: host_clock_ms() when the launch was enqueued).
void Runner::collect(double* ms, int64_t* launches, double* flops, double* bytes, cudaEvent_t ref) {
    H2_SPAN("collect");
    static const bool trace = std::getenv("H2_TRACE") != nullptr;
    if (!ref && !marks_.empty()) ref = marks_.front().a;
    for (auto& m : marks_) {
        float t0 = 0.f;
        if (trace) cudaEventElapsedTime(&t0, ref, m.a);
        float f = 0.f;
        cudaEventElapsedTime(&f, m.a, m.b);
        double df = 0.0;
        if (m.dflops) cudaMemcpy(&df, m.dflops, sizeof(double), cudaMemcpyDeviceToHost);
        if (ms) ms[m.fam] += f;
        if (launches) launches[m.fam] += 1;
        if (flops) flops[m.fam] += m.flops + df;
        if (bytes) bytes[m.fam] += m.bytes;
        if (m.tcand >= 0 && m.flops > 0.0) Tuner::get().report(m.tkey, m.tcand, f / (m.flops * 1e-9));
        if (trace)
            std::fprintf(stderr, "h2trace %d %lld %.6f %.3f %.6f %.3f %p %.3f\n", m.fam, (long long)m.units,
                         (m.flops + df) * 1e-9, m.bytes * 1e-6, f, t0, (void*)st_, m.host_ms);
        pool_.push_back(m.a);
        pool_.push_back(m.b);
    }
    marks_.clear();
}

// Bump allocation (256-byte aligned) from chunks of the library's
// stream-ordered pool.
double* Arena::alloc(size_t n) {
    if (n == 0) n = 1;
    size_t bytes = (n * sizeof(double) + 255) & ~(size_t)255;
#ifdef H2_EXACT_ALLOC
    const size_t chunk_min = 0;  // one pool allocation per buffer (bounds-checking builds)
#else
    const size_t chunk_min = (size_t)64 << 20;
#endif
    if (bytes > left_) {
        const size_t sz = std::max(bytes, chunk_min);
        // a chunk released earlier in the call is reused first: work on this stream
        // that used it is ordered before any later work
        int pick = -1;
        for (int i = 0; i < (int)spare_.size(); ++i)
            if (spare_[i].bytes >= sz && (pick < 0 || spare_[i].bytes < spare_[pick].bytes)) pick = i;
        if (pick >= 0) {
            chunks_.push_back(spare_[pick]);
            spare_.erase(spare_.begin() + pick);
        } else {
            const DevAlloc& src = current_alloc();
            void* p = dev_get(src, sz, st_, true);
            chunks_.push_back(Chunk{p, sz, src});
        }
        cur_ = (char*)chunks_.back().p;
        left_ = chunks_.back().bytes;
    }
    double* out = (double*)cur_;
    cur_ += bytes;
    left_ -= bytes;
    return out;
}

void Arena::release(const Mark& m) {
    // keep up to 256 MiB of released chunks for reuse (fewer allocator calls per
    // level); the rest goes back to its source, where other arenas can use it
    size_t kept = 0;
    for (const Chunk& c : spare_) kept += c.bytes;
    while (chunks_.size() > m.nchunks) {
        const Chunk& c = chunks_.back();
        if (kept + c.bytes <= ((size_t)256 << 20)) {
            kept += c.bytes;
            spare_.push_back(c);
        } else {
            dev_put(c.src, c.p, c.bytes, st_, true);
        }
        chunks_.pop_back();
    }
    cur_ = m.cur;
    left_ = m.left;
}

void Arena::release_all() {
    for (const Chunk& c : chunks_) dev_put(c.src, c.p, c.bytes, st_, true);
    for (const Chunk& c : spare_) dev_put(c.src, c.p, c.bytes, st_, true);
    chunks_.clear();
    spare_.clear();
    cur_ = nullptr;
    left_ = 0;
}

namespace {
std::mutex g_pinned_mu;
std::vector<Runner::Pinned> g_pinned_free;
constexpr size_t kPinnedChunk = size_t(32) << 20;
}  // namespace

const void* Runner::stage(const void* src, size_t bytes) {
    char* dh = nullptr;
    char* h = carve_pinned(bytes, &dh);
    std::memcpy(h, src, bytes);
    return dh;
}

void* Runner::pinned_host(size_t bytes) {
    char* dh = nullptr;
    return carve_pinned(bytes, &dh);
}

// `bytes` (rounded up to 256) of this runner's pinned staging: the host
// address, and the device address of the same memory in *dev
char* Runner::carve_pinned(size_t bytes, char** dev) {
    const size_t need = (bytes + 255) & ~size_t(255);
    if (pinned_.empty() || pinned_used_ + need > pinned_.back().size) {
        Pinned c{nullptr, nullptr, 0, nullptr};
        {
            std::lock_guard<std::mutex> lk(g_pinned_mu);
            for (size_t i = 0; i < g_pinned_free.size(); ++i)
                if (g_pinned_free[i].size >= need) {
                    c = g_pinned_free[i];
                    g_pinned_free.erase(g_pinned_free.begin() + i);
                    break;
                }
        }
        if (c.p) {
            HostWait hw("pinned_reuse", c.size);
            H2_CUDA(cudaEventSynchronize(c.done));  // its previous pulls have ended
        } else {
            c.size = std::max(need, kPinnedChunk);
            HostWait hw("cudaHostAlloc", c.size);
            H2_CUDA(cudaHostAlloc((void**)&c.p, c.size, cudaHostAllocMapped | cudaHostAllocPortable));
            H2_CUDA(cudaHostGetDevicePointer((void**)&c.dp, c.p, 0));
            H2_CUDA(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
        }
        pinned_.push_back(c);
        pinned_used_ = 0;
    }
    char* h = pinned_.back().p + pinned_used_;
    *dev = pinned_.back().dp + pinned_used_;
    pinned_used_ += need;
    return h;
}

void Runner::release_pinned() {
    if (pinned_.empty()) return;
    for (Pinned& c : pinned_) cudaEventRecord(c.done, st_);
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    for (Pinned& c : pinned_) g_pinned_free.push_back(c);
    pinned_.clear();
    pinned_used_ = 0;
}

// Uploads: staged in mapped pinned memory (256-byte granules) and pulled into
// the arena (256-byte granules) by k_pull on this stream.
template <class T>
T* Runner::upload(const std::vector<T>& v) {
    H2_SPAN("upload");
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 8);
    double* d = dalloc((bytes + 7) / 8);
    if (!v.empty()) {
        PullBatch b{};
        b.seg[0] = PullSeg{stage(v.data(), v.size() * sizeof(T)), d, v.size() * sizeof(T)};
        b.n = 1;
        launch_pull(b, st_);
        ++launches;
    }
    return (T*)d;
}

template <class A, class B, class C>
void Runner::upload3(const std::vector<A>& a, A*& da, const std::vector<B>& b, B*& db, const std::vector<C>& c,
                     C*& dc) {
    PullBatch pb{};
    auto one = [&](const void* src, size_t n, size_t esz) -> double* {
        const size_t bytes = std::max<size_t>(n * esz, 8);
        double* d = dalloc((bytes + 7) / 8);
        if (n) pb.seg[pb.n++] = PullSeg{stage(src, n * esz), d, n * esz};
        return d;
    };
    da = (A*)one(a.data(), a.size(), sizeof(A));
    db = (B*)one(b.data(), b.size(), sizeof(B));
    dc = (C*)one(c.data(), c.size(), sizeof(C));
    if (pb.n) {
        launch_pull(pb, st_);
        ++launches;
    }
}
template int* Runner::upload<int>(const std::vector<int>&);
template int64_t* Runner::upload<int64_t>(const std::vector<int64_t>&);
template double* Runner::upload<double>(const std::vector<double>&);
template double** Runner::upload<double*>(const std::vector<double*>&);

void Runner::release_all() {
    H2_SPAN("release_all");
    release_pinned();
    scratch_.release_all();
    persist_.release_all();
    d_flag_ = nullptr;
}

void Runner::ensure_flag() {
    if (!d_flag_) {
        d_flag_ = (int*)palloc(1);
        H2_CUDA(cudaMemsetAsync(d_flag_, 0, sizeof(int), st_));
    }
}

void Runner::job(double* C, int m, int n, int ldc, double beta, bool sym) {
    const int sy = (sym && m == n) ? 1 : 0;
    jobs_.push_back(GJob{C, m, n, ldc, (int)terms_.size(), 0, beta, sy});
    pend_bytes_ += 8.0 * m * n * (beta != 0.0 ? 2.0 : 1.0);
    const int64_t a32 = (m + 31) / 32, b32 = (n + 31) / 32, a64 = (m + 63) / 64, b64 = (n + 63) / 64;
    pend_tiles32_ += sy ? a32 * (a32 + 1) / 2 : a32 * b32;
    pend_tiles64_ += sy ? a64 * (a64 + 1) / 2 : a64 * b64;
}

void Runner::term(const double* A, int ta, int lda, const double* B, int tb, int ldb, int k, double alpha,
                  const double* scale) {
    if (k <= 0 || jobs_.empty()) return;
    terms_.push_back(GTerm{A, B, scale, alpha, k, lda, ldb, ta, tb});
    GJob& J = jobs_.back();
    J.nt++;
    pend_flops_ += (J.sym ? (double)J.m * (J.m + 1) : 2.0 * J.m * J.n) * k;
    pend_bytes_ += 8.0 * ((double)J.m * k + (double)k * J.n);
}

// ---------------------------------------------------------------- grouped launches
namespace {
thread_local Combiner* tl_comb = nullptr;
}
Combiner* current_combiner() { return tl_comb; }
CombinerScope::CombinerScope(Combiner* c) : prev_(tl_comb) { tl_comb = c; }
CombinerScope::~CombinerScope() { tl_comb = prev_; }

Combiner::Combiner(cudaStream_t st, int precision) : R_(st, precision) { R_.ensure_flag(); }

Combiner::~Combiner() {
    cudaStreamSynchronize(R_.stream());
    for (cudaEvent_t e : events_) cudaEventDestroy(e);
}

cudaEvent_t Combiner::event() {
    cudaEvent_t e;
    H2_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    events_.push_back(e);
    return e;
}

void Combiner::enter() {
    std::lock_guard<std::mutex> lk(mu_);
    ++active_;
}

void Combiner::leave() {
    std::lock_guard<std::mutex> lk(mu_);
    --active_;
    cv_.notify_all();
}

void Combiner::launch(std::vector<Sub*>& subs) {
    std::vector<int> prs;
    for (Sub* s : subs)
        if (std::find(prs.begin(), prs.end(), s->pr) == prs.end()) prs.push_back(s->pr);
    for (int pr : prs) {
        for (Sub* s : subs)
            if (s->pr == pr) H2_CUDA(cudaStreamWaitEvent(R_.stream(), s->ready, 0));
        const Arena::Mark mk = R_.mark();
        for (Sub* s : subs) {
            if (s->pr != pr) continue;
            for (const GJob& J : s->jobs) {
                R_.job(J.C, J.m, J.n, J.ldc, J.beta, J.sym != 0);
                for (int i = 0; i < J.nt; ++i) {
                    const GTerm& T = s->terms[J.t0 + i];
                    R_.term(T.A, T.ta, T.lda, T.B, T.tb, T.ldb, T.k, T.alpha, T.scale);
                }
            }
        }
        R_.flush_gemm(pr);
        R_.release(mk);         // descriptors and split-K slices: reused in stream order
        R_.recycle_staging();  // and their pinned host staging
        cudaEvent_t done = event();
        H2_CUDA(cudaEventRecord(done, R_.stream()));
        for (Sub* s : subs)
            if (s->pr == pr) H2_CUDA(cudaStreamWaitEvent(s->st, done, 0));
    }
}

void Combiner::submit(int pr, std::vector<GTerm>& terms, std::vector<GJob>& jobs, cudaStream_t from) {
    Sub s;
    s.pr = pr;
    s.terms.swap(terms);
    s.jobs.swap(jobs);
    s.st = from;
    H2_CUDA(cudaEventCreateWithFlags(&s.ready, cudaEventDisableTiming));
    H2_CUDA(cudaEventRecord(s.ready, from));
    const auto t0 = std::chrono::steady_clock::now();
    std::unique_lock<std::mutex> lk(mu_);
    pending_.push_back(&s);
    cv_.notify_all();
    while (!s.done) {
        const bool all_in = (int)pending_.size() >= active_;
        const bool late = std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(100);
        if (!leading_ && !pending_.empty() && (all_in || late)) {
            leading_ = true;
            std::vector<Sub*> take;
            take.swap(pending_);
            lk.unlock();
            std::string err;
            try {
                launch(take);
            } catch (const std::exception& e) {
                err = e.what();
            }
            lk.lock();
            for (Sub* t : take) {
                t->done = true;
                t->error = err;
            }
            leading_ = false;
            cv_.notify_all();
            continue;
        }
        cv_.wait_for(lk, std::chrono::microseconds(25));
    }
    lk.unlock();
    cudaEventDestroy(s.ready);
    if (!s.error.empty()) throw Error(H2_ERR_CUDA, "grouped launch failed: " + s.error);
}

// ---------------------------------------------------------------- autotuner
Tuner& Tuner::get() {
    static Tuner t;
    return t;
}

int Tuner::pick(uint64_t key, int ncand) {
    std::lock_guard<std::mutex> lk(mu_);
    Entry& e = map_[key];
    e.ncand = ncand;
    if (e.best >= 0) return e.best;
    // the candidate issued least so far (round robin until every one is timed twice)
    int c = 0;
    for (int i = 1; i < ncand; ++i)
        if (e.issued[i] < e.issued[c]) c = i;
    e.issued[c]++;
    return c;
}

void Tuner::report(uint64_t key, int cand, double ms_per_gflop) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = map_.find(key);
    if (it == map_.end() || cand < 0 || cand >= kCand) return;
    Entry& e = it->second;
    e.cost[cand] += ms_per_gflop;
    e.timed[cand]++;
    if (e.best >= 0) return;
    for (int i = 0; i < e.ncand; ++i)
        if (e.timed[i] < 1) return;
    int b = 0;
    for (int i = 1; i < e.ncand; ++i)
        if (e.cost[i] / e.timed[i] < e.cost[b] / e.timed[b]) b = i;
    e.best = b;
}

std::vector<std::pair<uint64_t, int>> Tuner::table() {
    std::lock_guard<std::mutex> lk(mu_);
    std::vector<std::pair<uint64_t, int>> out;
    for (auto& kv : map_) out.push_back({kv.first, kv.second.best});
    return out;
}

static int ilog2(double x) {
    int l = 0;
    while (x >= 2.0 && l < 62) {
        x *= 0.5;
        ++l;
    }
    return l;
}

void Runner::flush_gemm(int precision_override) {
    H2_SPAN("flush_gemm");
    if (jobs_.empty()) return;
    int pr = precision_override >= 0 ? precision_override : prec_;
    // FP64 products of the low-precision modes run in double-float arithmetic
    if (pr == H2_FP64 && prec_ != H2_FP64) pr = kGemmDF;
    if (comb_ && !tune_) {  // a product of a batched call: one launch for all products at this step
        pend_flops_ = pend_bytes_ = 0.0;
        pend_tiles32_ = pend_tiles64_ = 0;
        comb_->submit(pr, terms_, jobs_, st_);
        terms_.clear();
        jobs_.clear();
        return;
    }
    // autotuned schedule: the kernel of the FP32-class products and the split-K policy
    uint64_t tkey = 0;
    int tcand = -1, force_split = 0;
    if (tune_) {
        const bool f32class = (pr == H2_MIXED || tc_precision(pr));
        double chunks = 0.0;
        for (const GTerm& t : terms_) chunks += (t.k + 31) / 32;
        const int64_t tiles = std::max<int64_t>(1, pend_tiles64_);
        tkey = ((uint64_t)(pr & 0xff) << 16) | ((uint64_t)ilog2((double)tiles) << 8) |
               (uint64_t)ilog2(chunks / (double)tiles);
        tcand = Tuner::get().pick(tkey, 4);
        if (f32class) {  // (kernel: own, other) x (split-K: default rule, off)
            force_split = (tcand & 1) ? 1 : 0;
            if (tcand >= 2) pr = (pr == H2_MIXED) ? H2_TF32X3 : H2_MIXED;  // the other FP32-class kernel
        } else {  // split-K: default rule, off, 2 or 4 slices
            const int sp[4] = {0, 1, 2, 4};
            force_split = sp[tcand];
        }
    }
    // Without the tuner, a tensor-core batch whose jobs fit 64-row tiles runs on the
    // CUDA-core FP32 kernel: its 64 x 64 tiles cover such jobs as well as the 128 x 64
    // tensor-core tiles (which stage the same operand rows), and it finishes them
    // 1.4-2x sooner (64 x 64 jobs with 4 terms of k = 64: 22.7 against 16.3 TFLOP/s;
    // 30 x 50 jobs: 6.1 against 3.4).  Its FP32 accumulation is at least as accurate as
    // every tensor-core mode.  Wider jobs, which need half as many tensor-core tiles,
    // stay on the tensor cores.
    if (!tune_ && tc_precision(pr) && pend_tiles64_ > 0) {
        int64_t tc_tiles = 0;
        for (const GJob& J : jobs_)
            tc_tiles += (int64_t)((J.m + kTcTileM - 1) / kTcTileM) * ((J.n + kTcTileN - 1) / kTcTileN);
        if (2 * pend_tiles64_ < 3 * tc_tiles) pr = H2_MIXED;
    }
    const bool tc = tc_precision(pr);
    const bool f32 = (pr == H2_MIXED || pr == kGemmDF);
    const int tm = tc ? kTcTileM : f32 ? kF32Tile : 32, tn = tc ? kTcTileN : f32 ? kF32Tile : 32;
    // algorithmic work of the batch: every operand read once, every output written once
    const double fl = pend_flops_, by = pend_bytes_;
    const int64_t nt_est = (tm == 32 && tn == 32) ? pend_tiles32_ : (tm == 64 && tn == 64) ? pend_tiles64_ : -1;
    pend_flops_ = pend_bytes_ = 0.0;
    pend_tiles32_ = pend_tiles64_ = 0;
    static const bool trace = std::getenv("H2_TRACE") != nullptr;
    if (trace) {  // "h2gemm <prec> <jobs> <terms> <mean m> <mean n> <mean K per job> <jobs with m,n <= 64> <max m> <max n> <max K> <stream> <GFLOP>"
        double sm = 0, sn = 0, sk = 0;
        int64_t small = 0, mk = 0;
        int mm = 0, mn = 0;
        for (const GJob& J : jobs_) {
            sm += J.m;
            sn += J.n;
            int64_t kj = 0;
            for (int i = 0; i < J.nt; ++i) kj += terms_[J.t0 + i].k;
            sk += (double)kj;
            mk = std::max(mk, kj);
            small += (J.m <= 64 && J.n <= 64);
            mm = std::max(mm, J.m);
            mn = std::max(mn, J.n);
        }
        const double nj = (double)jobs_.size();
        std::fprintf(stderr, "h2gemm %d %zu %zu %.1f %.1f %.1f %lld %d %d %lld %p %.6f\n", pr, jobs_.size(),
                     terms_.size(), sm / nj, sn / nj, sk / nj, (long long)small, mm, mn, (long long)mk, (void*)st_,
                     fl * 1e-9);
    }
    std::vector<SliceSum> sums;
    int64_t nt_all = nt_est;
    if (nt_all < 0) {  // rectangular tiles (tensor cores): count them
        nt_all = 0;
        for (const GJob& J : jobs_) nt_all += (int64_t)((J.m + tm - 1) / tm) * ((J.n + tn - 1) / tn);
    }
    split_k(pr, tm, sums, nt_all, force_split);
    std::vector<GTile>& tiles = tiles_;
    tiles.clear();
    if (nt_est > 0) tiles.reserve((size_t)nt_est);
    for (int j = 0; j < (int)jobs_.size(); ++j) {
        GJob& J = jobs_[j];
        if (tm != tn) J.sym = 0;  // symmetric jobs need a square tile grid
        for (int i0 = 0; i0 < J.m; i0 += tm)
            for (int j0 = 0; j0 < J.n; j0 += tn)
                if (!J.sym || i0 <= j0) tiles.push_back(GTile{j, i0, j0});
    }
    if (!tiles.empty()) {
        GTerm* dt;
        GJob* dj;
        GTile* dti;
        upload3(terms_, dt, jobs_, dj, tiles, dti);
        const int fam = tc ? 10 : (pr == H2_MIXED) ? 1 : (pr == kGemmDF) ? 11 : 0;
        if (tc) ensure_flag();
        SliceSum* ds = sums.empty() ? nullptr : upload(sums);
        int max_n = 0;
        for (const SliceSum& s : sums) max_n = std::max(max_n, s.n);
        begin(fam);
        if (tc) {
            launch_gemm_tc(dt, dj, dti, (int)tiles.size(), pr, d_flag_, st_);
        } else {
            HostWait hw("launch_gemm", tiles.size());
            launch_gemm(dt, dj, dti, (int)tiles.size(), pr, st_);
        }
        launch_slice_sum(ds, (int)sums.size(), max_n, st_);
        if (!sums.empty()) ++launches;
        end(fam, fl, by, (int64_t)tiles.size());
        marks_.back().tkey = tkey;
        marks_.back().tcand = tcand;
        ++launches;
    }
    terms_.clear();
    jobs_.clear();
}

// Split-K: when a launch would not fill the GPU, jobs with long K are cut
// into segments of their (term, K chunk) sequence; each segment writes its
// partial product to a slice of scratch, and k_slice_sum adds the slices (in
// order, deterministic) into C with the job's beta.  Terms that straddle a
// cut are divided by offsetting their operands along K.
void Runner::split_k(int pr, int tile, std::vector<SliceSum>& sums, int64_t ntiles, int force) {
    if (force == 1) return;
    const int kc = (pr == kGemmDF || pr == H2_FP64) ? 16 : 32;  // K chunk of the kernel
    const int per_sm = (pr == kGemmDF || tc_precision(pr)) ? 2 : (pr == H2_MIXED) ? 3 : 4;  // resident CTAs
    const int64_t target = 2LL * device_sm_count() * per_sm;
    if (ntiles < 0) {  // tiles of the batch, unless counted while it was built
        ntiles = 0;
        for (const GJob& J : jobs_) {
            const int64_t ti = (int64_t)((J.m + tile - 1) / tile), tj = (int64_t)((J.n + tile - 1) / tile);
            ntiles += J.sym ? ti * (ti + 1) / 2 : ti * tj;
        }
    }
    int want = 0;
    if (force >= 2) {
        want = force;
    } else {
        if (ntiles == 0 || ntiles >= target) return;
        want = (int)std::min<int64_t>(16, (target + ntiles - 1) / ntiles);
    }
    if (want < 2) return;
    std::vector<GJob> jobs;
    std::vector<GTerm> terms;
    jobs.reserve(jobs_.size());
    terms.reserve(terms_.size());
    for (const GJob& J : jobs_) {
        int64_t chunks = 0;
        for (int i = 0; i < J.nt; ++i) chunks += (terms_[J.t0 + i].k + kc - 1) / kc;
        const int S = (int)std::min<int64_t>(want, chunks / (force >= 2 ? 4 : 8));
        if (S < 2) {
            GJob K = J;
            K.t0 = (int)terms.size();
            for (int i = 0; i < J.nt; ++i) terms.push_back(terms_[J.t0 + i]);
            jobs.push_back(K);
            continue;
        }
        const int64_t mn = (int64_t)J.m * J.n;
        double* W = dalloc((size_t)(mn * S));
        sums.push_back(SliceSum{J.C, W, J.m, J.n, J.ldc, S, J.beta});
        // walk the chunk sequence, starting a new slice job at each cut
        int s = 0;
        int64_t done = 0, cut = (chunks * 1) / S;
        GJob cur{W, J.m, J.n, J.m, (int)terms.size(), 0, 0.0, J.sym};
        for (int i = 0; i < J.nt; ++i) {
            const GTerm& T = terms_[J.t0 + i];
            int k0 = 0;
            while (k0 < T.k) {
                const int64_t left = (T.k - k0 + kc - 1) / kc;  // chunks left in this term
                int64_t take = left;
                if (s < S - 1 && done + left > cut) take = cut - done;
                if (take > 0) {
                    const int k1 = std::min(T.k, k0 + (int)(take * kc));
                    GTerm P = T;
                    P.k = k1 - k0;
                    P.A = T.ta ? T.A + k0 : T.A + (size_t)k0 * T.lda;
                    P.B = T.tb ? T.B + (size_t)k0 * T.ldb : T.B + k0;
                    terms.push_back(P);
                    ++cur.nt;
                    done += take;
                    k0 = k1;
                }
                if (s < S - 1 && done >= cut) {
                    jobs.push_back(cur);
                    ++s;
                    cur = GJob{W + (size_t)s * mn, J.m, J.n, J.m, (int)terms.size(), 0, 0.0, J.sym};
                    cut = (chunks * (s + 1)) / S;
                }
            }
        }
        jobs.push_back(cur);
        for (++s; s < S; ++s)  // slices that received no chunk (not expected) are zero
            jobs.push_back(GJob{W + (size_t)s * mn, J.m, J.n, J.m, (int)terms.size(), 0, 0.0, J.sym});
    }
    jobs_.swap(jobs);
    terms_.swap(terms);
}

void Runner::qr(double* A, int m, int n, int lda, double* R, int ldr, double* Q, int ldq, int q, bool fp32,
                int* piv) {
    if (m <= 0 || n <= 0) return;
    if (piv && n > kQRPivMax) throw Error(H2_ERR_UNSUPPORTED, "pivoted QR wider than 2048 columns");
    double* tau = dalloc(std::min(m, n));
    if (fp32) {
        float* a32 = (float*)dalloc(((size_t)m * n + 1) / 2);
        qrs32_.push_back(QRJob{A, R, nullptr, tau, a32, m, n, lda, ldr, ldq, 0, piv});
    } else {
        qrs_.push_back(QRJob{A, R, Q, tau, nullptr, m, n, lda, ldr, ldq, q, piv});
    }
}

void Runner::qr_wy(double* A, int m, int n, int lda, double* V, double* T) {
    if (m <= 0 || n <= 0) return;
    if (std::min(m, n) > kQRPivMax) throw Error(H2_ERR_UNSUPPORTED, "WY form of a QR with more than 2048 reflectors");
    double* tau = dalloc(std::min(m, n));
    QRJob j{A, nullptr, nullptr, tau, nullptr, m, n, lda, 1, 1, 0, nullptr};
    j.V = V;
    j.T = T;
    qrs_.push_back(j);
}

void Runner::flush_qr() {
    H2_SPAN("flush_qr");
    if (!qrs32_.empty()) {
        QRJob* d = upload(qrs32_);
        double fl = 0.0, by = 0.0;
        for (auto& j : qrs32_) {
            double m = j.m, n = j.n, p = std::min(j.m, j.n);
            fl += 4.0 * m * n * p - 2.0 * (m + n) * p * p + 4.0 / 3.0 * p * p * p;
            by += 8.0 * m * n + 8.0 * p * n;
        }
        begin(3);
        launch_qr32(d, (int)qrs32_.size(), st_);
        end(3, fl, by);
        ++launches;
        qrs32_.clear();
    }
    if (qrs_.empty()) return;
    QRJob* d = upload(qrs_);
    double fl = 0.0, by = 0.0;
    for (auto& j : qrs_) {
        double m = j.m, n = j.n, p = std::min(j.m, j.n);
        fl += 4.0 * m * n * p - 2.0 * (m + n) * p * p + 4.0 / 3.0 * p * p * p + (j.Q ? 4.0 * m * j.q * p : 0.0) +
              (j.V ? m * p * p - p * p * p / 3.0 : 0.0);
        by += 8.0 * (2.0 * m * n + (j.R ? p * n : 0.0) + (j.Q ? m * j.q : 0.0) + (j.V ? m * p + p * p : 0.0));
    }
    begin(2);
    launch_qr(d, (int)qrs_.size(), st_);
    end(2, fl, by);
    ++launches;
    qrs_.clear();
}

// With H2_TRACE set: "h2jobs <kind> <jobs> <max m> <max n> <mean m> <mean n>" per launch
template <class V>
static void trace_jobs(const char* kind, const V& jobs) {
    static const bool trace = std::getenv("H2_TRACE") != nullptr;
    if (!trace || jobs.empty()) return;
    double sm = 0, sn = 0;
    int mm = 0, mn = 0;
    for (const auto& j : jobs) {
        sm += j.m;
        sn += j.n;
        mm = std::max(mm, j.m);
        mn = std::max(mn, j.n);
    }
    std::fprintf(stderr, "h2jobs %s %zu %d %d %.1f %.1f\n", kind, jobs.size(), mm, mn, sm / jobs.size(),
                 sn / jobs.size());
}

void Runner::svd(double* B, int m, int n, int ldb, double* U, int ldu, double* sigma, int* count, double eps,
                 const int* rowperm, const int* ncols) {
    ensure_flag();
    svds_.push_back(SVDJob{B, U, sigma, count, d_flag_, nullptr, m, n, ldb, ldu, eps, rowperm, ncols});
    svd_maxn_ = std::max(svd_maxn_, n);
}

void Runner::flush_svd() {
    H2_SPAN("flush_svd");
    if (svds_.empty()) return;
    double* cnt = dev_counter();
    for (auto& j : svds_) j.flops = cnt;
    trace_jobs("svd", svds_);
    SVDJob* d = upload(svds_);
    double by = 0.0;
    for (auto& j : svds_) by += 8.0 * 3.0 * j.m * j.n;
    begin(5);
    // the low-precision forms run the row and column sides on two streams at once: a
    // cluster launch holds whole SMs that the other side's kernels could use (measured
    // on the n = 32768 workload: 235 -> 224 ms per product without clusters there; the
    // FP64 form, one stream, is faster with them: 1.33 against 1.34 s)
    launch_svd(d, (int)svds_.size(), svd_maxn_, st_, !low_precision(prec_));
    end(5, 0.0, by);
    marks_.back().dflops = cnt;
    ++launches;
    svds_.clear();
    svd_maxn_ = 0;
}

void Runner::jacobi_pre(const double* B, int m, int n, int ldb, double* V64, double* W64, const int* ncols) {
    if (V64 && ncols) throw Error(H2_ERR_ARG, "jacobi_pre: accumulated rotations with a device column count");
    float* W = (float*)dalloc(((size_t)m * n + 1) / 2);
    float* V = V64 ? (float*)dalloc(((size_t)n * n + 1) / 2) : nullptr;
    pres_.push_back(PreJob{B, W, V, V64, W64, nullptr, m, n, ldb, ncols});
}

void Runner::flush_pre() {
    H2_SPAN("flush_pre");
    if (pres_.empty()) return;
    double* cnt = dev_counter();
    for (auto& j : pres_) j.flops = cnt;
    PreJob* d = upload(pres_);
    double by = 0.0;
    for (auto& j : pres_) by += 8.0 * ((double)j.m * j.n + (double)j.n * j.n);
    size_t max_mn = 0, max_mnv = 0;
    for (auto& j : pres_) {
        max_mn = std::max(max_mn, (size_t)j.m * j.n);
        max_mnv = std::max(max_mnv, (size_t)(j.m + (j.V ? j.n : 0)) * j.n);
    }
    trace_jobs("pre", pres_);
    begin(6);
    launch_jacobi_pre(d, (int)pres_.size(), max_mn, max_mnv, st_, !low_precision(prec_));
    end(6, 0.0, by);
    marks_.back().dflops = cnt;
    ++launches;
    pres_.clear();
}

void Runner::pchol(const double* G, int k, int ldg, double* Z, int zrows, double rel_tol, double abs_tol,
                   int* rank) {
    if (k <= 0 || zrows <= 0) return;
    if (k > 1024) throw Error(H2_ERR_UNSUPPORTED, "weight matrix larger than 1024");
    chols_.push_back(CholJob{G, dalloc((size_t)k * k), Z, k, ldg, zrows, rel_tol, abs_tol, rank});
}

void Runner::flush_pchol() {
    H2_SPAN("flush_pchol");
    if (chols_.empty()) return;
    CholJob* d = upload(chols_);
    double fl = 0.0, by = 0.0;
    int max_k = 0;
    for (auto& j : chols_) {
        fl += (double)j.k * j.k * j.k / 3.0;
        by += 16.0 * j.k * j.k;
        max_k = std::max(max_k, j.k);
    }
    begin(4);
    launch_pchol(d, (int)chols_.size(), max_k, st_);
    end(4, fl, by);
    ++launches;
    chols_.clear();
}

void Runner::norm(const double* A, int m, int n, int lda, double* inv, double* nrm) {
    if (m > 2048 || n > 2048) throw Error(H2_ERR_UNSUPPORTED, "block too large for the norm kernel");
    norms_.push_back(NormJob{A, inv, nrm, m, n, lda});
}

void Runner::flush_norm() {
    H2_SPAN("flush_norm");
    if (norms_.empty()) return;
    NormJob* d = upload(norms_);
    double by = 0.0, fl = 0.0;
    for (auto& j : norms_) {
        by += 8.0 * j.m * j.n;
        fl += 4.0 * 61.0 * j.m * j.n;
    }
    begin(7);
    launch_norm(d, (int)norms_.size(), low_precision(prec_) ? H2_MIXED : H2_FP64, st_);
    end(7, fl, by);
    ++launches;
    norms_.clear();
}

void Runner::copy(const double* src, int lds, double* dst, int ldd, int rows, int cols, int trans, double alpha,
                  const double* scale, double beta) {
    if (rows <= 0 || cols <= 0) return;
    copies_.push_back(CopyJob{src, dst, scale, alpha, beta, rows, cols, lds, ldd, trans});
}

void Runner::flush_copy() {
    H2_SPAN("flush_copy");
    if (copies_.empty()) return;
    CopyJob* d = upload(copies_);
    double by = 0.0;
    for (auto& j : copies_) by += 8.0 * j.rows * j.cols * (j.beta != 0.0 ? 3.0 : 2.0);
    begin(8);
    launch_copy(d, (int)copies_.size(), st_);
    end(8, 0.0, by);
    ++launches;
    copies_.clear();
}

void Runner::flush_all() {
    flush_copy();
    flush_gemm();
    flush_norm();
    flush_qr();
    flush_svd();
}

template GTerm* Runner::upload<GTerm>(const std::vector<GTerm>&);
template GJob* Runner::upload<GJob>(const std::vector<GJob>&);
template GTile* Runner::upload<GTile>(const std::vector<GTile>&);
template QRJob* Runner::upload<QRJob>(const std::vector<QRJob>&);
template SVDJob* Runner::upload<SVDJob>(const std::vector<SVDJob>&);
template PreJob* Runner::upload<PreJob>(const std::vector<PreJob>&);
template CholJob* Runner::upload<CholJob>(const std::vector<CholJob>&);
template NormJob* Runner::upload<NormJob>(const std::vector<NormJob>&);
template CopyJob* Runner::upload<CopyJob>(const std::vector<CopyJob>&);
template SumSqJob* Runner::upload<SumSqJob>(const std::vector<SumSqJob>&);

cudaStream_t stream_of(const h2_opts* o) { return o ? (cudaStream_t)o->stream : (cudaStream_t)0; }

}  // namespace h2

using namespace h2;

static thread_local std::string g_last_error;

void h2_set_last_error(const char* m) { g_last_error = m ? m : ""; }


static int run_guarded(const std::function<void()>& f) {
    try {
        f();
        return H2_OK;
    } catch (const Error& e) {
        g_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return H2_ERR_OOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return H2_ERR_CUDA;
    }
}

extern "C" {

const char* h2_error_string(int code) {
    switch (code) {
        case H2_OK: return "success";
        case H2_ERR_ARG: return "invalid argument";
        case H2_ERR_SHAPE: return "operands do not share one cluster tree and block tree";
        case H2_ERR_OOM: return "out of memory";
        case H2_ERR_NUMERIC: return "non-finite value";
        case H2_ERR_TIMEOUT: return "iteration limit reached";
        case H2_ERR_UNSUPPORTED: return "unsupported case";
        case H2_ERR_CUDA: return "CUDA runtime error";
        default: return "unknown error";
    }
}

const char* h2_last_error_message(void) { return g_last_error.c_str(); }

// widening of the double-layer interpolation boxes (each extent >= this fraction of the largest)
constexpr double kDlpFat = 0.25;

// A host view of n x 3 doubles given in host memory or in device memory of the
// current device (copied to `buf` in the latter case).
static const double* host_view(const double* p, int64_t n, std::vector<double>& buf) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // plain host memory on older drivers
        return p;
    }
    if (at.type != cudaMemoryTypeDevice) return p;  // host, registered or managed memory
    buf.resize((size_t)3 * n);
    H2_CUDA(cudaMemcpy(buf.data(), p, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost));
    return buf.data();
}

static int build_interp(const double* points_in, const double* normals_in, int64_t n, int kernel, int leaf_size,
                        double eta, int cheb_order, const h2_opts* opts, h2_matrix** out) {
    if (!points_in || !out || n < 1 || leaf_size < 1 || cheb_order < 1 || cheb_order > 8 || !(eta >= 0.0) ||
        !std::isfinite(eta) || kernel < H2_K_LAPLACE || kernel > H2_K_DLP)
        return H2_ERR_ARG;
    const bool dlp = (kernel == H2_K_DLP);
    if (dlp && !normals_in) return H2_ERR_ARG;
    std::vector<double> pbuf, nbuf;
    const double* points = points_in;
    const double* normals = normals_in;
    int rc = run_guarded([&] {
        points = host_view(points_in, n, pbuf);
        if (dlp) normals = host_view(normals_in, n, nbuf);
    });
    if (rc != H2_OK) return rc;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!std::isfinite(points[i]) || (dlp && !std::isfinite(normals[i]))) return H2_ERR_NUMERIC;
    return run_guarded([&] {
        cudaStream_t st = stream_of(opts);
        AllocScope scope(alloc_of(opts), st);
        auto M = std::make_unique<h2_matrix>();
        H2_CUDA(cudaGetDevice(&M->device));
        M->st = build_structure(points, n, leaf_size, eta);
        M->kernel = kernel;
        M->order = cheb_order;
        const Tree& T = M->st->tree;
        const BlockTree& B = M->st->blocks;
        const int m = cheb_order, k = m * m * m;
        Runner R(st, H2_FP64);
        // structure arrays on the device
        double* d_pts = R.upload(M->st->points);
        int64_t* d_perm = R.upload(T.perm);
        int64_t* d_off = R.upload(T.off);
        int64_t* d_size = R.upload(T.size);
        // interpolation boxes: the bounding boxes, or for the double-layer kernel the
        // bounding boxes with every extent widened to >= 1/4 of the largest (the normal
        // derivative across the vanishing extent of a flat surface cluster is ill-conditioned)
        std::vector<double> blo = T.lo, bhi = T.hi;
        if (dlp) {
            for (int c = 0; c < T.nc; ++c) {
                double* l = &blo[3 * c];
                double* h = &bhi[3 * c];
                const double need = kDlpFat * std::max({h[0] - l[0], h[1] - l[1], h[2] - l[2]});
                for (int a = 0; a < 3; ++a)
                    if (h[a] - l[a] < need) {
                        const double mid = 0.5 * (l[a] + h[a]);
                        l[a] = mid - 0.5 * need;
                        h[a] = mid + 0.5 * need;
                    }
            }
        }
        double* d_lo = R.upload(blo);
        double* d_hi = R.upload(bhi);
        // basis: leaves + transfers in one chunk
        auto V = std::make_shared<Basis>();
        V->rank.assign(T.nc, k);
        V->leaf.assign(T.nc, nullptr);
        V->tr.assign(T.nc, nullptr);
        size_t total = 0;
        for (int c = 0; c < T.nc; ++c) {
            if (T.is_leaf(c)) total += (size_t)T.size[c] * k;
            if (c > 0) total += (size_t)k * k;
        }
        auto chunk = std::make_shared<DevBuf>();
        chunk->alloc(total);
        V->chunks.push_back(chunk);
        size_t o = 0;
        int64_t max_size = 0;
        for (int c = 0; c < T.nc; ++c) {
            if (T.is_leaf(c)) {
                V->leaf[c] = chunk->p + o;
                o += (size_t)T.size[c] * k;
                max_size = std::max(max_size, T.size[c]);
            }
            if (c > 0) {
                V->tr[c] = chunk->p + o;
                o += (size_t)k * k;
            }
        }
        double** d_leafp = R.upload(V->leaf);
        double** d_trp = R.upload(V->tr);
        launch_interp_leaf(d_pts, nullptr, d_perm, d_off, d_size, d_lo, d_hi, d_leafp, Tree::first(T.L),
                           Tree::count(T.L), m, max_size, st);
        launch_interp_transfer(d_lo, d_hi, d_trp, T.nc, m, st);
        // double-layer kernel: the column basis holds the normal derivatives (own leaves and transfers)
        std::shared_ptr<Basis> W = V;
        double* d_nrm = nullptr;
        if (dlp) {
            d_nrm = R.upload(std::vector<double>(normals, normals + 3 * n));
            W = std::make_shared<Basis>();
            W->rank = V->rank;
            W->leaf.assign(T.nc, nullptr);
            W->tr.assign(T.nc, nullptr);
            auto wchunk = std::make_shared<DevBuf>();
            wchunk->alloc(total);
            W->chunks.push_back(wchunk);
            for (int c = 0; c < T.nc; ++c) {
                if (V->leaf[c]) W->leaf[c] = wchunk->p + (V->leaf[c] - chunk->p);
                if (V->tr[c]) W->tr[c] = wchunk->p + (V->tr[c] - chunk->p);
            }
            launch_interp_leaf(d_pts, d_nrm, d_perm, d_off, d_size, d_lo, d_hi, R.upload(W->leaf), Tree::first(T.L),
                               Tree::count(T.L), m, max_size, st);
            launch_interp_transfer(d_lo, d_hi, R.upload(W->tr), T.nc, m, st);
            uint64_t h = 1469598103934665603ull;  // FNV-1a over the normals' bytes
            const unsigned char* b = (const unsigned char*)normals;
            for (size_t i = 0; i < sizeof(double) * 3 * (size_t)n; ++i) h = (h ^ b[i]) * 1099511628211ull;
            M->wtag = h | 1;
            M->vtag = 1;
        }
        // couplings and dense blocks
        size_t stot = 0, ntot = 0;
        int nb = (int)B.kind.size();
        M->blk.assign(nb, nullptr);
        for (int b = 0; b < nb; ++b) {
            if (B.kind[b] == ADM) stot += (size_t)k * k;
            if (B.kind[b] == DENSE) ntot += (size_t)T.size[B.t[b]] * T.size[B.s[b]];
        }
        auto cs = std::make_shared<DevBuf>(), cn = std::make_shared<DevBuf>();
        cs->alloc(stot);
        cn->alloc(ntot);
        M->chunks = {cs, cn};
        std::vector<int> at, as, dt, ds;
        std::vector<double*> ap, dp;
        size_t so = 0, no = 0;
        for (int b = 0; b < nb; ++b) {
            if (B.kind[b] == ADM) {
                M->blk[b] = cs->p + so;
                so += (size_t)k * k;
                at.push_back(B.t[b]);
                as.push_back(B.s[b]);
                ap.push_back(M->blk[b]);
            } else if (B.kind[b] == DENSE) {
                M->blk[b] = cn->p + no;
                no += (size_t)T.size[B.t[b]] * T.size[B.s[b]];
                dt.push_back(B.t[b]);
                ds.push_back(B.s[b]);
                dp.push_back(M->blk[b]);
            }
        }
        launch_interp_coupling(d_lo, d_hi, R.upload(at), R.upload(as), R.upload(ap), (int)at.size(), m, kernel, st);
        launch_interp_dense(d_pts, d_nrm, d_perm, d_off, d_size, R.upload(dt), R.upload(ds), R.upload(dp),
                            (int)dt.size(), kernel, st);
        M->V = V;
        M->W = W;
        H2_CUDA(cudaGetLastError());
        R.release_all();
        H2_CUDA(cudaStreamSynchronize(st));
        *out = M.release();
    });
}

int h2_build_interp(const double* points, int64_t n, int kernel, int leaf_size, double eta, int cheb_order,
                    const h2_opts* opts, h2_matrix** out) {
    return build_interp(points, nullptr, n, kernel, leaf_size, eta, cheb_order, opts, out);
}

int h2_build_interp_normals(const double* points, const double* normals, int64_t n, int kernel, int leaf_size,
                            double eta, int cheb_order, const h2_opts* opts, h2_matrix** out) {
    return build_interp(points, normals, n, kernel, leaf_size, eta, cheb_order, opts, out);
}

int h2_to_dense(const h2_matrix* A, double* out, int64_t ld, int out_on_device, const h2_opts* opts) {
    if (!A || !out || ld < A->st->tree.n) return H2_ERR_ARG;
    return run_guarded([&] {
        cudaStream_t st = stream_of(opts);
        AllocScope scope(alloc_of(opts), st);
        const Tree& T = A->st->tree;
        const BlockTree& B = A->st->blocks;
        const int64_t n = T.n;
        Runner R(st, H2_FP64);
        // expanded bases per cluster: rows of the cluster x rank
        auto expand = [&](const Basis& b) {
            std::vector<double*> ex(T.nc, nullptr);
            for (int c = 0; c < T.nc; ++c) ex[c] = R.dalloc((size_t)T.size[c] * std::max(1, b.rank[c]));
            for (int c = Tree::first(T.L); c < T.nc; ++c)
                R.copy(b.leaf[c], (int)T.size[c], ex[c], (int)T.size[c], (int)T.size[c], b.rank[c], 0);
            R.flush_copy();
            for (int l = T.L - 1; l >= 0; --l) {
                for (int c = Tree::first(l); c < Tree::first(l) + Tree::count(l); ++c) {
                    for (int i = 0; i < 2; ++i) {
                        int ch = Tree::child(c, i);
                        R.job(ex[c] + (T.off[ch] - T.off[c]), (int)T.size[ch], b.rank[c], (int)T.size[c], 0.0);
                        R.term(ex[ch], 0, (int)T.size[ch], b.tr[ch], 0, b.rank[ch], b.rank[ch]);
                    }
                }
                R.flush_gemm(H2_FP64);
            }
            return ex;
        };
        auto ev = expand(*A->V);
        auto ew = (A->W == A->V) ? ev : expand(*A->W);
        double* dense = R.dalloc((size_t)n * n);
        H2_CUDA(cudaMemsetAsync(dense, 0, sizeof(double) * n * n, st));
        std::vector<double*> tmp(B.kind.size(), nullptr);
        for (int b = 0; b < (int)B.kind.size(); ++b) {
            int t = B.t[b], s = B.s[b];
            if (B.kind[b] == ADM) {
                tmp[b] = R.dalloc((size_t)T.size[t] * std::max(1, A->W->rank[s]));
                R.job(tmp[b], (int)T.size[t], A->W->rank[s], (int)T.size[t], 0.0);
                R.term(ev[t], 0, (int)T.size[t], A->blk[b], 0, A->V->rank[t], A->V->rank[t]);
            } else if (B.kind[b] == DENSE) {
                R.copy(A->blk[b], (int)T.size[t], dense + T.off[t] + T.off[s] * n, (int)n, (int)T.size[t],
                       (int)T.size[s], 0);
            }
        }
        R.flush_gemm(H2_FP64);
        R.flush_copy();
        for (int b = 0; b < (int)B.kind.size(); ++b) {
            int t = B.t[b], s = B.s[b];
            if (B.kind[b] != ADM) continue;
            R.job(dense + T.off[t] + T.off[s] * n, (int)T.size[t], (int)T.size[s], (int)n, 0.0);
            R.term(tmp[b], 0, (int)T.size[t], ew[s], 1, (int)T.size[s], A->W->rank[s]);
        }
        R.flush_gemm(H2_FP64);
        int64_t* d_perm = R.upload(T.perm);
        double* target = out;
        if (!out_on_device) target = R.dalloc((size_t)ld * n);
        launch_scatter_dense(dense, n, d_perm, target, ld, st);
        if (!out_on_device)
            H2_CUDA(cudaMemcpyAsync(out, target, sizeof(double) * ld * n, cudaMemcpyDeviceToHost, st));
        H2_CUDA(cudaGetLastError());
        H2_CUDA(cudaStreamSynchronize(st));
        R.release_all();
        H2_CUDA(cudaStreamSynchronize(st));
    });
}

int h2_info(const h2_matrix* A, h2_info_t* info) {
    if (!A || !info) return H2_ERR_ARG;
    const Tree& T = A->st->tree;
    const BlockTree& B = A->st->blocks;
    info->n = T.n;
    info->depth = T.L;
    info->nclusters = T.nc;
    info->nblocks = (int64_t)B.kind.size();
    info->nadmissible = B.count(ADM);
    info->ndense = B.count(DENSE);
    info->leaf_size = T.leaf_size;
    info->order = A->order;
    info->eta = A->st->eta;
    info->max_row_rank = A->V->max_rank();
    info->max_col_rank = A->W->max_rank();
    double bytes = A->V->bytes() + (A->W != A->V ? A->W->bytes() : 0.0);
    for (auto& c : A->chunks) bytes += 8.0 * c->len;
    info->device_bytes = bytes;
    return H2_OK;
}

int h2_get_structure(const h2_matrix* A, int64_t* perm, int64_t* offsets, int64_t* sizes, int* row_ranks,
                     int* col_ranks) {
    if (!A) return H2_ERR_ARG;
    const Tree& T = A->st->tree;
    if (perm) std::copy(T.perm.begin(), T.perm.end(), perm);
    if (offsets) std::copy(T.off.begin(), T.off.end(), offsets);
    if (sizes) std::copy(T.size.begin(), T.size.end(), sizes);
    if (row_ranks) std::copy(A->V->rank.begin(), A->V->rank.end(), row_ranks);
    if (col_ranks) std::copy(A->W->rank.begin(), A->W->rank.end(), col_ranks);
    return H2_OK;
}

int h2_clone(const h2_matrix* A, const h2_opts* opts, h2_matrix** out) {
    if (!A || !out) return H2_ERR_ARG;
    return run_guarded([&] {
        cudaStream_t st = stream_of(opts);
        AllocScope scope(alloc_of(opts), st);
        auto M = std::make_unique<h2_matrix>();
        M->st = A->st;
        M->kernel = A->kernel;
        M->order = A->order;
        M->device = A->device;
        M->vtag = A->vtag;
        M->wtag = A->wtag;
        // copy every chunk and translate the pointers into it
        std::vector<std::pair<const DevBuf*, DevBuf*>> map;
        auto dup = [&](const std::vector<std::shared_ptr<DevBuf>>& src, std::vector<std::shared_ptr<DevBuf>>& dst) {
            for (auto& c : src) {
                auto d = std::make_shared<DevBuf>();
                d->alloc(c->len);
                if (c->len) H2_CUDA(cudaMemcpyAsync(d->p, c->p, 8 * c->len, cudaMemcpyDeviceToDevice, st));
                map.push_back({c.get(), d.get()});
                dst.push_back(d);
            }
        };
        auto tr = [&](const double* p) -> double* {
            if (!p) return nullptr;
            for (auto& [a, b] : map)
                if (p >= a->p && p < a->p + a->len) return b->p + (p - a->p);
            throw Error(H2_ERR_ARG, "pointer outside the handle's buffers");
        };
        auto cloneb = [&](const Basis& B) {
            auto nb = std::make_shared<Basis>();
            nb->rank = B.rank;
            dup(B.chunks, nb->chunks);
            for (double* p : B.leaf) nb->leaf.push_back(tr(p));
            for (double* p : B.tr) nb->tr.push_back(tr(p));
            return nb;
        };
        M->V = cloneb(*A->V);
        M->W = (A->W == A->V) ? M->V : cloneb(*A->W);
        dup(A->chunks, M->chunks);
        for (double* p : A->blk) M->blk.push_back(tr(p));
        H2_CUDA(cudaStreamSynchronize(st));
        *out = M.release();
    });
}

int h2_plan_structure(const double* points, int64_t n, int leaf_size, double eta, int64_t* perm, int64_t* counts) {
    if (!points || n < 1 || leaf_size < 1 || !(eta >= 0.0) || !std::isfinite(eta)) return H2_ERR_ARG;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!std::isfinite(points[i])) return H2_ERR_NUMERIC;
    return run_guarded([&] {
        auto st = build_structure(points, n, leaf_size, eta);
        if (perm) std::copy(st->tree.perm.begin(), st->tree.perm.end(), perm);
        if (counts) {
            ProductTree P = build_product_tree(st->blocks, st->blocks);
            int64_t tri = 0;
            for (auto& v : P.triples) tri += (int64_t)v.size();
            counts[0] = st->tree.L;
            counts[1] = st->blocks.count(ADM);
            counts[2] = st->blocks.count(DENSE);
            counts[3] = st->blocks.count(SPLIT);
            counts[4] = P.nodes.count(ADM);
            counts[5] = P.nodes.count(DENSE);
            counts[6] = P.nodes.count(SPLIT);
            counts[7] = tri;
        }
    });
}

int h2_library_memory(int64_t* current_bytes, int64_t* peak_bytes, int reset_peak) {
    if (current_bytes) *current_bytes = g_own_bytes.load();
    if (peak_bytes) *peak_bytes = g_own_peak.load();
    if (reset_peak) g_own_peak.store(g_own_bytes.load());
    return H2_OK;
}

// Every entry point returns after its work on the handle has finished, so the
// buffers are free to go without waiting for the device.
void h2_free(h2_matrix* A) {
    if (!A) return;
    delete A;
}

}  // extern "C"
