// Device kernels of the H^2 product library (sm_103a).
//
// Batched small dense linear algebra: every launch covers all clusters or all
// blocks of one tree level at once.  Each batched kernel reads a device array
// of job descriptors built by the host executor.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>

#include "h2_internal.h"

namespace h2 {

// ------------------------------------------------------------------ GEMM
// C = beta C + sum_terms alpha_t op(A_t) op(B_t) over 32 x 32 output tiles,
// in FP64 (H2_FP64).
constexpr int GB = 32;   // tile edge
constexpr int GK = 16;   // k-chunk
constexpr int GT = 256;  // threads: 16 x 16, each 2 x 2 outputs

template <class T>
__global__ void __launch_bounds__(GT) k_gemm(const GTerm* __restrict__ terms, const GJob* __restrict__ jobs,
                                             const GTile* __restrict__ tiles) {
    __shared__ T As[GK][GB + 1];
    __shared__ T Bs[GK][GB + 1];
    const GTile tile = tiles[blockIdx.x];
    const GJob J = jobs[tile.job];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // warp-uniform halves of the 2 x 2 register block that hold no output of the
    // job (edge tiles of ranks that are not multiples of 32): their FMAs are skipped
    const bool row1 = tile.i0 + 16 < J.m;
    const int wty = (threadIdx.x >> 5) * 2;  // the warp's first column index ty
    const bool col0 = tile.j0 + wty < J.n, col1 = tile.j0 + wty + 16 < J.n;
    T acc[2][2] = {{0, 0}, {0, 0}};
    for (int it = 0; it < J.nt; ++it) {
        const GTerm P = terms[J.t0 + it];
        const double f = P.alpha * (P.scale ? *P.scale : 1.0);
        if (f == 0.0) continue;
        const bool scaled = (f != 1.0);
        for (int k0 = 0; k0 < P.k; k0 += GK) {
            // stage op(A)[i0:i0+32, k0:k0+16] and op(B)[k0:k0+16, j0:j0+32]
            for (int e = threadIdx.x; e < GK * GB; e += GT) {
                int i, kk;
                if (!P.ta) { i = e % GB; kk = e / GB; } else { kk = e % GK; i = e / GK; }
                int gi = tile.i0 + i, gk = k0 + kk;
                double v = 0.0;
                if (gi < J.m && gk < P.k) v = P.ta ? P.A[gk + (size_t)gi * P.lda] : P.A[gi + (size_t)gk * P.lda];
                As[kk][i] = (T)(scaled ? f * v : v);
                int j;
                if (!P.tb) { kk = e % GK; j = e / GK; } else { j = e % GB; kk = e / GB; }
                int gj = tile.j0 + j;
                gk = k0 + kk;
                double w = 0.0;
                if (gj < J.n && gk < P.k) w = P.tb ? P.B[gj + (size_t)gk * P.ldb] : P.B[gk + (size_t)gj * P.ldb];
                Bs[kk][j] = (T)w;
            }
            __syncthreads();
            auto mac = [&](int kk) {
                T a0 = As[kk][tx], a1 = As[kk][tx + 16];
                T b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
                if (col0) {
                    acc[0][0] += a0 * b0;
                    if (row1) acc[1][0] += a1 * b0;
                }
                if (col1) {
                    acc[0][1] += a0 * b1;
                    if (row1) acc[1][1] += a1 * b1;
                }
            };
            const int kc = min(GK, P.k - k0);  // the last chunk of a term is partial: skip its zero padding
            if (kc == GK) {
#pragma unroll
                for (int kk = 0; kk < GK; ++kk) mac(kk);
            } else {
#pragma unroll 2
                for (int kk = 0; kk < kc; ++kk) mac(kk);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int gi = tile.i0 + tx + 16 * a, gj = tile.j0 + ty + 16 * b;
            if (gi < J.m && gj < J.n) {
                double* c = J.C + gi + (size_t)gj * J.ldc;
                double v = (double)acc[a][b];
                *c = (J.beta == 0.0) ? v : J.beta * *c + v;
                if (J.sym && tile.i0 != tile.j0) {
                    double* ct = J.C + gj + (size_t)gi * J.ldc;
                    *ct = (J.beta == 0.0) ? v : J.beta * *ct + v;
                }
            }
        }
}

// FP32 forms on kF32Tile x kF32Tile output tiles: 256 threads, each a 4 x 4
// register block.  The (term, K chunk) sequence of a job is pipelined: while
// one chunk is multiplied from shared memory, the next one is in flight as raw
// FP64 values in registers and is converted only when it is stored to shared
// memory.  The term descriptors and their factors are cached in shared memory,
// 32 at a time.
//  DF = false (H2_MIXED products): operands rounded to FP32, FP32 accumulation.
//  DF = true (FP64-accurate products of the low-precision modes): double-float
//    arithmetic (Dekker 1971).  Every operand is split as v = hi + lo with two
//    FP32 values (48 bits); a product contributes hi_a hi_b exactly (the FMA
//    residual) plus the cross terms hi_a lo_b + lo_a hi_b, and the sum is kept
//    as an unevaluated pair S + s with an error-free TwoSum (Knuth) per term.
//    Relative accuracy about 2^-46 per product at ~12 FP32 operations per
//    multiply-add, against the 1/64-rate FP64 pipe.
constexpr int G32TB = 32;  // cached term descriptors

// FP64 -> FP32 with round to nearest (ties away from zero) by integer
// operations on the IEEE 754 encodings, so that the conversion stays off the
// FP64 pipe.  Magnitudes below the FP32 normal range give zero, magnitudes
// from 2^128 up (and NaN) give infinity.
__device__ __forceinline__ float f64_to_f32(double v) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned e = (hi >> 20) & 0x7ffu;
    unsigned r = __funnelshift_r(lo, hi, 29);  // 9 low exponent bits, 23 leading mantissa bits
    r += (lo >> 28) & 1u;                      // round on the 29 dropped bits
    r -= 896u << 23;                           // exponent bias 1023 -> 127
    const unsigned mag = (e < 897u) ? 0u : (e > 1150u) ? 0x7f800000u : r;
    return __uint_as_float((hi & 0x80000000u) | mag);
}

// exact FP32 -> FP64 widening by integer operations (FP32 subnormals give
// zero, infinities and NaN keep their class)
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned sgn = u & 0x80000000u;
    if (e == 0u) return __hiloint2double((int)sgn, 0);
    const unsigned eh = (e == 255u) ? 0x7ff00000u : ((e + 896u) << 20);
    return __hiloint2double((int)(sgn | eh | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}

// v = hi + lo with hi = v rounded to FP32 (f64_to_f32) and lo = the remainder
// v - hi (exact in FP64) rounded to FP32, without the FP64 pipe: the remainder
// is R 2^(e-1075) with R the 29 mantissa bits that hi drops, less 2^29 where hi
// rounded up (|R| <= 2^28), converted to FP32 and scaled by powers of two.
// lo is zero where hi is zero or infinite.
__device__ __forceinline__ void split_f64(double v, float& hi, float& lo) {
    const unsigned h = (unsigned)__double2hiint(v), l = (unsigned)__double2loint(v);
    const unsigned e = (h >> 20) & 0x7ffu;
    hi = f64_to_f32(v);
    const int R = (int)(l & 0x1fffffffu) - (int)(l & 0x10000000u) * 2;
    const unsigned c = (e < 1011u) ? 64u : 0u;  // keeps the first scale factor normal
    const float s1 = __uint_as_float((h & 0x80000000u) | ((e + c - 948u) << 23));  // +-2^(e-1075+c)
    const float s2 = __uint_as_float((127u - c) << 23);                              // 2^-c
    lo = (e < 897u || e > 1150u) ? 0.f : __fmul_rn(__fmul_rn(__int2float_rn(R), s1), s2);
}

// the 4 values of a 16-byte shared-memory load whose elements are permuted by c -> c ^ Q
template <int Q>
__device__ __forceinline__ void unpack4(const float4 v, float* o) {
    const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = w[c ^ Q];
}

template <bool DF>
__global__ void __launch_bounds__(GT, DF ? 2 : 3) k_gemm_f32(const GTerm* __restrict__ terms,
                                                              const GJob* __restrict__ jobs,
                                                              const GTile* __restrict__ tiles) {
    constexpr int KC = DF ? 16 : 32;            // K chunk
    constexpr int NE = kF32Tile * KC / GT;      // staged elements per thread and operand
    constexpr int NP = DF ? 2 : 1;              // FP32 planes per operand
    // Row kk of a staged tile holds 64 values in 16 groups of 4: group g sits
    // at g ^ sh(kk) and element c of a group at c ^ sq(kk).  Staging along a
    // row and along a column is then free of bank conflicts, and each thread
    // reads its 4 values of a row as one 16-byte load (2 wavefronts a warp).
    // two stages: the chunk being multiplied and the next one being stored
    __shared__ __align__(16) float As[2][NP][KC][kF32Tile];
    __shared__ __align__(16) float Bs[2][NP][KC][kF32Tile];
    __shared__ GTerm tc[G32TB];
    __shared__ double tf[G32TB];
    __shared__ int tbase;
    const GTile tile = tiles[blockIdx.x];
    const GJob J = jobs[tile.job];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // rows 4 tx + x, columns 4 ty + y
    // warp w holds the columns 8 w .. 8 w + 7 of the tile (ty = 2 w, 2 w + 1): in an
    // edge tile the warps wholly beyond the job skip their multiply-adds (warp-uniform)
    const bool cols_live = tile.j0 + 8 * (int)(threadIdx.x >> 5) < J.n;
    auto sh = [](int kk) { return DF ? (kk >> 1) & 7 : (kk >> 2) & 7; };
    auto sidx = [&](int kk, int i) { return (((i >> 2) ^ sh(kk)) << 2) | ((i & 3) ^ (DF ? (kk & 1) << 1 : kk & 3)); };
    float acc[4][4], cor[4][4];  // cor: low parts of the double-float sums (DF only)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = cor[a][b] = 0.f;
    if (threadIdx.x == 0) tbase = -G32TB;
    __syncthreads();
    // term it of the job from the cache (loads the batch holding it; all threads call this together)
    auto term_at = [&](int it, GTerm& P, double& f) {
        if (it < tbase || it >= tbase + G32TB) {
            __syncthreads();
            const int b0 = it - it % G32TB;
            if (threadIdx.x < G32TB && b0 + (int)threadIdx.x < J.nt) {
                const GTerm t = terms[J.t0 + b0 + threadIdx.x];
                tc[threadIdx.x] = t;
                tf[threadIdx.x] = t.alpha * (t.scale ? *t.scale : 1.0);
            }
            if (threadIdx.x == 0) tbase = b0;
            __syncthreads();
        }
        P = tc[it - tbase];
        f = tf[it - tbase];
    };
    // the chunk after (it, k0), skipping terms with a zero factor or no columns
    auto advance = [&](int& it, int& k0, GTerm& P, double& f) -> bool {
        if (it >= 0 && k0 + KC < P.k) {
            k0 += KC;
            return true;
        }
        for (++it; it < J.nt; ++it) {
            term_at(it, P, f);
            if ((__double_as_longlong(f) << 1) != 0 && P.k > 0) {  // nonzero factor (an integer test)
                k0 = 0;
                return true;
            }
        }
        return false;
    };
    // Element r of a thread (e = threadIdx.x + r GT) lies in one of two
    // families: "N" at (row, k) = (e mod 64, e / 64) = (n_i, n_k + (GT/64) r)
    // and "T" at (k, row) = (e mod KC, e / KC) = (t_k, t_i + (GT/KC) r).  A
    // plain A and a transposed B use N, the others T; addresses and staged
    // offsets are a base plus a compile-time step per r (the swizzle adds an
    // XOR: r << 2 or r << 3 for N, r << 3 or r << 4 for T).
    const int n_i = threadIdx.x % kF32Tile, n_k = threadIdx.x / kF32Tile;
    const int t_k = threadIdx.x % KC, t_i = threadIdx.x / KC;
    const int offN = n_k * kF32Tile + sidx(n_k, n_i), offT = t_k * kF32Tile + sidx(t_k, t_i);
    auto soff = [&](bool tfam, int r) {
        return tfam ? (offT ^ (r << (DF ? 4 : 3))) : ((offN ^ (r << (DF ? 3 : 2))) + r * (GT / kF32Tile) * kF32Tile);
    };
    double ra[NE], rb[NE];
    auto fetch = [&](const GTerm& P, int k0) {
        {  // A (m x k): N when plain, T when transposed
            const bool tf_ = P.ta;
            const int row = tile.i0 + (tf_ ? t_i : n_i), rs = tf_ ? GT / KC : 0;
            const int kq = k0 + (tf_ ? t_k : n_k), ks = tf_ ? 0 : GT / kF32Tile;
            const double* a = tf_ ? P.A + kq + (size_t)row * P.lda : P.A + row + (size_t)kq * P.lda;
            const size_t as = (size_t)(tf_ ? rs : ks) * P.lda;
#pragma unroll
            for (int r = 0; r < NE; ++r) ra[r] = (row + rs * r < J.m && kq + ks * r < P.k) ? a[r * as] : 0.0;
        }
        {  // B (k x n): T when plain, N when transposed
            const bool tf_ = !P.tb;
            const int col = tile.j0 + (tf_ ? t_i : n_i), cs = tf_ ? GT / KC : 0;
            const int kq = k0 + (tf_ ? t_k : n_k), ks = tf_ ? 0 : GT / kF32Tile;
            const double* b = tf_ ? P.B + kq + (size_t)col * P.ldb : P.B + col + (size_t)kq * P.ldb;
            const size_t bs = (size_t)(tf_ ? cs : ks) * P.ldb;
#pragma unroll
            for (int r = 0; r < NE; ++r) rb[r] = (col + cs * r < J.n && kq + ks * r < P.k) ? b[r * bs] : 0.0;
        }
    };
    // one k step; D = kk mod 4, known at compile time, fixes the in-group order
    auto mac = [&](int sg, int kk, auto D) {
        constexpr int q = DF ? (decltype(D)::value & 1) << 1 : decltype(D)::value;
        float a[4], b[4];
        const float4 va = *reinterpret_cast<const float4*>(&As[sg][0][kk][(tx ^ sh(kk)) << 2]);
        const float4 vb = *reinterpret_cast<const float4*>(&Bs[sg][0][kk][(ty ^ sh(kk)) << 2]);
        unpack4<q>(va, a);
        unpack4<q>(vb, b);
        if constexpr (!DF) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        } else {
            float al[4], bl[4];
            unpack4<q>(*reinterpret_cast<const float4*>(&As[sg][NP - 1][kk][(tx ^ sh(kk)) << 2]), al);
            unpack4<q>(*reinterpret_cast<const float4*>(&Bs[sg][NP - 1][kk][(ty ^ sh(kk)) << 2]), bl);
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const float p = __fmul_rn(a[x], b[y]);
                    float e = __fmaf_rn(a[x], b[y], -p);  // a_hi b_hi - p exactly
                    e = __fmaf_rn(a[x], bl[y], e);
                    e = __fmaf_rn(al[x], b[y], e);
                    const float S = acc[x][y];
                    const float t = __fadd_rn(S, p);  // TwoSum(S, p)
                    const float z = __fsub_rn(t, S);
                    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(p, z));
                    cor[x][y] = __fadd_rn(cor[x][y], __fadd_rn(err, e));
                    acc[x][y] = t;
                }
        }
    };
    // the staged chunk (raw values of term P in ra / rb) goes to shared-memory stage sg,
    // A scaled by the term's factor f
    auto store = [&](int sg, const GTerm& P, double f) {
        const float cf32 = DF ? 0.f : f64_to_f32(f);
        const bool unit = (f == 1.0 || f == -1.0);  // the same for the whole block
        const float sgn = (f < 0.0) ? -1.f : 1.f;
        float fh = 0.f, fl = 0.f;  // the factor as a double-float pair (DF)
        if constexpr (DF) split_f64(f, fh, fl);
        float* const as0 = &As[sg][0][0][0];
        float* const bs0 = &Bs[sg][0][0][0];
        constexpr int PL = KC * kF32Tile;  // floats per plane
#pragma unroll
        for (int r = 0; r < NE; ++r) {
            const int pa = soff(P.ta != 0, r), pb = soff(P.tb == 0, r);
            if constexpr (!DF) {
                as0[pa] = cf32 * f64_to_f32(ra[r]);
                bs0[pb] = f64_to_f32(rb[r]);
            } else {
                float ah, al, bh, bl;
                if (unit) {  // factor +-1: applied to the split exactly
                    split_f64(ra[r], ah, al);
                    ah *= sgn;
                    al *= sgn;
                } else {
                    // the factor applied in double-float arithmetic on the FP32 pipe
                    // (an FP64 multiply per element would load the 1/64-rate FP64 pipe):
                    // (xh + xl)(fh + fl) = p + e exactly up to xl fl, then Fast2Sum
                    float xh, xl;
                    split_f64(ra[r], xh, xl);
                    const float p = __fmul_rn(xh, fh);
                    float e = __fmaf_rn(xh, fh, -p);
                    e = __fmaf_rn(xh, fl, e);
                    e = __fmaf_rn(xl, fh, e);
                    ah = __fadd_rn(p, e);
                    al = __fsub_rn(e, __fsub_rn(ah, p));
                }
                split_f64(rb[r], bh, bl);
                as0[pa] = ah;
                as0[PL + pa] = al;
                bs0[pb] = bh;
                bs0[PL + pb] = bl;
            }
        }
    };
    int cit = -1, ck0 = 0;
    GTerm CP;
    double cf = 0.0;
    bool have = advance(cit, ck0, CP, cf);
    int sg = 0;
    if (have) {
        fetch(CP, ck0);
        store(0, CP, cf);
    }
    __syncthreads();
    // one barrier per chunk: the next chunk is fetched before the multiply-adds of
    // this one and stored into the other stage after them
    while (have) {
        const int kc = min(KC, CP.k - ck0);
        int nit = cit, nk0 = ck0;
        GTerm NP_ = CP;
        double nf = cf;
        const bool more = advance(nit, nk0, NP_, nf);  // may sync (term cache)
        if (more) fetch(NP_, nk0);
        // rows kc .. KC-1 hold zeros, so a partial chunk may run to a multiple of 4
        constexpr std::integral_constant<int, 0> d0;
        constexpr std::integral_constant<int, 1> d1;
        constexpr std::integral_constant<int, 2> d2;
        constexpr std::integral_constant<int, 3> d3;
        if (!cols_live) {
            // this warp's 8 columns lie wholly beyond the job (an edge tile): nothing to add
        } else if (!DF && kc == KC) {  // (the double-float step is long: its loop stays rolled for the instruction cache)
#pragma unroll
            for (int kk = 0; kk < KC; kk += 4) {
                mac(sg, kk, d0);
                mac(sg, kk + 1, d1);
                mac(sg, kk + 2, d2);
                mac(sg, kk + 3, d3);
            }
        } else {
#pragma unroll 1
            for (int kk = 0; kk < kc; kk += 4) {
                mac(sg, kk, d0);
                mac(sg, kk + 1, d1);
                mac(sg, kk + 2, d2);
                mac(sg, kk + 3, d3);
            }
        }
        if constexpr (DF) {
            // renormalise the pairs so that the low parts stay small (Fast2Sum)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const float t = __fadd_rn(acc[x][y], cor[x][y]);
                    cor[x][y] = __fsub_rn(cor[x][y], __fsub_rn(t, acc[x][y]));
                    acc[x][y] = t;
                }
        }
        // the other stage was last read in the previous chunk, before the barrier below it
        if (more) store(sg ^ 1, NP_, nf);
        __syncthreads();
        sg ^= 1;
        cit = nit;
        ck0 = nk0;
        CP = NP_;
        cf = nf;
        have = more;
    }
    const bool beta0 = (__double_as_longlong(J.beta) << 1) == 0;  // (integer tests keep the
    const bool mirror = J.sym && tile.i0 != tile.j0;                 //  FP64 pipe for the sums)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gi = tile.i0 + 4 * tx + a, gj = tile.j0 + 4 * ty + b;
            if (gi < J.m && gj < J.n) {
                double* c = J.C + gi + (size_t)gj * J.ldc;
                const double v = DF ? (double)acc[a][b] + (double)cor[a][b] : f32_to_f64(acc[a][b]);
                *c = beta0 ? v : J.beta * *c + v;
                if (mirror) {
                    double* ct = J.C + gj + (size_t)gi * J.ldc;
                    *ct = beta0 ? v : J.beta * *ct + v;
                }
            }
        }
}

// C = beta C + sum_s W_s over the partial products of split-K jobs (slices
// of m x n, ld m, contiguous), summed in slice order.  One CTA per job and
// 64-column group.
__global__ void k_slice_sum(const SliceSum* __restrict__ jobs) {
    const SliceSum J = jobs[blockIdx.x];
    const int64_t mn = (int64_t)J.m * J.n;
    const int64_t c0 = (int64_t)blockIdx.y * 64 * J.m;
    const int64_t c1 = min(mn, c0 + (int64_t)64 * J.m);
    for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < J.slices; ++s) v += J.W[e + (size_t)s * mn];
        const int i = (int)(e % J.m), j = (int)(e / J.m);
        double* c = J.C + i + (size_t)j * J.ldc;
        *c = (J.beta == 0.0) ? v : J.beta * *c + v;
    }
}

void launch_slice_sum(const SliceSum* jobs, int njobs, int max_n, cudaStream_t st) {
    if (njobs <= 0 || max_n <= 0) return;
    k_slice_sum<<<dim3(njobs, (max_n + 63) / 64), 256, 0, st>>>(jobs);
}

void launch_gemm(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int precision,
                 cudaStream_t st) {
    if (ntiles <= 0) return;
    if (precision == H2_MIXED)
        k_gemm_f32<false><<<ntiles, GT, 0, st>>>(terms, jobs, tiles);
    else if (precision == kGemmDF)
        k_gemm_f32<true><<<ntiles, GT, 0, st>>>(terms, jobs, tiles);
    else
        k_gemm<double><<<ntiles, GT, 0, st>>>(terms, jobs, tiles);
}

// ------------------------------------------------------------------ GEMM on tcgen05
// Same contract as k_gemm on the 5th-generation tensor cores, for the FP32-class
// products of the tensor-core modes.  One CTA of 8 warps computes a 128 x 64
// output tile of one job:
//   - every warp stages its share of each K chunk of 32 (term, k) pairs: the
//     FP64 operands are read, rounded to FP32 (integer operations), split into
//     pieces and stored in shared memory in the K-major core-matrix layout
//     (8 rows x 16 bytes per core matrix, the cores of a row group contiguous
//     along K), two stages deep;
//   - thread 0 issues tcgen05.mma for each staged chunk and commits the stage
//     and the accumulator groups to mbarriers;
//   - every warp adds finished accumulator groups into registers and writes the
//     tile at the end: tcgen05.ld of TMEM lanes 32 (w mod 4) .. + 31 (those tile
//     rows) and columns 32 (w / 4) .. + 31.
// Pieces and products per mode:
//   TF32X3  x = a0 + a1 (two TF32 values, each rounded to nearest);
//           a0 b0 into D0, a0 b1 + a1 b0 into D1
//   TF32    a0 b0 into D0
//   BF16X3  x = a0 + a1 (two BF16 values); a0 b0 into D0, a0 b1 + a1 b0 into D1
// The tensor cores' FP32 accumulation rounds toward zero, so its error is a
// bias that grows with the number of accumulation steps.  In the three-term
// modes D0 (the leading product) therefore holds one chunk at a time: three D0
// buffers rotate, and while the MMAs fill one, the producers add the one two
// chunks back into FP32 registers with round to nearest.  D1 is 2^-11 (TF32) or 2^-8
// (BF16) smaller, so its bias is negligible and it accumulates over the whole
// job; so does D0 in the one-product mode, whose operand rounding (2^-11) is far
// above that bias.  Every wait is bounded (about a second): on timeout the CTA
// sets bit 4 of *err, stops, drains its MMAs and frees its TMEM.
constexpr int TC_M = 128, TC_N = 64, TC_K = 32, TC_T = 256;  // 8 warps, all producers
constexpr int TC_PRODUCERS = 256, TC_PW = TC_PRODUCERS / 32;
constexpr int TC_TCACHE = 64;  // term descriptors cached in shared memory

template <int MODE>
struct TcCfg {
    static constexpr bool bf16 = (MODE == H2_BF16X3);
    static constexpr bool three = (MODE != H2_TF32);
    static constexpr int esize = bf16 ? 2 : 4;         // bytes per element
    static constexpr int ke = 16 / esize;              // elements per 16-byte core row
    static constexpr int cores_k = TC_K / ke;          // core matrices along K per row group
    static constexpr int a_piece = TC_M * TC_K * esize;  // bytes of one piece of A
    static constexpr int b_piece = TC_N * TC_K * esize;
    static constexpr int pieces = three ? 2 : 1;
    static constexpr int stage = pieces * (a_piece + b_piece);
    static constexpr int flush = three ? 1 : (1 << 30);  // chunks per D0 group
    static constexpr int kstep = bf16 ? 16 : 8;          // K of one MMA
    static constexpr int cols = 256;                     // TMEM columns: D0 x 3 (+ D1)
    // shared memory: two stages, then the barriers and the stage flags; at least
    // 80 KB, so that at most two CTAs share an SM (their TMEM columns always fit)
    static constexpr int bar_off = 2 * stage;
    static constexpr int smem = (2 * stage + 256) > 80 * 1024 ? (2 * stage + 256) : 80 * 1024;
    // instruction descriptor: D FP32, A and B TF32 (kind::tf32) or BF16 (kind::f16),
    // both K-major, N = 64, M = 128
    static constexpr uint32_t idesc = (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) |
                                      ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
};

// shared memory descriptor, K-major without swizzle: LBO = 128 B (next core
// matrix along K), SBO = cores_k * 128 B (next 8-row group)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, int cores_k) {
    const uint64_t lbo = 128, sbo = (uint64_t)cores_k * 128;
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46);
}

template <int MODE>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (MODE == H2_BF16X3) {
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                     "l"(a), "l"(b), "r"(TcCfg<MODE>::idesc), "r"(acc));
    } else {
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                     "l"(a), "l"(b), "r"(TcCfg<MODE>::idesc), "r"(acc));
    }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t* u = (uint32_t*)v;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
          "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
          "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait for the phase of the given parity: false when the CTA was
// aborted, or about a second passed (then the CTA is aborted and *err flagged).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_try(bar, parity)) return true;
        if ((spin & 63u) == 0) {
            // another CTA of this or an earlier launch of the call timed out: give up too
            if (*abort_flag || (err && (*(volatile int*)err & 4))) {
                *abort_flag = 1;
                return false;
            }
            if (global_ns() - t0 > 1000000000ull) {
                *abort_flag = 1;
                if (err) atomicOr(err, 4);
                return false;
            }
        }
    }
}

__device__ __forceinline__ uint32_t tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t* w) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
}

// Staging of one operand tile of a K chunk (producer warps), in two steps so
// that the loads of both operands are in flight together: tc_load reads this
// thread's items from global memory, tc_store converts and stores them.  Item
// (row r, K group q) is the 16 bytes of row r in core matrix q of its row group
// (ke consecutive k); a warp stores 8 rows x 4 K groups, i.e. 4 consecutive
// 128-byte cores: conflict-free 16-byte stores.  Element (r, k) of the tile is
// base[r * ld + k] (kcontig) or base[r + k * ld]; rows >= rows_valid are not
// written (they were zeroed once), k >= kvalid is stored as zero.  The second
// piece (three-term modes) goes to dst + pstride.  Warp w takes the row groups
// w, w + 8, ... (NI items per thread).
template <int MODE, int NROWS>
struct TcOp {
    static constexpr int QW = TcCfg<MODE>::cores_k / 4;  // K groups of 4 cores per row group
    static constexpr int NI = (NROWS / 8) * QW / TC_PW;   // items per producer thread
    static constexpr int KE = TcCfg<MODE>::ke;
};

template <int MODE, int NROWS>
__device__ __forceinline__ void tc_load(double (&v)[TcOp<MODE, NROWS>::NI][TcOp<MODE, NROWS>::KE], const double* base,
                                        int ld, bool kcontig, int rows_valid, int kvalid, int warp, int lane) {
    using O = TcOp<MODE, NROWS>;
#pragma unroll
    for (int h = 0; h < O::NI; ++h) {
        const int g = warp + TC_PW * h;
        const int r = (g / O::QW) * 8 + (lane & 7), q = (g % O::QW) * 4 + (lane >> 3);
#pragma unroll
        for (int e = 0; e < O::KE; ++e) {
            const int k = q * O::KE + e;
            const bool in = r < rows_valid && k < kvalid;
            v[h][e] = in ? (kcontig ? base[(size_t)r * ld + k] : base[r + (size_t)k * ld]) : 0.0;
        }
    }
}

template <int MODE, int NROWS>
__device__ __forceinline__ void tc_store(const double (&v)[TcOp<MODE, NROWS>::NI][TcOp<MODE, NROWS>::KE], uint32_t dst,
                                         uint32_t pstride, int rows_valid, float scale, int warp, int lane) {
    using C = TcCfg<MODE>;
    using O = TcOp<MODE, NROWS>;
#pragma unroll
    for (int h = 0; h < O::NI; ++h) {
        const int g = warp + TC_PW * h;
        const int r8 = g / O::QW, q = (g % O::QW) * 4 + (lane >> 3);
        if (r8 * 8 >= rows_valid) continue;
        const uint32_t addr = dst + (uint32_t)((r8 * C::cores_k + q) * 128 + (lane & 7) * 16);
        uint32_t w0[4], w1[4];
        if constexpr (C::bf16) {
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                const float x0 = scale * f64_to_f32(v[h][e]), x1 = scale * f64_to_f32(v[h][e + 1]);
                const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                w0[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                w1[e / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = (scale == 1.f) ? f64_to_f32(v[h][e]) : scale * f64_to_f32(v[h][e]);
                w0[e] = tf32_rn(x);
                w1[e] = C::three ? tf32_rn(x - __uint_as_float(w0[e])) : 0u;
            }
        }
        st_shared_v4(addr, w0);
        if constexpr (C::three) st_shared_v4(addr + pstride, w1);
    }
}

// One CTA per output tile; its 8 warps stage the K chunks (all of them), and
// thread 0 also issues the MMAs: after arriving on a stage's barrier it waits
// for the other warps' arrivals (their shared-memory stores are then visible),
// issues the stage's MMAs and commits them to the stage's "empty" barrier and,
// at the end of a D0 group, to the group's "full" barrier.  Two CTAs share an
// SM (16 warps, 4 per SM sub-partition: at most 128 registers a thread), so one
// CTA's epilogue and prologue overlap the other's main loop.
template <int MODE>
__global__ void __maxnreg__(128) k_gemm_tc(const GTerm* __restrict__ terms, const GJob* __restrict__ jobs,
                                           const GTile* __restrict__ tiles, int* err) {
    using C = TcCfg<MODE>;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tc_smem);
    // barriers: full[2] 0..1, empty[2] 2..3, accf[3] 4..6, acce[3] 7..9, drain 10
    const uint32_t bar0 = sbase + C::bar_off;
    volatile int* abort_flag = (volatile int*)(tc_smem + C::bar_off + 96);
    uint32_t* tmem_slot = (uint32_t*)(tc_smem + C::bar_off + 112);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 16u + 8u * s; };
    auto accf = [&](int b) { return bar0 + 32u + 8u * b; };
    auto acce = [&](int b) { return bar0 + 56u + 8u * b; };
    const uint32_t drain = bar0 + 80u;
    // after a timeout anywhere in the call, later CTAs do nothing (one read, shared by the CTA)
    __shared__ int skip;
    __shared__ GTerm tcache[TC_TCACHE];
    __shared__ float tfact[TC_TCACHE];
    if (threadIdx.x == 0) skip = err ? (*(volatile int*)err & 4) : 0;
    __syncthreads();
    if (skip) return;
    const GTile tile = tiles[blockIdx.x];
    const GJob J = jobs[tile.job];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tmem_slot)),
                     "r"(C::cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(full(s), TC_PRODUCERS);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 3; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), TC_PRODUCERS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // the job's first term descriptors, with their factors in FP32 (0: skipped)
    for (int q = threadIdx.x; q < min(J.nt, TC_TCACHE); q += TC_T) {
        const GTerm t = terms[J.t0 + q];
        const double f = t.alpha * (t.scale ? *t.scale : 1.0);
        tcache[q] = t;
        tfact[q] = (f != 0.0 && t.k > 0) ? f64_to_f32(f) : 0.f;
    }
    // rows of A and B beyond the job stay zero in both stages
    const int mrows = min(TC_M, J.m - tile.i0), ncols = min(TC_N, J.n - tile.j0);
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < C::pieces; ++p) {
            uint4* a = (uint4*)(tc_smem + s * C::stage + p * C::a_piece);
            uint4* b = (uint4*)(tc_smem + s * C::stage + C::pieces * C::a_piece + p * C::b_piece);
            for (int e = threadIdx.x; e < C::a_piece / 16; e += TC_T)
                if ((e / (8 * C::cores_k)) * 8 + (e & 7) >= mrows) a[e] = make_uint4(0, 0, 0, 0);
            for (int e = threadIdx.x; e < C::b_piece / 16; e += TC_T)
                if ((e / (8 * C::cores_k)) * 8 + (e & 7) >= ncols) b[e] = make_uint4(0, 0, 0, 0);
        }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    // accumulators: warp w reads tile rows 32 (w mod 4) .. + 31 (its TMEM lanes)
    // and columns 32 (w / 4) .. + 31
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    const int quarter = warp & 3, chalf = warp >> 2;
    const uint32_t lane_base = ((uint32_t)(quarter * 32) << 16) + (uint32_t)(chalf * 32);
    // adds D0 group g into acc; its MMAs are complete once accf(g mod 3) fires
    auto read_group = [&](int g) -> bool {
        const int b = g % 3;
        // one decision per warp: tcgen05.ld needs the whole warp
        if (!__all_sync(0xffffffffu, mbar_wait(accf(b), (uint32_t)((g / 3) & 1), abort_flag, err))) return false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(b * TC_N), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += v[j];
        asm volatile("tcgen05.fence::before_thread_sync;");
        mbar_arrive(acce(b));
        return true;
    };
    // chunk sequence: (term it, k0) over the job's terms, skipping zero factors.
    // The first TC_TCACHE term descriptors and their FP32 factors were staged
    // in shared memory above (a branch on a descriptor fresh from global memory
    // would stall the warp for a full load latency); later terms of long jobs
    // are read from global memory.
    int it = -1, k0 = 0;
    GTerm P{};
    float fs = 0.f;
    auto term_at = [&](int i) {
        if (i < TC_TCACHE) {
            P = tcache[i];
            fs = tfact[i];
        } else {
            P = terms[J.t0 + i];
            const double f = P.alpha * (P.scale ? *P.scale : 1.0);
            fs = (f != 0.0 && P.k > 0) ? f64_to_f32(f) : 0.f;
        }
    };
    auto advance = [&]() -> bool {
        if (it >= 0 && k0 + TC_K < P.k) {
            k0 += TC_K;
            return true;
        }
        for (++it; it < J.nt; ++it) {
            term_at(it);
            if (fs != 0.f) {
                k0 = 0;
                return true;
            }
        }
        return false;
    };
    bool ok = true, d1_started = false;
    bool have = advance();
    int c = 0, in_group = 0, g = 0, g_read = 0;
    while (have) {
        const int s = c & 1;
        const GTerm Q = P;
        const int q0 = k0;
        const float qs = fs;
        const bool more = advance();
        const int kvalid = min(TC_K, Q.k - q0);
        // A (m x k) rows i0.., k q0..: plain A[i + k lda], transposed A[k + i lda]
        const double* ab = Q.ta ? Q.A + q0 + (size_t)tile.i0 * Q.lda : Q.A + tile.i0 + (size_t)q0 * Q.lda;
        // B (k x n) as rows j0.. of B^T: plain B[k + j ldb], transposed B[j + k ldb]
        const double* bb = Q.tb ? Q.B + tile.j0 + (size_t)q0 * Q.ldb : Q.B + q0 + (size_t)tile.j0 * Q.ldb;
        double va[TcOp<MODE, TC_M>::NI][TcOp<MODE, TC_M>::KE], vb[TcOp<MODE, TC_N>::NI][TcOp<MODE, TC_N>::KE];
        tc_load<MODE, TC_M>(va, ab, Q.lda, Q.ta != 0, mrows, kvalid, warp, lane);
        tc_load<MODE, TC_N>(vb, bb, Q.ldb, Q.tb == 0, ncols, kvalid, warp, lane);
        // the stage's previous chunk (c - 2) must be consumed before it is overwritten
        if (c >= 2 &&
            !__all_sync(0xffffffffu, mbar_wait(empty(s), (uint32_t)(((c >> 1) + 1) & 1), abort_flag, err))) {
            ok = false;
            break;
        }
        const uint32_t sa = sbase + s * C::stage, sb = sa + C::pieces * C::a_piece;
        tc_store<MODE, TC_M>(va, sa, C::a_piece, mrows, qs, warp, lane);
        tc_store<MODE, TC_N>(vb, sb, C::b_piece, ncols, 1.f, warp, lane);
        const bool opens = (in_group == 0);
        const bool closes = (in_group + 1 == C::flush) || !more;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full(s));
        if (threadIdx.x == 0) {
            // the MMAs of this chunk, once every warp has staged it; D0 group g uses
            // buffer g mod 3, whose last use (group g - 3) was read out before
            // the warps arrived on this stage
            const int b = g % 3;
            bool go = mbar_wait(full(s), (uint32_t)((c >> 1) & 1), abort_flag, err);
            if (go && opens && g >= 3) go = mbar_wait(acce(b), (uint32_t)((g / 3 - 1) & 1), abort_flag, err);
            if (go) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t d0 = tmem + (uint32_t)(b * TC_N), d1 = tmem + 3u * TC_N;
#pragma unroll
                for (int ks = 0; ks < TC_K / C::kstep; ++ks) {
                    const uint32_t off = ks * 256;  // two core matrices along K per MMA
                    const uint64_t a0 = tc_desc(sa + off, C::cores_k), b0 = tc_desc(sb + off, C::cores_k);
                    tc_mma<MODE>(d0, a0, b0, (opens && ks == 0) ? 0u : 1u);
                    if constexpr (C::three) {
                        const uint64_t a1 = tc_desc(sa + C::a_piece + off, C::cores_k);
                        const uint64_t b1 = tc_desc(sb + C::b_piece + off, C::cores_k);
                        tc_mma<MODE>(d1, a0, b1, d1_started ? 1u : 0u);
                        d1_started = true;
                        tc_mma<MODE>(d1, a1, b0, 1u);
                    }
                }
                tc_commit(empty(s));  // the stage may be refilled once these MMAs are done
                if (closes) tc_commit(accf(b));
            }
        }
        __syncwarp();
        // the group two before this one is long complete: add it up while the MMAs run
        if (opens && g >= 2 && g_read <= g - 2) {
            if (!read_group(g_read)) {
                ok = false;
                break;
            }
            ++g_read;
        }
        in_group = closes ? 0 : in_group + 1;
        if (closes) ++g;
        ++c;
        have = more;
    }
    while (ok && g_read < g) ok = read_group(g_read++);
    if (ok && c > 0 && C::three) {  // D1 (complete with the last group)
        asm volatile("tcgen05.fence::after_thread_sync;");
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(3 * TC_N), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += v[j];
    }
    if (ok && !*abort_flag) {
        const int row = tile.i0 + quarter * 32 + lane;
        if (row < J.m) {
            const bool beta0 = (__double_as_longlong(J.beta) << 1) == 0;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const int j = chalf * 32 + jj;
                if (j < ncols) {
                    double* cp = J.C + row + (size_t)(tile.j0 + j) * J.ldc;
                    const double val = f32_to_f64(acc[jj]);
                    *cp = beta0 ? val : J.beta * *cp + val;
                }
            }
        }
    }
    if (threadIdx.x == 0 && c > 0) {  // drain: every MMA issued has completed before TMEM is freed
        tc_commit(drain);
        const uint64_t t0 = global_ns();
        while (!mbar_try(drain, 0u) && global_ns() - t0 < 1000000000ull) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::cols));
}

template <int MODE>
static void launch_tc(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int* err, cudaStream_t st) {
    static bool attr_set[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            cudaFuncSetAttribute(k_gemm_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<MODE>::smem);
            // all of the unified L1/shared storage as shared memory: two CTAs per SM
            cudaFuncSetAttribute(k_gemm_tc<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            attr_set[dev] = true;
        }
    }
    k_gemm_tc<MODE><<<ntiles, TC_T, TcCfg<MODE>::smem, st>>>(terms, jobs, tiles, err);
}

void launch_gemm_tc(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int mode, int* err,
                    cudaStream_t st) {
    if (ntiles <= 0) return;
    if (mode == H2_TF32)
        launch_tc<H2_TF32>(terms, jobs, tiles, ntiles, err, st);
    else if (mode == H2_BF16X3)
        launch_tc<H2_BF16X3>(terms, jobs, tiles, ntiles, err, st);
    else
        launch_tc<H2_TF32X3>(terms, jobs, tiles, ntiles, err, st);
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NT>
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) red[0] = s;
    }
    __syncthreads();
    return red[0];
}

// ------------------------------------------------------------------ Householder QR
// Column-by-column Householder reflections H_j = I - tau_j v_j v_j^* with
// v_j(j) = 1 (Golub & Van Loan, Sec. 5.1-5.2), applied in place; the
// orthogonal factor is accumulated backwards when requested.
//
// With a pivot array the factorisation is A P = Q R with column pivoting
// (Businger & Golub 1965; Golub & Van Loan, Sec. 5.4.2): step j moves the
// column of largest remaining norm to position j.  The remaining norms are
// downdated by the new row of R after each step and recomputed from the
// column when the downdate has cancelled below the square root of the unit
// roundoff (the safeguard of Drmac & Bujanovic 2008).  The norms only steer
// the pivot choice, so they are kept and downdated in FP32 (recomputations
// accumulate in FP64).
constexpr int QT = 256;

template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// T = double: in place on A.  T = float: A (FP64) is converted into the FP32
// workspace A32 first and the factorisation runs there.
template <class T>
__global__ void __launch_bounds__(QT) k_qr(const QRJob* __restrict__ jobs) {
    __shared__ double red[QT / 32];
    __shared__ int redi[QT / 32];
    __shared__ float redf[QT / 32];
    // remaining / last recomputed column norms (pivoting); V^T v_j (WY form)
    __shared__ __align__(8) float vnbuf[2 * kQRPivMax];
    float* vn1 = vnbuf;
    float* vn2 = vnbuf + kQRPivMax;
    const QRJob J = jobs[blockIdx.x];
    const int m = J.m, n = J.n, p = m < n ? m : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = QT / 32;
    const bool pivot = J.piv != nullptr && n <= kQRPivMax;
    const float ptol = 3.4526698e-4f;  // sqrt(FP32 unit roundoff)
    T* A;
    int lda;
    if constexpr (sizeof(T) == 4) {
        A = (T*)J.A32;
        lda = m;
        for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += QT)
            A[e] = (T)J.A[(e % m) + (size_t)(e / m) * J.lda];
        __syncthreads();
    } else {
        A = (T*)J.A;
        lda = J.lda;
    }
    if (pivot) {
        for (int c = warp; c < n; c += nw) {
            const T* a = A + (size_t)c * lda;
            double s = 0.0;
            for (int i = lane; i < m; i += 32) s += (double)a[i] * (double)a[i];
            s = warp_sum(s);
            if (lane == 0) {
                vn1[c] = vn2[c] = (float)sqrt(s);
                J.piv[c] = c;
            }
        }
        __syncthreads();
    }
    for (int j = 0; j < p; ++j) {
        if (pivot) {
            // the column of largest remaining norm (lowest index on ties) moves to j
            float bv = -1.f;
            int bi = j;
            for (int c = j + threadIdx.x; c < n; c += QT)
                if (vn1[c] > bv) {
                    bv = vn1[c];
                    bi = c;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, bv, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                redf[warp] = bv;
                redi[warp] = bi;
            }
            __syncthreads();
            int pc = redi[0];
            float pv = redf[0];
            for (int w = 1; w < nw; ++w)
                if (redf[w] > pv || (redf[w] == pv && redi[w] < pc)) {
                    pv = redf[w];
                    pc = redi[w];
                }
            if (pc != j) {
                T* a = A + (size_t)j * lda;
                T* b = A + (size_t)pc * lda;
                for (int i = threadIdx.x; i < m; i += QT) {
                    T t = a[i];
                    a[i] = b[i];
                    b[i] = t;
                }
                if (threadIdx.x == 0) {
                    float t = vn1[j];
                    vn1[j] = vn1[pc];
                    vn1[pc] = t;
                    t = vn2[j];
                    vn2[j] = vn2[pc];
                    vn2[pc] = t;
                    int ti = J.piv[j];
                    J.piv[j] = J.piv[pc];
                    J.piv[pc] = ti;
                }
            }
            __syncthreads();
        }
        T* col = A + (size_t)j * lda;
        double s = 0.0;
        for (int i = j + 1 + threadIdx.x; i < m; i += QT) s += (double)col[i] * (double)col[i];
        s = block_sum<QT>(s, red);
        const double x0 = col[j];
        double tau = 0.0, beta = x0, sc = 0.0;
        if (s > 0.0) {
            beta = -copysign(sqrt(x0 * x0 + s), x0);
            tau = (beta - x0) / beta;
            sc = 1.0 / (x0 - beta);
        }
        __syncthreads();
        if (s > 0.0)
            for (int i = j + 1 + threadIdx.x; i < m; i += QT) col[i] = (T)(col[i] * sc);
        if (threadIdx.x == 0) {
            col[j] = (T)beta;
            J.tau[j] = tau;
        }
        __syncthreads();
        if (tau != 0.0 || pivot) {
            const T tt = (T)tau;
            for (int c = j + 1 + warp; c < n; c += nw) {
                T* a = A + (size_t)c * lda;
                if (tau != 0.0) {
                    T w = 0;
                    for (int i = j + 1 + lane; i < m; i += 32) w += col[i] * a[i];
                    w = warp_sum_t<T>(w);
                    __syncwarp();
                    w = (w + a[j]) * tt;
                    __syncwarp();
                    if (lane == 0) a[j] -= w;
                    for (int i = j + 1 + lane; i < m; i += 32) a[i] -= w * col[i];
                }
                if (pivot) {
                    // row j of R is final: remove it from the remaining norm
                    __syncwarp();
                    float v1 = vn1[c];
                    bool recompute = false;
                    if (v1 != 0.f) {
                        const float r = fabsf((float)a[j]) / v1;
                        const float rest = fmaxf(0.f, (1.f - r) * (1.f + r));
                        const float g = v1 / vn2[c];
                        if (rest * g * g <= ptol)
                            recompute = true;
                        else
                            v1 *= sqrtf(rest);
                    }
                    if (recompute) {
                        double s2 = 0.0;
                        for (int i = j + 1 + lane; i < m; i += 32) s2 += (double)a[i] * (double)a[i];
                        v1 = (float)sqrt(warp_sum(s2));
                    }
                    __syncwarp();
                    if (lane == 0) {
                        vn1[c] = v1;
                        if (recompute) vn2[c] = v1;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (J.R) {
        for (int e = threadIdx.x; e < p * n; e += QT) {
            int i = e % p, c = e / p;
            J.R[i + (size_t)c * J.ldr] = (i <= c) ? (double)A[i + (size_t)c * lda] : 0.0;
        }
    }
    if (sizeof(T) == 8 && J.V && p <= kQRPivMax) {
        // compact WY form (forward, column by column): T_jj = tau_j and
        // T(0:j, j) = -tau_j T(0:j, 0:j) y with y_l = v_l^T v_j (l < j); v_j is
        // zero above row j and one at row j
        for (int e = threadIdx.x; e < m * p; e += QT) {
            const int i = e % m, c = e / m;
            J.V[e] = (i < c) ? 0.0 : (i == c) ? 1.0 : (double)A[i + (size_t)c * lda];
        }
        double* y = reinterpret_cast<double*>(vnbuf);
        for (int j = 0; j < p; ++j) {
            const T* vj = A + (size_t)j * lda;
            for (int l = warp; l < j; l += nw) {
                const T* vl = A + (size_t)l * lda;
                double s = 0.0;
                for (int r = j + 1 + lane; r < m; r += 32) s += (double)vl[r] * (double)vj[r];
                s = warp_sum(s);
                if (lane == 0) y[l] = s + (double)vl[j];
            }
            __syncthreads();
            const double tau = J.tau[j];
            for (int i = threadIdx.x; i < p; i += QT) {
                double v = 0.0;
                if (i < j) {
                    double s = 0.0;
                    for (int l = i; l < j; ++l) s += J.T[i + (size_t)l * p] * y[l];
                    v = -tau * s;
                } else if (i == j) {
                    v = tau;
                }
                J.T[i + (size_t)j * p] = v;
            }
            __syncthreads();
        }
    }
    if (sizeof(T) == 8 && J.Q) {
        for (int e = threadIdx.x; e < m * J.q; e += QT) {
            int i = e % m, c = e / m;
            J.Q[i + (size_t)c * J.ldq] = (i == c) ? 1.0 : 0.0;
        }
        __syncthreads();
        for (int j = p - 1; j >= 0; --j) {
            const double tau = J.tau[j];
            if (tau == 0.0) continue;
            const T* v = A + (size_t)j * lda;
            for (int c = warp; c < J.q; c += nw) {
                double* a = J.Q + (size_t)c * J.ldq;
                double w = 0.0;
                for (int i = j + 1 + lane; i < m; i += 32) w += (double)v[i] * a[i];
                w = warp_sum(w);
                __syncwarp();
                w = (w + a[j]) * tau;
                __syncwarp();
                if (lane == 0) a[j] -= w;
                for (int i = j + 1 + lane; i < m; i += 32) a[i] -= w * (double)v[i];
            }
            __syncthreads();
        }
    }
}

void launch_qr(const QRJob* jobs, int njobs, cudaStream_t st) {
    if (njobs > 0) k_qr<double><<<njobs, QT, 0, st>>>(jobs);
}

void launch_qr32(const QRJob* jobs, int njobs, cudaStream_t st) {
    if (njobs > 0) k_qr<float><<<njobs, QT, 0, st>>>(jobs);
}

// ------------------------------------------------------------------ one-sided Jacobi SVD
// Hestenes' method: plane rotations from the right make the columns of B
// mutually orthogonal, B J = U Sigma; pairs follow a round-robin tournament so
// that the pairs of one round are disjoint and run in parallel warps.  The
// sweep count is bounded; *flag reports a run that hit the bound.  A sweep
// whose rotation measures |g| / sqrt(a b) all stay below 0.1 sqrt(tol) leaves
// an off-diagonality below tol (quadratic convergence), so the verifying
// sweep is skipped.
constexpr int JT = 512;
constexpr int JMAXSWEEP = 40;
constexpr int JMAXN = 2048;

__device__ __forceinline__ int rr_player(int pos, int round, int np) {
    if (pos == 0) return 0;
    return 1 + (pos - 1 + round) % (np - 1);
}

// FP32 preconditioning sweeps: Hestenes rotations on an FP32 copy W of B,
// accumulated into V (V starts as the identity).  Bounded sweeps.
constexpr int PMAXSWEEP = 30;

// W lives in dynamic shared memory when its m * n floats fit in the launch's
// smem_bytes (sized for the largest job, at most kPreSmem), else in its
// global workspace; V joins it there when (m + n) n floats fit.
// (Carrying the squared column norms under the rotations, as the FP64 sweeps
// do, was measured slower here: in FP32 the carried norms of columns that
// shrink lose their accuracy within a sweep, and the convergence test then
// asks for more sweeps.  Each pair forms its three inner products.)
constexpr int kPreSmem = 200 * 1024;

__global__ void __launch_bounds__(JT) k_jacobi_pre(const PreJob* __restrict__ jobs, int smem_bytes) {
    extern __shared__ float pre_smem[];
    __shared__ int rotated;
    const PreJob J = jobs[blockIdx.x];
    const int m = J.m, n = J.ncols ? min(J.n, max(*J.ncols, 0)) : J.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    const bool in_smem = (size_t)m * n * sizeof(float) <= (size_t)smem_bytes;
    const bool v_smem = in_smem && J.V && (size_t)(m + n) * n * sizeof(float) <= (size_t)smem_bytes;
    float* W = in_smem ? pre_smem : J.W;
    float* V = v_smem ? pre_smem + (size_t)m * n : J.V;
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += JT) W[e] = (float)J.B[(e % m) + (size_t)(e / m) * J.ldb];
    if (V)
        for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += JT) V[e] = ((e % n) == (e / n)) ? 1.f : 0.f;
    __syncthreads();
    const int np = n + (n & 1);
    const float tol = (float)(m > 1 ? m : 1) * FLT_EPSILON;
    const float skip = 0.1f * sqrtf(tol);
    __shared__ int large;
    bool converged = (n < 2);
    int sweep = 0;
    for (; sweep < PMAXSWEEP && !converged; ++sweep) {
        if (threadIdx.x == 0) {
            rotated = 0;
            large = 0;
        }
        __syncthreads();
        for (int round = 0; round < np - 1; ++round) {
            for (int pr = warp; pr < np / 2; pr += nw) {
                int p = rr_player(pr, round, np), q = rr_player(np - 1 - pr, round, np);
                if (p >= n || q >= n) continue;
                if (p > q) { int t = p; p = q; q = t; }
                float* ap = W + (size_t)p * m;
                float* aq = W + (size_t)q * m;
                float al = 0.f, be = 0.f, ga = 0.f;
                for (int i = lane; i < m; i += 32) {
                    float x = ap[i], y = aq[i];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum_t<float>(al);
                be = warp_sum_t<float>(be);
                ga = warp_sum_t<float>(ga);
                if (ga != 0.f && al > 0.f && be > 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
                    float zeta = (be - al) / (2.f * ga);
                    float t = (fabsf(zeta) > 1e18f) ? 0.5f / zeta
                                                    : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    float c = 1.f / sqrtf(1.f + t * t), s = c * t;
                    for (int i = lane; i < m; i += 32) {
                        float x = ap[i], y = aq[i];
                        ap[i] = c * x - s * y;
                        aq[i] = s * x + c * y;
                    }
                    if (V) {
                        float* vp = V + (size_t)p * n;
                        float* vq = V + (size_t)q * n;
                        for (int i = lane; i < n; i += 32) {
                            float x = vp[i], y = vq[i];
                            vp[i] = c * x - s * y;
                            vq[i] = s * x + c * y;
                        }
                    }
                    if (lane == 0) {
                        rotated = 1;
                        if (fabsf(ga) > skip * sqrtf(al) * sqrtf(be)) large = 1;
                    }
                }
            }
            __syncthreads();
        }
        converged = (rotated == 0) || (large == 0);
        __syncthreads();
    }
    if (J.V64)
        for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += JT) J.V64[e] = (double)V[e];
    if (J.W64)
        for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += JT) J.W64[e] = (double)W[e];
    if (threadIdx.x == 0 && J.flops)
        atomicAdd(J.flops, 12.0 * (m + (J.V ? n : 0)) * (0.5 * n * (n - 1.0)) * sweep);
}

// ------------------------------------------------------------------ clustered FP32 preconditioning
// The FP32 preconditioning sweeps with one matrix shared by a thread-block
// cluster: the disjoint pairs of a round are spread over the cluster's CTAs
// (one CTA per SM), a cluster barrier separates rounds, columns move through
// L2 (ld/st.cg), and the rotation flags of a sweep are OR-ed across the
// cluster through distributed shared memory.  Used when a level has fewer
// matrices than SMs.
namespace cg = cooperative_groups;

__device__ __forceinline__ void rot_pair32(float* ap, float* aq, int m, float c, float s, int lane) {
    for (int i = lane; i < m; i += 32) {
        float x = __ldcg(ap + i), y = __ldcg(aq + i);
        __stcg(ap + i, c * x - s * y);
        __stcg(aq + i, s * x + c * y);
    }
}

__global__ void __launch_bounds__(JT) k_jacobi_pre_cluster(const PreJob* __restrict__ jobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    const PreJob& J = jobs[blockIdx.x / cs];
    __shared__ int rotated, large;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    const int m = J.m, n = J.ncols ? min(J.n, max(*J.ncols, 0)) : J.n;
    float* B = J.W;  // m x n, ld m
    float* V = J.V;  // n x n, ld n
    for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)m * n; e += (int64_t)JT * cs)
        __stcg(B + e, (float)J.B[(e % m) + (size_t)(e / m) * J.ldb]);
    if (V)
        for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)n * n; e += (int64_t)JT * cs)
            __stcg(V + e, ((e % n) == (e / n)) ? 1.f : 0.f);
    cl.sync();
    const int np = n + (n & 1);
    const float tol = (float)(m > 1 ? m : 1) * FLT_EPSILON;
    const float skip = 0.1f * sqrtf(tol);
    bool converged = (n < 2);
    int sweep = 0;
    for (; sweep < PMAXSWEEP && !converged; ++sweep) {
        if (threadIdx.x == 0) {
            rotated = 0;
            large = 0;
        }
        cl.sync();
        for (int round = 0; round < np - 1; ++round) {
            for (int pr = cr * nw + warp; pr < np / 2; pr += nw * cs) {
                int p = rr_player(pr, round, np), q = rr_player(np - 1 - pr, round, np);
                if (p >= n || q >= n) continue;
                if (p > q) { int t = p; p = q; q = t; }
                float* ap = B + (size_t)p * m;
                float* aq = B + (size_t)q * m;
                float al = 0.f, be = 0.f, ga = 0.f;
                for (int i = lane; i < m; i += 32) {
                    float x = __ldcg(ap + i), y = __ldcg(aq + i);
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum_t<float>(al);
                be = warp_sum_t<float>(be);
                ga = warp_sum_t<float>(ga);
                if (ga != 0.f && al > 0.f && be > 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
                    float zeta = (be - al) / (2.f * ga);
                    float t = (fabsf(zeta) > 1e18f) ? 0.5f / zeta
                                                    : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    float c = 1.f / sqrtf(1.f + t * t), s = c * t;
                    rot_pair32(ap, aq, m, c, s, lane);
                    if (V) rot_pair32(V + (size_t)p * n, V + (size_t)q * n, n, c, s, lane);
                    if (lane == 0) {
                        rotated = 1;
                        if (fabsf(ga) > skip * sqrtf(al) * sqrtf(be)) large = 1;
                    }
                }
            }
            cl.sync();
        }
        int any = 0, anylarge = 0;
        for (int r = 0; r < cs; ++r) {
            any |= *cl.map_shared_rank(&rotated, r);
            anylarge |= *cl.map_shared_rank(&large, r);
        }
        converged = (any == 0) || (anylarge == 0);
        cl.sync();
    }
    if (J.V64)
        for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)n * n; e += (int64_t)JT * cs)
            J.V64[e] = (double)__ldcg(V + e);
    if (J.W64)
        for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)m * n; e += (int64_t)JT * cs)
            J.W64[e] = (double)__ldcg(B + e);
    if (cr == 0 && threadIdx.x == 0 && J.flops)
        atomicAdd(J.flops, 12.0 * (m + (V ? n : 0)) * (0.5 * n * (n - 1.0)) * sweep);
}

// ------------------------------------------------------------------ FP64 Jacobi
// Hestenes sweeps in FP64, arranged so that few FP64 warp instructions are
// spent per column pair (the FP64 pipe bounds this kernel):
//  * the squared column norms are carried along under the rotations
//    (a' = a - t g, b' = b + t g for the pair's inner product g) and
//    recomputed from the columns at every rescaling point, so a pair costs one
//    inner product instead of three;
//  * rotations are applied in scaled form, like Gentleman's square-root-free
//    Givens transformations (1973): column c is held as x_c with true column
//    d_c x_c, so a rotation costs two FMAs per element (x_p - t1 x_q and
//    x_q + t2 x_p) and multiplies d_p and d_q by cos(theta); the scales are
//    folded back into the columns every kFoldRounds rounds and at the end;
//  * each round first forms the inner products of its pairs (one warp per
//    pair), then the rotation parameters with one thread per pair, so that the
//    scalar FP64 work is shared by 32 pairs per instruction, then applies the
//    rotations (one warp per pair).
// t = tan(theta) comes from FP32 arithmetic on exactly rescaled FP64 inputs:
// an angle error of relative size 1e-7 leaves an off-diagonal remainder 1e-7
// times the one removed, which later sweeps take out (in the final sweeps t is
// itself tiny).  cos(theta) = (1 + t^2)^(-1/2) is refined to FP64 by Newton's
// iteration for the reciprocal square root, so that every rotation applied is
// orthogonal to FP64 rounding.
//
// CLUSTER: one matrix per thread-block cluster, the pairs of a round spread
// over its CTAs (one CTA per SM), the column state (norms, scales) in the
// shared memory of CTA 0 reached through distributed shared memory, columns
// through L2 (ld/st.cg) and a cluster barrier between rounds.  Otherwise one
// CTA per matrix.
constexpr int kFoldRounds = 64;

template <bool CG>
__device__ __forceinline__ double ldcol(const double* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}
template <bool CG>
__device__ __forceinline__ void stcol(double* p, double v) {
    if constexpr (CG) __stcg(p, v);
    else *p = v;
}
template <bool CLUSTER>
__device__ __forceinline__ void sync_all() {
    if constexpr (CLUSTER) cg::this_cluster().sync();
    else __syncthreads();
}

// w^(-1/2) for w in [1, 2]: FP32 seed (relative error about 2^-22), then two
// Newton steps y <- y + y (1 - w y^2) / 2, each squaring the relative error.
__device__ __forceinline__ double rsqrt_newton(double w) {
    double y = (double)rsqrtf((float)w);
    double h = fma(-w * y, y, 1.0);
    y = fma(0.5 * y, h, y);
    h = fma(-w * y, y, 1.0);
    return fma(0.5 * y, h, y);
}

// t = sign(z) / (|z| + sqrt(1 + z^2)) with z = (b - a) / (2 g): the root of
// t^2 + 2 z t - 1 = 0 of modulus <= 1, the tangent of the rotation that makes
// the pair orthogonal.  Both z operands are scaled by the same power of two
// (exact) so that FP32 can take their quotient.
__device__ __forceinline__ double jacobi_tan(double a, double b, double g) {
    const double diff = b - a, g2 = g + g;
    int e = ((__double2hiint(g2) >> 20) & 0x7ff) - 1023;
    e = max(-1022, min(1022, e));
    const double sc = __hiloint2double((1023 - e) << 20, 0);  // 2^-e
    const double ds = diff * sc;
    if (fabs(ds) < 1e30) {
        const float zf = (float)ds / (float)(g2 * sc);
        const float af = fabsf(zf);
        const float tf = af > 1e18f ? 0.5f / zf : copysignf(1.f, zf) / (af + sqrtf(fmaf(zf, zf, 1.f)));
        return (double)tf;
    }
    return g / diff;  // |z| > 1e29: t = 1 / (2 z) to relative 1e-58
}

// Scales folded into the columns (x_c <- d_c x_c, d_c = 1) and squared norms
// recomputed; first: the scales are not set yet (all one).
template <bool CLUSTER>
__device__ void j64_fold(double* B, int ldb, int m, int n, double* nrm, double* dsc, double* dinv, bool first,
                         int cs, int cr) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    for (int c = cr * nw + warp; c < n; c += nw * cs) {
        double* x = B + (size_t)c * ldb;
        const double d = first ? 1.0 : dsc[c];
        double s = 0.0;
        if (d == 1.0) {
            for (int i = lane; i < m; i += 32) {
                const double v = ldcol<CLUSTER>(x + i);
                s = fma(v, v, s);
            }
        } else {
            for (int i = lane; i < m; i += 32) {
                const double v = ldcol<CLUSTER>(x + i) * d;
                stcol<CLUSTER>(x + i, v);
                s = fma(v, v, s);
            }
        }
        s = warp_sum(s);
        if (lane == 0) {
            nrm[c] = s;
            dsc[c] = 1.0;
            dinv[c] = 1.0;
        }
    }
}

// dynamic shared memory of k_jacobi64: column state (3 n) + per-CTA pair slots (2 kmax)
static size_t j64_smem_bytes(int n, int cs) {
    const int np = n + (n & 1), kmax = (np / 2 + cs - 1) / cs;
    return sizeof(double) * (3 * (size_t)n + 2 * (size_t)kmax);
}

template <bool CLUSTER>
__global__ void __launch_bounds__(JT) k_jacobi64(const SVDJob* __restrict__ jobs) {
    extern __shared__ double j64[];
    __shared__ int rotated, large, nrot;
    int cs = 1, cr = 0;
    if constexpr (CLUSTER) {
        cs = (int)cg::this_cluster().num_blocks();
        cr = (int)cg::this_cluster().block_rank();
    }
    const SVDJob& J = jobs[blockIdx.x / cs];
    const int m = J.m, n = J.ncols ? min(J.n, max(*J.ncols, 0)) : J.n, ldb = J.ldb, np = n + (n & 1),
              half = np / 2;
    const int kmax = (half + cs - 1) / cs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    double* B = J.B;
    double* st = j64;
    if constexpr (CLUSTER) st = cg::this_cluster().map_shared_rank(j64, 0);
    double* nrm = st;           // squared column norms
    double* dsc = st + n;       // column scales d_c
    double* dinv = st + 2 * n;  // 1 / d_c
    double* gk = j64 + 3 * n;   // per pair of this CTA: inner product, then t1
    double* t2k = gk + kmax;    // per pair: t2
    const double tol = (double)(m > 1 ? m : 1) * DBL_EPSILON;
    const double tol2 = tol * tol, skip2 = 0.01 * tol;  // skip2 = (0.1 sqrt(tol))^2
    if (threadIdx.x == 0) nrot = 0;
    int myrot = 0;
    j64_fold<CLUSTER>(B, ldb, m, n, nrm, dsc, dinv, true, cs, cr);
    sync_all<CLUSTER>();
    bool converged = (n < 2);
    int sweep = 0;
    for (; sweep < JMAXSWEEP && !converged; ++sweep) {
        if (threadIdx.x == 0) {
            rotated = 0;
            large = 0;
        }
        for (int round = 0; round < np - 1; ++round) {
            if (round % kFoldRounds == 0 && (sweep > 0 || round > 0)) {
                j64_fold<CLUSTER>(B, ldb, m, n, nrm, dsc, dinv, false, cs, cr);
                sync_all<CLUSTER>();
            }
            // inner products of the stored columns, one warp per pair
            for (int k = warp; k < kmax; k += nw) {
                const int pr = cr + k * cs;
                if (pr >= half) break;
                const int p = rr_player(pr, round, np), q = rr_player(np - 1 - pr, round, np);
                double g = 0.0;
                if (p < n && q < n) {
                    const double* x = B + (size_t)p * ldb;
                    const double* y = B + (size_t)q * ldb;
                    for (int i = lane; i < m; i += 32) g = fma(ldcol<CLUSTER>(x + i), ldcol<CLUSTER>(y + i), g);
                    g = warp_sum(g);
                }
                if (lane == 0) gk[k] = g;
            }
            __syncthreads();
            // rotation parameters, one thread per pair
            for (int k = threadIdx.x; k < kmax; k += JT) {
                const int pr = cr + k * cs;
                double t1 = 0.0, t2 = 0.0;
                int p = 0, q = 0;
                if (pr < half) {
                    p = rr_player(pr, round, np);
                    q = rr_player(np - 1 - pr, round, np);
                }
                if (pr < half && p < n && q < n) {
                    if (p > q) {
                        const int t = p;
                        p = q;
                        q = t;
                    }
                    const double dp = dsc[p], dq = dsc[q];
                    const double ga = gk[k] * dp * dq, al = nrm[p], be = nrm[q];
                    if (ga != 0.0 && al > 0.0 && be > 0.0 && ga * ga > tol2 * (al * be)) {
                        const double t = jacobi_tan(al, be, ga);
                        const double w = fma(t, t, 1.0);
                        const double c = rsqrt_newton(w), ci = w * c;  // cos and 1 / cos
                        t1 = t * dq * dinv[p];
                        t2 = t * dp * dinv[q];
                        dsc[p] = c * dp;
                        dsc[q] = c * dq;
                        dinv[p] *= ci;
                        dinv[q] *= ci;
                        nrm[p] = fma(-t, ga, al);
                        nrm[q] = fma(t, ga, be);
                        rotated = 1;
                        if (ga * ga > skip2 * (al * be)) large = 1;
                        ++myrot;
                    }
                }
                gk[k] = t1;
                t2k[k] = t2;
            }
            __syncthreads();
            // scaled rotations, one warp per pair (the pair's smaller index first)
            for (int k = warp; k < kmax; k += nw) {
                const double t1 = gk[k], t2 = t2k[k];
                if (t1 == 0.0 && t2 == 0.0) continue;
                const int pr = cr + k * cs;
                int p = rr_player(pr, round, np), q = rr_player(np - 1 - pr, round, np);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                double* x = B + (size_t)p * ldb;
                double* y = B + (size_t)q * ldb;
                for (int i = lane; i < m; i += 32) {
                    const double u = ldcol<CLUSTER>(x + i), v = ldcol<CLUSTER>(y + i);
                    stcol<CLUSTER>(x + i, fma(-t1, v, u));
                    stcol<CLUSTER>(y + i, fma(t2, u, v));
                }
            }
            sync_all<CLUSTER>();
        }
        int any = rotated, anylarge = large;
        if constexpr (CLUSTER) {
            for (int r = 0; r < cs; ++r) {
                any |= *cg::this_cluster().map_shared_rank(&rotated, r);
                anylarge |= *cg::this_cluster().map_shared_rank(&large, r);
            }
        }
        converged = (any == 0) || (anylarge == 0);
        sync_all<CLUSTER>();
    }
    j64_fold<CLUSTER>(B, ldb, m, n, nrm, dsc, dinv, false, cs, cr);
    if (myrot) atomicAdd(&nrot, myrot);
    sync_all<CLUSTER>();
    // executed FP64 flops: 2 m per inner product, 4 m per rotation
    if (threadIdx.x == 0 && J.flops)
        atomicAdd(J.flops, 4.0 * m * nrot + (cr == 0 ? 2.0 * m * (0.5 * n * (n - 1.0)) * sweep : 0.0));
    if (cr != 0) return;
    if (threadIdx.x == 0 && !converged && J.flag) atomicOr(J.flag, 1);
    for (int c = threadIdx.x; c < n; c += JT) nrm[c] = sqrt(nrm[c]);  // now the singular values
    __syncthreads();
    for (int c = warp; c < n; c += nw) {
        const double sc = nrm[c];
        int pos = 0;
        for (int q = lane; q < n; q += 32) pos += (nrm[q] > sc) || (nrm[q] == sc && q < c);
        pos = __reduce_add_sync(0xffffffffu, pos);
        const double* a = B + (size_t)c * ldb;
        double* u = J.U + (size_t)pos * J.ldu;
        const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
        if (J.rowperm)
            for (int i = lane; i < m; i += 32) u[J.rowperm[i]] = ldcol<CLUSTER>(a + i) * inv;
        else
            for (int i = lane; i < m; i += 32) u[i] = ldcol<CLUSTER>(a + i) * inv;
        if (lane == 0) J.sigma[pos] = sc;
    }
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int q = 0; q < n; ++q) cnt += (nrm[q] > J.eps);
        *J.count = cnt;
    }
}

int device_sm_count();
static int num_sms() { return device_sm_count(); }
int device_sm_count() {
    static int sms[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    if (!sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = v > 0 ? v : 1;
    }
    return sms[dev];
}

// cluster size for njobs matrices: the largest power of two <= 8 that keeps
// njobs * size within the SM count (1 = plain kernel)
static int jacobi_cluster_size(int njobs) {
    int sms = num_sms(), cs = 1;
    while (cs < 8 && njobs * cs * 2 <= sms) cs *= 2;
    return cs;
}

// one CTA per SM: request enough dynamic shared memory that two do not fit
constexpr size_t kClusterDynSmem = 120 * 1024;

// cluster launch of nblocks CTAs in clusters of cs; returns false (and clears
// the error) when the launch is refused
template <typename... Args>
static bool launch_clustered(void (*kern)(Args...), int nblocks, int cs, size_t smem, cudaStream_t st, Args... args) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks, 1, 1);
    cfg.blockDim = dim3(JT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

void launch_svd(const SVDJob* jobs, int njobs, int max_n, cudaStream_t st, bool clusters) {
    if (max_n > JMAXN) throw Error(H2_ERR_UNSUPPORTED, "SVD wider than 2048 columns");
    if (njobs <= 0) return;
    const int cs = clusters ? jacobi_cluster_size(njobs) : 1;
    if (cs > 1 && launch_clustered(k_jacobi64<true>, njobs * cs, cs,
                                   std::max(j64_smem_bytes(max_n, cs), kClusterDynSmem), st, jobs))
        return;
    // The attribute is a per-function limit shared by every host thread: it is set
    // once per device to the largest size any launch asks for.  (Set per launch to
    // that launch's size, a concurrent product's smaller setting could land between
    // another thread's setting and its launch, and that launch would be refused.)
    static bool attr_set[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            cudaFuncSetAttribute(k_jacobi64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)j64_smem_bytes(JMAXN, 1));
            attr_set[dev] = true;
        }
    }
    const size_t smem = j64_smem_bytes(max_n, 1);
    k_jacobi64<false><<<njobs, JT, smem, st>>>(jobs);
}

void launch_jacobi_pre(const PreJob* jobs, int njobs, size_t max_mn, size_t max_mnv, cudaStream_t st,
                       bool clusters) {
    if (njobs <= 0) return;
    int cs = clusters ? jacobi_cluster_size(njobs) : 1;
    if (cs <= 1 || !launch_clustered(k_jacobi_pre_cluster, njobs * cs, cs, kClusterDynSmem, st, jobs)) {
        static bool attr_set[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            cudaFuncSetAttribute(k_jacobi_pre, cudaFuncAttributeMaxDynamicSharedMemorySize, kPreSmem);
            attr_set[dev] = true;
        }
        // W (and V) of the largest job in shared memory when they fit
        const size_t want = (max_mnv * sizeof(float) <= (size_t)kPreSmem) ? max_mnv : max_mn;
        const int smem = (want * sizeof(float) <= (size_t)kPreSmem) ? (int)(want * sizeof(float)) : 0;
        k_jacobi_pre<<<njobs, JT, smem, st>>>(jobs, smem);
    }
}

// ------------------------------------------------------------------ pivoted Cholesky
// Symmetric pivoting on the largest remaining diagonal entry (Higham,
// "Accuracy and Stability of Numerical Algorithms", Sec. 10.3), stopped when
// the pivot falls below rel_tol times the largest initial diagonal entry, or
// when the trace of the remaining Schur complement (the sum of the remaining
// diagonal entries) is at most abs_tol.  Only the lower triangle of the
// working copy is read and updated.  It lives in shared memory, packed by
// columns, when k (k + 1) / 2 doubles fit (SMEM): each column step then waits on
// shared-memory latency instead of L2 latency.  Otherwise it is the job's
// k x k workspace in global memory.
constexpr int CT = 256;
constexpr int CMAXK = 1024;
constexpr int kCholSmem = 96 * 1024;

template <bool SMEM>
__global__ void __launch_bounds__(CT) k_pchol(const CholJob* __restrict__ jobs) {
    extern __shared__ double cw[];
    __shared__ int perm[CMAXK];
    __shared__ double rv[CT / 32], rt[CT / 32];
    __shared__ int ri[CT / 32];
    __shared__ int piv;
    __shared__ double pval, ptrace;
    const CholJob J = jobs[blockIdx.x];
    const int k = J.k;
    double* const W = SMEM ? cw : J.W;
    // entry (i, j), i >= j, of the lower triangle
    auto at = [&](int i, int j) -> double& {
        if constexpr (SMEM)
            return W[(size_t)j * k - ((size_t)j * (j - 1)) / 2 + (i - j)];
        else
            return W[i + (size_t)j * k];
    };
    for (int e = threadIdx.x; e < k * k; e += CT) {
        const int i = e % k, j = e / k;
        if (i >= j) at(i, j) = J.G[i + (size_t)j * J.ldg];
    }
    for (int i = threadIdx.x; i < k; i += CT) perm[i] = i;
    for (int e = threadIdx.x; e < J.zrows * k; e += CT) J.Z[e] = 0.0;
    __syncthreads();
    // largest initial diagonal entry
    double md = 0.0;
    for (int i = threadIdx.x; i < k; i += CT) md = fmax(md, at(i, i));
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    if ((threadIdx.x & 31) == 0) rv[threadIdx.x >> 5] = md;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < CT / 32; ++w) m = fmax(m, rv[w]);
        pval = m;
    }
    __syncthreads();
    const double tol = J.rel_tol * pval;
    const int jmax = J.zrows < k ? J.zrows : k;
    int rank = jmax;
    for (int j = 0; j < jmax; ++j) {
        // pivot: argmax of the remaining diagonal (lowest index on ties), and its trace
        double best = -1.0, tr = 0.0;
        int bi = j;
        for (int i = j + threadIdx.x; i < k; i += CT) {
            double d = at(i, i);
            if (d > best) { best = d; bi = i; }
            tr += fmax(d, 0.0);
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            tr += __shfl_xor_sync(0xffffffffu, tr, o);
        }
        if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = best; ri[threadIdx.x >> 5] = bi; rt[threadIdx.x >> 5] = tr; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = rv[0], t = rt[0];
            int i0 = ri[0];
            for (int w = 1; w < CT / 32; ++w) {
                if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
                t += rt[w];
            }
            piv = i0;
            pval = b;
            ptrace = t;
        }
        __syncthreads();
        if (!(pval > tol) || !(pval > 0.0) || ptrace <= J.abs_tol) {
            rank = j;
            break;
        }
        const int p = piv;
        if (p != j) {  // symmetric swap of j and p (j < p) on the lower triangle
            auto sw = [&](double& x, double& y) {
                double t = x;
                x = y;
                y = t;
            };
            for (int c = threadIdx.x; c < k; c += CT) {
                if (c < j)
                    sw(at(j, c), at(p, c));  // rows j and p left of column j
                else if (c > j && c < p)
                    sw(at(c, j), at(p, c));  // column j between j and p <-> row p
                else if (c > p)
                    sw(at(c, j), at(c, p));  // columns j and p below row p
                else if (c == j)
                    sw(at(j, j), at(p, p));  // the diagonal entries
            }
            if (threadIdx.x == 0) {
                int t = perm[j];
                perm[j] = perm[p];
                perm[p] = t;
            }
            __syncthreads();
        }
        const double d = sqrt(at(j, j));
        const double inv = 1.0 / d;
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < k; i += CT) at(i, j) *= inv;
        if (threadIdx.x == 0) at(j, j) = d;
        __syncthreads();
        // trailing update of the lower triangle (one warp per column)
        {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int l = j + 1 + warp; l < k; l += CT / 32) {
                const double wl = at(l, j);
                if (wl == 0.0) continue;
                for (int i = l + lane; i < k; i += 32) at(i, l) -= at(i, j) * wl;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && J.rank) *J.rank = rank;
    // Z = L^* P^*: Z[j, perm[i]] = L[i, j] for i >= j, j < rank
    for (int64_t e = threadIdx.x; e < (int64_t)k * rank; e += CT) {
        int i = (int)(e % k), j = (int)(e / k);
        if (i >= j) J.Z[j + (size_t)perm[i] * J.zrows] = at(i, j);
    }
}

void launch_pchol(const CholJob* jobs, int njobs, int max_k, cudaStream_t st) {
    if (njobs <= 0) return;
    const size_t tri = (size_t)max_k * (max_k + 1) / 2 * sizeof(double);
    if (tri <= (size_t)kCholSmem) {
        static bool attr_set[64] = {};
        static std::mutex mu;
        int dev = 0;
        cudaGetDevice(&dev);
        {
            std::lock_guard<std::mutex> lk(mu);
            if (dev >= 0 && dev < 64 && !attr_set[dev]) {
                cudaFuncSetAttribute(k_pchol<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmem);
                attr_set[dev] = true;
            }
        }
        k_pchol<true><<<njobs, CT, tri, st>>>(jobs);
    } else {
        k_pchol<false><<<njobs, CT, 0, st>>>(jobs);
    }
}

// ------------------------------------------------------------------ spectral norm
// Power iteration x <- A^* A x with normalisation; returns ||A x|| for the
// final unit vector (a lower bound that converges to ||A||_2).  Stops when
// the estimate changes by less than rtol (relative) or after NITER steps.
// T = float in the mixed mode: the norm only scales a block.
constexpr int NT = 128;
constexpr int NMAX = 2048;
constexpr int NITER = 60;

template <class T>
__global__ void __launch_bounds__(NT) k_norm(const NormJob* __restrict__ jobs, T rtol) {
    __shared__ T x[NMAX];
    __shared__ T y[NMAX];
    __shared__ double red[NT / 32];
    const NormJob J = jobs[blockIdx.x];
    const int m = J.m, n = J.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double nx = 0.0;
    for (int j = threadIdx.x; j < n; j += NT) {
        x[j] = (T)(1.0 + 0.37 * (double)j / (double)(n > 0 ? n : 1));
        nx += (double)x[j] * x[j];
    }
    nx = block_sum<NT>(nx, red);
    double sigma = 0.0, prev = -1.0;
    for (int it = 0; it <= NITER && nx > 0.0; ++it) {
        const T ix = (T)(1.0 / sqrt(nx));
        for (int j = threadIdx.x; j < n; j += NT) x[j] *= ix;
        __syncthreads();
        double ny = 0.0;
        for (int i = threadIdx.x; i < m; i += NT) {
            T s = 0;
            for (int j = 0; j < n; ++j) s += (T)J.A[i + (size_t)j * J.lda] * x[j];
            y[i] = s;
            ny += (double)s * s;
        }
        ny = block_sum<NT>(ny, red);
        sigma = sqrt(ny);
        if (it == NITER || ny == 0.0 || fabs(sigma - prev) <= (double)rtol * sigma) break;
        prev = sigma;
        nx = 0.0;
        for (int j = warp; j < n; j += NT / 32) {
            const double* a = J.A + (size_t)j * J.lda;
            T s = 0;
            for (int i = lane; i < m; i += 32) s += (T)a[i] * y[i];
            s = warp_sum_t<T>(s);
            if (lane == 0) x[j] = s;
            nx += (lane == 0) ? (double)s * s : 0.0;
        }
        nx = block_sum<NT>(nx, red);
    }
    if (threadIdx.x == 0) {
        if (J.nrm) *J.nrm = sigma;
        if (J.inv) *J.inv = sigma > 1e-300 ? 1.0 / sigma : 0.0;
    }
}

void launch_norm(const NormJob* jobs, int njobs, int precision, cudaStream_t st) {
    if (njobs <= 0) return;
    if (precision == H2_MIXED)
        k_norm<float><<<njobs, NT, 0, st>>>(jobs, 1e-5f);
    else
        k_norm<double><<<njobs, NT, 0, st>>>(jobs, 1e-10);
}

// ------------------------------------------------------------------ copies
__global__ void k_copy(const CopyJob* __restrict__ jobs) {
    const CopyJob J = jobs[blockIdx.x];
    const double f = J.alpha * (J.scale ? *J.scale : 1.0);
    const int64_t tot = (int64_t)J.rows * J.cols;
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
        int i = (int)(e % J.rows), j = (int)(e / J.rows);
        double v = J.trans ? J.src[j + (size_t)i * J.lds] : J.src[i + (size_t)j * J.lds];
        double* d = J.dst + i + (size_t)j * J.ldd;
        *d = (J.beta == 0.0) ? f * v : J.beta * *d + f * v;
    }
}

// Copy of the descriptor arrays of a launch from mapped pinned host memory, in
// stream order on the SMs: no copy engine, so the uploads of one stream never
// queue behind the copies of another.
__global__ void k_pull(PullBatch b) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int s = 0; s < b.n; ++s) {
        const uint4* src = (const uint4*)b.seg[s].src;
        uint4* dst = (uint4*)b.seg[s].dst;
        const size_t n = (b.seg[s].bytes + 15) / 16;
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
    }
}

void launch_pull(const PullBatch& b, cudaStream_t st) {
    size_t words = 0;
    for (int s = 0; s < b.n; ++s) words = std::max(words, (b.seg[s].bytes + 15) / 16);
    if (words == 0) return;
    const int grid = (int)std::min<size_t>((words + 255) / 256, (size_t)2 * device_sm_count());
    k_pull<<<grid, 256, 0, st>>>(b);
}

void launch_copy(const CopyJob* jobs, int njobs, cudaStream_t st) {
    if (njobs > 0) k_copy<<<njobs, 256, 0, st>>>(jobs);
}

__global__ void k_identity(double* A, int m, int n, int lda) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % m), j = (int)(e / m);
        A[i + (size_t)j * lda] = (i == j) ? 1.0 : 0.0;
    }
}

void launch_set_identity(double* A, int m, int n, int lda, cudaStream_t st) {
    int64_t tot = (int64_t)m * n;
    if (tot > 0) k_identity<<<(int)std::min<int64_t>(ceil_div(tot, 256), 4096), 256, 0, st>>>(A, m, n, lda);
}

__global__ void k_finite(const double* A, size_t len, int* flag) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(A[e])) {
            atomicOr(flag, 2);
            return;
        }
}

void launch_check_finite(const double* A, size_t len, int* flag, cudaStream_t st) {
    if (len > 0) k_finite<<<(int)std::min<size_t>(ceil_div(len, 256), 2048), 256, 0, st>>>(A, len, flag);
}

// ------------------------------------------------------------------ interpolation
// First-kind Chebyshev nodes on [a, b] and Lagrange polynomials (Example
// "Integral operator"), tensor index nu = ix + m iy + m^2 iz.
__device__ __forceinline__ double cheb_node(double a, double b, int i, int m) {
    return 0.5 * (a + b) + 0.5 * (b - a) * cos((2 * i + 1) * M_PI / (2 * m));
}

// l_i(x) = prod_{j != i} (x - x_j) / (x_i - x_j) for the nodes xs[0..m-1] (the
// values cheb_node gives, computed once per cluster and kept in shared memory)
__device__ double lagrange_n(const double* xs, int m, int i, double x) {
    const double xi = xs[i];
    double v = 1.0;
    for (int j = 0; j < m; ++j)
        if (j != i) v *= (x - xs[j]) / (xi - xs[j]);
    return v;
}

// l_i'(x) from the nodes xs[0..m-1]: the product rule over the factors of l_i
__device__ double lagrange_deriv_n(const double* xs, int m, int i, double x) {
    const double xi = xs[i];
    double sum = 0.0;
    for (int k = 0; k < m; ++k) {
        if (k == i) continue;
        double term = 1.0 / (xi - xs[k]);
        for (int j = 0; j < m; ++j)
            if (j != i && j != k) term *= (x - xs[j]) / (xi - xs[j]);
        sum += term;
    }
    return sum;
}

// ny: the normal at y (H2_K_DLP only)
__device__ double kernel_eval(int kernel, const double* x, const double* y, const double* ny = nullptr) {
    if (kernel == H2_K_DLP) {
        const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 == 0.0) return 0.0;
        const double r = sqrt(r2);
        return (ny[0] * d0 + ny[1] * d1 + ny[2] * d2) / (4.0 * M_PI * r2 * r);
    }
    if (kernel == H2_K_POLY2) {
        double d = 1.0 + x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
        return d * d;
    }
    if (kernel == H2_K_CONST) return 1.0;
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (kernel == H2_K_DELTA) return r == 0.0 ? 1.0 : 0.0;
    if (r == 0.0) return 0.0;
    if (kernel == H2_K_LAPLACE) return 1.0 / (4.0 * M_PI * r);
    return exp(-r) / r;
}

// leaf bases: one thread per (point, nu); with normals the normal derivative
__global__ void k_interp_leaf(const double* pts, const double* nrm, const int64_t* perm, const int64_t* off,
                              const int64_t* size, const double* lo, const double* hi, double* const* leafp,
                              int first_leaf, int m) {
    __shared__ double ln[3][8];  // the leaf's nodes (m <= 8)
    const int leaf = first_leaf + blockIdx.y;
    const int k = m * m * m;
    const int64_t cnt = size[leaf];
    if (threadIdx.x < 3 * m) {
        const int a = threadIdx.x / m, j = threadIdx.x % m;
        ln[a][j] = cheb_node(lo[3 * leaf + a], hi[3 * leaf + a], j, m);
    }
    __syncthreads();
    double* out = leafp[leaf];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt * k; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % cnt;
        int nu = (int)(e / cnt);
        int ix = nu % m, iy = (nu / m) % m, iz = nu / (m * m);
        const int64_t p = perm[off[leaf] + i];
        const double* x = pts + 3 * p;
        const double lx = lagrange_n(ln[0], m, ix, x[0]), ly = lagrange_n(ln[1], m, iy, x[1]),
                     lz = lagrange_n(ln[2], m, iz, x[2]);
        double v;
        if (nrm) {
            const double* nv = nrm + 3 * p;
            v = lagrange_deriv_n(ln[0], m, ix, x[0]) * ly * lz * nv[0] +
                lx * lagrange_deriv_n(ln[1], m, iy, x[1]) * lz * nv[1] +
                lx * ly * lagrange_deriv_n(ln[2], m, iz, x[2]) * nv[2];
        } else {
            v = lx * ly * lz;
        }
        out[i + (size_t)nu * cnt] = v;
    }
}

void launch_interp_leaf(const double* pts, const double* nrm, const int64_t* perm, const int64_t* off,
                        const int64_t* size, const double* lo, const double* hi, double* const* leafp, int first_leaf,
                        int nleaves, int m, int64_t max_size, cudaStream_t st) {
    int k = m * m * m;
    int gx = (int)std::min<int64_t>(ceil_div(max_size * k, 128), 1024);
    dim3 grid(gx, nleaves);
    if (nleaves > 0) k_interp_leaf<<<grid, 128, 0, st>>>(pts, nrm, perm, off, size, lo, hi, leafp, first_leaf, m);
}

// transfers: E_c[nu', nu] = l_{parent, nu}(xi_{c, nu'}), one block per cluster c >= 1
__global__ void k_interp_transfer(const double* lo, const double* hi, double* const* trp, int m) {
    __shared__ double cn[3][8], pn[3][8];  // the child's and the parent's nodes (m <= 8)
    const int c = blockIdx.x + 1, p = (c - 1) / 2;
    const int k = m * m * m;
    const double *lc = lo + 3 * c, *hc = hi + 3 * c, *lp = lo + 3 * p, *hp = hi + 3 * p;
    if (threadIdx.x < 3 * m) {
        const int a = threadIdx.x / m, i = threadIdx.x % m;
        cn[a][i] = cheb_node(lc[a], hc[a], i, m);
        pn[a][i] = cheb_node(lp[a], hp[a], i, m);
    }
    __syncthreads();
    double* out = trp[c];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        int nu1 = e % k, nu = e / k;
        int a0 = nu1 % m, a1 = (nu1 / m) % m, a2 = nu1 / (m * m);
        int b0 = nu % m, b1 = (nu / m) % m, b2 = nu / (m * m);
        out[nu1 + (size_t)nu * k] = lagrange_n(pn[0], m, b0, cn[0][a0]) * lagrange_n(pn[1], m, b1, cn[1][a1]) *
                                    lagrange_n(pn[2], m, b2, cn[2][a2]);
    }
}

void launch_interp_transfer(const double* lo, const double* hi, double* const* trp, int nc, int m, cudaStream_t st) {
    if (nc > 1) k_interp_transfer<<<nc - 1, 256, 0, st>>>(lo, hi, trp, m);
}

// couplings: S_ts[nu, mu] = g(xi_{t,nu}, xi_{s,mu}), one block per admissible block
__global__ void k_interp_coupling(const double* lo, const double* hi, const int* bt, const int* bs,
                                  double* const* bp, int m, int kernel) {
    // the 3 m node coordinates of each cluster, once per block: every entry of the
    // coupling reuses them (a cosine per coordinate per entry had dominated the kernel)
    __shared__ double xn[3][8], yn[3][8];  // m <= 8
    const int b = blockIdx.x, t = bt[b], s = bs[b];
    const int k = m * m * m;
    const double *lt = lo + 3 * t, *ht = hi + 3 * t, *ls = lo + 3 * s, *hs = hi + 3 * s;
    if (threadIdx.x < 3 * m) {
        const int a = threadIdx.x / m, i = threadIdx.x % m;
        xn[a][i] = cheb_node(lt[a], ht[a], i, m);
        yn[a][i] = cheb_node(ls[a], hs[a], i, m);
    }
    __syncthreads();
    double* out = bp[b];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        int nu = e % k, mu = e / k;
        double x[3] = {xn[0][nu % m], xn[1][(nu / m) % m], xn[2][nu / (m * m)]};
        double y[3] = {yn[0][mu % m], yn[1][(mu / m) % m], yn[2][mu / (m * m)]};
        // the double-layer kernel is the normal derivative (carried by W) of the Laplace kernel
        out[nu + (size_t)mu * k] = kernel_eval(kernel == H2_K_DLP ? H2_K_LAPLACE : kernel, x, y);
    }
}

void launch_interp_coupling(const double* lo, const double* hi, const int* bt, const int* bs, double* const* bp,
                            int nblocks, int m, int kernel, cudaStream_t st) {
    if (nblocks > 0) k_interp_coupling<<<nblocks, 256, 0, st>>>(lo, hi, bt, bs, bp, m, kernel);
}

// dense blocks: N_ts[i, j] = g(x_i, x_j) (normals of the column points for H2_K_DLP)
__global__ void k_interp_dense(const double* pts, const double* nrm, const int64_t* perm, const int64_t* off,
                               const int64_t* size, const int* bt, const int* bs, double* const* bp, int kernel) {
    const int b = blockIdx.x, t = bt[b], s = bs[b];
    const int64_t mt = size[t], ms = size[s];
    double* out = bp[b];
    for (int64_t e = threadIdx.x; e < mt * ms; e += blockDim.x) {
        int64_t i = e % mt, j = e / mt;
        const int64_t pj = perm[off[s] + j];
        out[e] = kernel_eval(kernel, pts + 3 * perm[off[t] + i], pts + 3 * pj, nrm ? nrm + 3 * pj : nullptr);
    }
}

void launch_interp_dense(const double* pts, const double* nrm, const int64_t* perm, const int64_t* off,
                         const int64_t* size, const int* bt, const int* bs, double* const* bp, int nblocks, int kernel,
                         cudaStream_t st) {
    if (nblocks > 0) k_interp_dense<<<nblocks, 256, 0, st>>>(pts, nrm, perm, off, size, bt, bs, bp, kernel);
}

// ------------------------------------------------------------------ block norms
__global__ void k_sumsq(const SumSqJob* __restrict__ jobs, double* part) {
    __shared__ double red[256 / 32];
    const SumSqJob J = jobs[blockIdx.x];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)J.rows * J.cols; e += 256) {
        double v = J.A[(e % J.rows) + (size_t)(e / J.rows) * J.lda];
        s += v * v;
    }
    s = block_sum<256>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// the jobs' sums added per slot in job order (no atomics: the same inputs give the
// same bits on every run)
__global__ void k_segment_sum(const double* __restrict__ part, const int* __restrict__ seg, int nslots,
                              double* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nslots) return;
    double s = 0.0;
    for (int j = seg[b]; j < seg[b + 1]; ++j) s += part[j];
    out[b] = s;
}

void launch_sumsq(const SumSqJob* jobs, int njobs, double* part, const int* seg, int nslots, double* out,
                  cudaStream_t st) {
    if (njobs > 0) k_sumsq<<<njobs, 256, 0, st>>>(jobs, part);
    if (nslots > 0) k_segment_sum<<<(int)ceil_div(nslots, 256), 256, 0, st>>>(part, seg, nslots, out);
}

std::vector<int> sumsq_segments(std::vector<SumSqJob>& jobs, int nslots) {
    std::stable_sort(jobs.begin(), jobs.end(), [](const SumSqJob& a, const SumSqJob& b) { return a.slot < b.slot; });
    std::vector<int> seg((size_t)nslots + 1, 0);
    for (const SumSqJob& j : jobs) ++seg[(size_t)j.slot + 1];
    for (int b = 0; b < nslots; ++b) seg[(size_t)b + 1] += seg[b];
    return seg;
}

__global__ void k_inv_sqrt(const double* v, double* w, double* w2, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        w[i] = v[i] > 0.0 ? 1.0 / sqrt(v[i]) : 0.0;
        if (w2) w2[i] = v[i] > 0.0 ? 1.0 / v[i] : 0.0;
    }
}

void launch_inv_sqrt(const double* v, double* w, double* w2, int n, cudaStream_t st) {
    if (n > 0) k_inv_sqrt<<<(int)ceil_div(n, 256), 256, 0, st>>>(v, w, w2, n);
}

// row permutation of an n x nv matrix (gather or scatter)
__global__ void k_permute_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* perm,
                               int64_t n, int64_t nv, int scatter) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nv; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % n, j = e / n;
        if (scatter)
            dst[perm[i] + j * ldd] = src[i + j * lds];
        else
            dst[i + j * ldd] = src[perm[i] + j * lds];
    }
}

void launch_permute_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* perm, int64_t n,
                         int64_t nv, int scatter, cudaStream_t st) {
    if (n > 0 && nv > 0)
        k_permute_rows<<<(int)std::min<int64_t>(ceil_div(n * nv, 256), 8192), 256, 0, st>>>(src, lds, dst, ldd, perm,
                                                                                             n, nv, scatter);
}

// dense n x n matrix in tree order -> original order
__global__ void k_scatter(const double* src, int64_t n, const int64_t* perm, double* out, int64_t ld) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % n, j = e / n;
        out[perm[i] + perm[j] * ld] = src[e];
    }
}

void launch_scatter_dense(const double* src, int64_t n, const int64_t* perm, double* out, int64_t ld, cudaStream_t st) {
    if (n > 0) k_scatter<<<(int)std::min<int64_t>(ceil_div(n * n, 256), 8192), 256, 0, st>>>(src, n, perm, out, ld);
}

}  // namespace h2
