// Device kernels of the H^2 product library (sm_103a).
//
// Batched small dense linear algebra: every launch covers all clusters or all
// blocks of one tree level at once.  Each batched kernel reads a device array
// of job descriptors built by the host executor.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "h2_internal.h"

namespace h2 {

// ------------------------------------------------------------------ GEMM
// C = beta C + sum_terms alpha_t op(A_t) op(B_t) over 32 x 32 output tiles.
// T is the arithmetic type: double (H2_FP64) or float (H2_MIXED; operands are
// rounded to FP32 when staged in shared memory, accumulation in FP32).
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
    T acc[2][2] = {{0, 0}, {0, 0}};
    for (int it = 0; it < J.nt; ++it) {
        const GTerm P = terms[J.t0 + it];
        const double f = P.alpha * (P.scale ? *P.scale : 1.0);
        if (f == 0.0) continue;
        for (int k0 = 0; k0 < P.k; k0 += GK) {
            // stage op(A)[i0:i0+32, k0:k0+16] and op(B)[k0:k0+16, j0:j0+32]
            for (int e = threadIdx.x; e < GK * GB; e += GT) {
                int i, kk;
                if (!P.ta) { i = e % GB; kk = e / GB; } else { kk = e % GK; i = e / GK; }
                int gi = tile.i0 + i, gk = k0 + kk;
                double v = 0.0;
                if (gi < J.m && gk < P.k) v = P.ta ? P.A[gk + (size_t)gi * P.lda] : P.A[gi + (size_t)gk * P.lda];
                As[kk][i] = (T)(f * v);
                int j;
                if (!P.tb) { kk = e % GK; j = e / GK; } else { j = e % GB; kk = e / GB; }
                int gj = tile.j0 + j;
                gk = k0 + kk;
                double w = 0.0;
                if (gj < J.n && gk < P.k) w = P.tb ? P.B[gj + (size_t)gk * P.ldb] : P.B[gk + (size_t)gj * P.ldb];
                Bs[kk][j] = (T)w;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < GK; ++kk) {
                T a0 = As[kk][tx], a1 = As[kk][tx + 16];
                T b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
                acc[0][0] += a0 * b0;
                acc[1][0] += a1 * b0;
                acc[0][1] += a0 * b1;
                acc[1][1] += a1 * b1;
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
            }
        }
}

void launch_gemm(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int precision,
                 cudaStream_t st) {
    if (ntiles <= 0) return;
    if (precision == H2_MIXED)
        k_gemm<float><<<ntiles, GT, 0, st>>>(terms, jobs, tiles);
    else
        k_gemm<double><<<ntiles, GT, 0, st>>>(terms, jobs, tiles);
}

// ------------------------------------------------------------------ GEMM on tcgen05 (H2_TC)
// Same contract as k_gemm on the 5th-generation tensor cores.  One CTA of 128
// threads computes a 128 x 64 output tile.  The operands of each K chunk are
// rounded to FP32 and staged in shared memory as three TF32 pieces x = x0 + x1
// + x2 (each rna of the remainder; together they hold the 24 bits of the FP32
// value exactly) in the K-major core-matrix layout (8 rows x 16 bytes per core
// matrix).  One thread issues tcgen05.mma.kind::tf32: a0 b0 into accumulator
// D0 and the five correction products of order 2^-11 .. 2^-22 (a0 b1, a1 b0,
// a0 b2, a1 b1, a2 b0) into D1 (two 128-lane x 64-column FP32 accumulators in
// TMEM).  The tensor cores' FP32 accumulation rounds toward zero, so the
// accumulators only live for one chunk: after each chunk tcgen05.ld moves them
// into registers, where a compensated (Kahan) FP32 sum carries the result.
// Waits on the MMA completion barrier are bounded: on timeout the kernel
// records the error, frees its TMEM and returns.
constexpr int TC_M = 128, TC_N = 64, TC_K = 32, TC_T = 128;
constexpr int TC_A = TC_M * TC_K, TC_B = TC_N * TC_K;  // elements per operand tile
constexpr int TC_PIECES = 3;
constexpr int TC_COLS = 2 * TC_N;  // two accumulators
constexpr size_t TC_SMEM = TC_PIECES * (size_t)(TC_A + TC_B) * 4 + 64;

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// element (row r, k) of a K-major tile with TC_K columns
__device__ __forceinline__ int core_index(int r, int k) {
    return ((r >> 3) * (TC_K / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// shared memory descriptor: K-major, no swizzle; LBO = 128 B (next core in K),
// SBO = (TC_K / 4) * 128 B (next 8-row group)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    const uint64_t lbo = 128, sbo = (TC_K / 4) * 128;
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
    uint32_t* u = (uint32_t*)v;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
        "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
          "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
          "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31]),
          "=r"(u[32]), "=r"(u[33]), "=r"(u[34]), "=r"(u[35]), "=r"(u[36]), "=r"(u[37]), "=r"(u[38]), "=r"(u[39]),
          "=r"(u[40]), "=r"(u[41]), "=r"(u[42]), "=r"(u[43]), "=r"(u[44]), "=r"(u[45]), "=r"(u[46]), "=r"(u[47]),
          "=r"(u[48]), "=r"(u[49]), "=r"(u[50]), "=r"(u[51]), "=r"(u[52]), "=r"(u[53]), "=r"(u[54]), "=r"(u[55]),
          "=r"(u[56]), "=r"(u[57]), "=r"(u[58]), "=r"(u[59]), "=r"(u[60]), "=r"(u[61]), "=r"(u[62]), "=r"(u[63])
        : "r"(taddr));
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

__global__ void __launch_bounds__(TC_T) k_gemm_tc(const GTerm* __restrict__ terms, const GJob* __restrict__ jobs,
                                                  const GTile* __restrict__ tiles, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    uint32_t* as = (uint32_t*)tc_smem;     // pieces 0..2 of A, TC_A elements each
    uint32_t* bs = as + TC_PIECES * TC_A;  // pieces 0..2 of B, TC_B elements each
    uint64_t* mbar = (uint64_t*)(bs + TC_PIECES * TC_B);
    uint32_t* tmem_slot = (uint32_t*)(mbar + 1);
    const GTile tile = tiles[blockIdx.x];
    const GJob J = jobs[tile.job];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tmem_slot)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_s));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    float sum[TC_N], comp[TC_N], v[TC_N];
#pragma unroll
    for (int c = 0; c < TC_N; ++c) sum[c] = comp[c] = 0.f;
    uint32_t phase = 0;
    bool failed = false;
    for (int it = 0; it < J.nt && !failed; ++it) {
        const GTerm P = terms[J.t0 + it];
        const double f = P.alpha * (P.scale ? *P.scale : 1.0);
        if (f == 0.0) continue;
        const float ff = (float)f;
        for (int k0 = 0; k0 < P.k && !failed; k0 += TC_K) {
            // stage op(A)[i0:i0+128, k0:k0+32] and op(B)^T[j0:j0+64, k0:k0+32]
            for (int e = threadIdx.x; e < TC_A; e += TC_T) {
                int r, kk;
                if (!P.ta) { r = e % TC_M; kk = e / TC_M; } else { kk = e % TC_K; r = e / TC_K; }
                int gi = tile.i0 + r, gk = k0 + kk;
                float x = 0.f;
                if (gi < J.m && gk < P.k)
                    x = ff * (float)(P.ta ? P.A[gk + (size_t)gi * P.lda] : P.A[gi + (size_t)gk * P.lda]);
                const int ci = core_index(r, kk);
                const uint32_t p0 = tf32_rna(x);
                const float r1 = x - __uint_as_float(p0);
                const uint32_t p1 = tf32_rna(r1);
                as[ci] = p0;
                as[TC_A + ci] = p1;
                as[2 * TC_A + ci] = tf32_rna(r1 - __uint_as_float(p1));
            }
            for (int e = threadIdx.x; e < TC_B; e += TC_T) {
                int c, kk;
                if (!P.tb) { kk = e % TC_K; c = e / TC_K; } else { c = e % TC_N; kk = e / TC_N; }
                int gj = tile.j0 + c, gk = k0 + kk;
                float x = 0.f;
                if (gj < J.n && gk < P.k) x = (float)(P.tb ? P.B[gj + (size_t)gk * P.ldb] : P.B[gk + (size_t)gj * P.ldb]);
                const int ci = core_index(c, kk);
                const uint32_t p0 = tf32_rna(x);
                const float r1 = x - __uint_as_float(p0);
                const uint32_t p1 = tf32_rna(r1);
                bs[ci] = p0;
                bs[TC_B + ci] = p1;
                bs[2 * TC_B + ci] = tf32_rna(r1 - __uint_as_float(p1));
            }
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(as);
                const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(bs);
                constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
                constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                for (int ks = 0; ks < TC_K / 8; ++ks) {
                    const uint32_t off = ks * 2 * 128;  // two core matrices of K per MMA
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const uint64_t da = smem_desc(a0 + (uint32_t)(pa[q] * TC_A * 4) + off);
                        const uint64_t db = smem_desc(b0 + (uint32_t)(pb[q] * TC_B * 4) + off);
                        // D0 (columns 0..63) takes a0 b0, D1 (columns 64..127) the corrections;
                        // each starts afresh in every chunk
                        const uint32_t d = (q == 0) ? tmem : tmem + TC_N;
                        const uint32_t acc = (ks > 0 || q > 1) ? 1u : 0u;
                        tc_mma(d, da, db, acc);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    mbar_s));
            }
            // bounded wait for the MMAs of this chunk
            uint32_t done = 0;
            for (long spin = 0; spin < (1L << 24) && !done; ++spin) {
                asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                             : "=r"(done)
                             : "r"(mbar_s), "r"(phase));
            }
            // one decision for the whole CTA (the barriers above and below must match)
            failed = __syncthreads_or(done ? 0 : 1) != 0;
            if (failed && threadIdx.x == 0 && err) atomicOr(err, 4);
            phase ^= 1;
            if (!failed) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                // move both accumulators into the compensated register sums
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    tmem_ld64(tmem + lane_base + (uint32_t)(half * TC_N), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int c = 0; c < TC_N; ++c) {
                        const float y = v[c] - comp[c];
                        const float t = sum[c] + y;
                        comp[c] = (t - sum[c]) - y;
                        sum[c] = t;
                    }
                }
                // the next chunk's MMAs overwrite the accumulators only after these loads
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
            }
        }
    }
    if (!failed) {
        const int gi = tile.i0 + warp * 32 + lane;
        if (gi < J.m) {
#pragma unroll
            for (int c = 0; c < TC_N; ++c) {
                const int gj = tile.j0 + c;
                if (gj < J.n) {
                    double* cp = J.C + gi + (size_t)gj * J.ldc;
                    const double val = (double)sum[c] - (double)comp[c];
                    *cp = (J.beta == 0.0) ? val : J.beta * *cp + val;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

void launch_gemm_tc(const GTerm* terms, const GJob* jobs, const GTile* tiles, int ntiles, int* err, cudaStream_t st) {
    if (ntiles <= 0) return;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        attr_set[dev] = true;
    }
    k_gemm_tc<<<ntiles, TC_T, TC_SMEM, st>>>(terms, jobs, tiles, err);
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
    const QRJob J = jobs[blockIdx.x];
    const int m = J.m, n = J.n, p = m < n ? m : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = QT / 32;
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
    for (int j = 0; j < p; ++j) {
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
        if (tau != 0.0) {
            const T tt = (T)tau;
            for (int c = j + 1 + warp; c < n; c += nw) {
                T* a = A + (size_t)c * lda;
                T w = 0;
                for (int i = j + 1 + lane; i < m; i += 32) w += col[i] * a[i];
                w = warp_sum_t<T>(w);
                __syncwarp();
                w = (w + a[j]) * tt;
                __syncwarp();
                if (lane == 0) a[j] -= w;
                for (int i = j + 1 + lane; i < m; i += 32) a[i] -= w * col[i];
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
// sweep count is bounded; *flag reports a run that hit the bound.
constexpr int JT = 512;
constexpr int JMAXSWEEP = 40;
constexpr int JMAXN = 2048;

__device__ __forceinline__ int rr_player(int pos, int round, int np) {
    if (pos == 0) return 0;
    return 1 + (pos - 1 + round) % (np - 1);
}

__global__ void __launch_bounds__(JT) k_svd(const SVDJob* __restrict__ jobs) {
    __shared__ int rotated;
    __shared__ double sig[JMAXN];
    const SVDJob J = jobs[blockIdx.x];
    const int m = J.m, n = J.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    const int np = n + (n & 1);
    const double tol = (double)(m > 1 ? m : 1) * DBL_EPSILON;
    // a sweep whose rotation measures all stay below skip = 0.1 sqrt(tol) leaves an
    // off-diagonality below tol (quadratic convergence): the verifying sweep is skipped
    const double skip = 0.1 * sqrt(tol);
    __shared__ int large;
    int sweep = 0;
    bool converged = (n < 2);
    for (; sweep < JMAXSWEEP && !converged; ++sweep) {
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
                double* ap = J.B + (size_t)p * J.ldb;
                double* aq = J.B + (size_t)q * J.ldb;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < m; i += 32) {
                    double x = ap[i], y = aq[i];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga != 0.0 && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
                    double zeta = (be - al) / (2.0 * ga);
                    double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                                     : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    for (int i = lane; i < m; i += 32) {
                        double x = ap[i], y = aq[i];
                        ap[i] = c * x - s * y;
                        aq[i] = s * x + c * y;
                    }
                    if (lane == 0) {
                        rotated = 1;
                        if (fabs(ga) > skip * sqrt(al) * sqrt(be)) large = 1;
                    }
                }
            }
            __syncthreads();
        }
        converged = (rotated == 0) || (large == 0);
        __syncthreads();
    }
    if (threadIdx.x == 0 && !converged && J.flag) atomicOr(J.flag, 1);
    if (threadIdx.x == 0 && J.flops) atomicAdd(J.flops, 12.0 * m * (0.5 * n * (n - 1.0)) * sweep);
    for (int c = warp; c < n; c += nw) {
        const double* a = J.B + (size_t)c * J.ldb;
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += a[i] * a[i];
        s = warp_sum(s);
        if (lane == 0) sig[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = warp; c < n; c += nw) {
        const double sc = sig[c];
        int pos = 0;
        for (int q = 0; q < n; ++q) pos += (sig[q] > sc) || (sig[q] == sc && q < c);
        const double* a = J.B + (size_t)c * J.ldb;
        double* u = J.U + (size_t)pos * J.ldu;
        const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
        for (int i = lane; i < m; i += 32) u[i] = a[i] * inv;
        if (lane == 0) J.sigma[pos] = sc;
    }
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int q = 0; q < n; ++q) cnt += (sig[q] > J.eps);
        *J.count = cnt;
    }
}

// FP32 preconditioning sweeps: the same rotations as k_svd on an FP32 copy W
// of B, accumulated into V (V starts as the identity).  Bounded sweeps.
constexpr int PMAXSWEEP = 30;

// W lives in dynamic shared memory when its m * n floats fit in the launch's
// smem_bytes (sized for the largest job, at most kPreSmem), else in its
// global workspace.
constexpr int kPreSmem = 160 * 1024;

__global__ void __launch_bounds__(JT) k_jacobi_pre(const PreJob* __restrict__ jobs, int smem_bytes) {
    extern __shared__ float pre_smem[];
    __shared__ int rotated;
    const PreJob J = jobs[blockIdx.x];
    const int m = J.m, n = J.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    const bool in_smem = (size_t)m * n * sizeof(float) <= (size_t)smem_bytes;
    float* W = in_smem ? pre_smem : J.W;
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += JT) W[e] = (float)J.B[(e % m) + (size_t)(e / m) * J.ldb];
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += JT) J.V[e] = ((e % n) == (e / n)) ? 1.f : 0.f;
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
                    float* vp = J.V + (size_t)p * n;
                    float* vq = J.V + (size_t)q * n;
                    for (int i = lane; i < n; i += 32) {
                        float x = vp[i], y = vq[i];
                        vp[i] = c * x - s * y;
                        vq[i] = s * x + c * y;
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
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += JT) J.V64[e] = (double)J.V[e];
    if (threadIdx.x == 0 && J.flops) atomicAdd(J.flops, 12.0 * (m + n) * (0.5 * n * (n - 1.0)) * sweep);
}

// ------------------------------------------------------------------ clustered Jacobi
// The same sweeps with one matrix shared by a thread-block cluster: the
// disjoint pairs of a round are spread over the cluster's CTAs (one CTA per
// SM), a cluster barrier separates rounds, columns move through L2
// (ld/st.cg), and the rotation flag of a sweep is OR-ed across the cluster
// through distributed shared memory.  Used when a level has fewer matrices
// than SMs.  T = double: SVDJob (FP64 sweeps + singular vectors); T = float:
// PreJob (FP32 preconditioning with accumulated rotations).
namespace cg = cooperative_groups;

__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tsign(float x) { return copysignf(1.f, x); }
__device__ __forceinline__ double tsign(double x) { return copysign(1.0, x); }

template <class T>
__device__ __forceinline__ void rot_pair(T* ap, T* aq, int m, T c, T s, int lane) {
    for (int i = lane; i < m; i += 32) {
        T x = __ldcg(ap + i), y = __ldcg(aq + i);
        __stcg(ap + i, c * x - s * y);
        __stcg(aq + i, s * x + c * y);
    }
}

template <class T>
__global__ void __launch_bounds__(JT) k_jacobi_cluster(const SVDJob* __restrict__ sjobs,
                                                       const PreJob* __restrict__ pjobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    const int job = blockIdx.x / cs;
    __shared__ int rotated;
    __shared__ double sig[JMAXN];
    constexpr bool PRE = sizeof(T) == 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = JT / 32;
    int m, n;
    T* B;
    T* V = nullptr;
    if constexpr (PRE) {
        const PreJob& J = pjobs[job];
        m = J.m;
        n = J.n;
        B = (T*)J.W;
        V = (T*)J.V;
        for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)m * n; e += (int64_t)JT * cs)
            __stcg(B + e, (T)J.B[(e % m) + (size_t)(e / m) * J.ldb]);
        for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)n * n; e += (int64_t)JT * cs)
            __stcg(V + e, ((e % n) == (e / n)) ? (T)1 : (T)0);
    } else {
        const SVDJob& J = sjobs[job];
        m = J.m;
        n = J.n;
        B = (T*)J.B;
    }
    const int ldb = PRE ? m : (int)sjobs[job].ldb;
    cl.sync();
    const int np = n + (n & 1);
    const T tol = (T)(m > 1 ? m : 1) * (PRE ? (T)FLT_EPSILON : (T)DBL_EPSILON);
    const int maxsweep = PRE ? PMAXSWEEP : JMAXSWEEP;
    const T skip = (T)0.1 * tsqrt(tol);
    __shared__ int large;
    bool converged = (n < 2);
    int sweep = 0;
    for (; sweep < maxsweep && !converged; ++sweep) {
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
                T* ap = B + (size_t)p * ldb;
                T* aq = B + (size_t)q * ldb;
                T al = 0, be = 0, ga = 0;
                for (int i = lane; i < m; i += 32) {
                    T x = __ldcg(ap + i), y = __ldcg(aq + i);
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum_t<T>(al);
                be = warp_sum_t<T>(be);
                ga = warp_sum_t<T>(ga);
                if (ga != (T)0 && al > (T)0 && be > (T)0 && tabs(ga) > tol * tsqrt(al) * tsqrt(be)) {
                    T zeta = (be - al) / ((T)2 * ga);
                    const T big = PRE ? (T)1e18 : (T)1e150;
                    T t = (tabs(zeta) > big) ? (T)0.5 / zeta : tsign(zeta) / (tabs(zeta) + tsqrt((T)1 + zeta * zeta));
                    T c = (T)1 / tsqrt((T)1 + t * t), s = c * t;
                    rot_pair<T>(ap, aq, m, c, s, lane);
                    if (PRE) rot_pair<T>(V + (size_t)p * n, V + (size_t)q * n, n, c, s, lane);
                    if (lane == 0) {
                        rotated = 1;
                        if (tabs(ga) > skip * tsqrt(al) * tsqrt(be)) large = 1;
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
    if constexpr (PRE) {
        const PreJob& J = pjobs[job];
        for (int64_t e = threadIdx.x + (int64_t)cr * JT; e < (int64_t)n * n; e += (int64_t)JT * cs)
            J.V64[e] = (double)__ldcg(V + e);
        if (cr == 0 && threadIdx.x == 0 && J.flops) atomicAdd(J.flops, 12.0 * (m + n) * (0.5 * n * (n - 1.0)) * sweep);
        return;
    } else {
        const SVDJob& J = sjobs[job];
        if (cr != 0) return;
        if (threadIdx.x == 0 && !converged && J.flag) atomicOr(J.flag, 1);
        if (threadIdx.x == 0 && J.flops) atomicAdd(J.flops, 12.0 * m * (0.5 * n * (n - 1.0)) * sweep);
        for (int c = warp; c < n; c += nw) {
            const T* a = B + (size_t)c * ldb;
            double s = 0.0;
            for (int i = lane; i < m; i += 32) {
                double v = (double)__ldcg(a + i);
                s += v * v;
            }
            s = warp_sum(s);
            if (lane == 0) sig[c] = sqrt(s);
        }
        __syncthreads();
        for (int c = warp; c < n; c += nw) {
            const double sc = sig[c];
            int pos = 0;
            for (int q = 0; q < n; ++q) pos += (sig[q] > sc) || (sig[q] == sc && q < c);
            const T* a = B + (size_t)c * ldb;
            double* u = J.U + (size_t)pos * J.ldu;
            const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
            for (int i = lane; i < m; i += 32) u[i] = (double)__ldcg(a + i) * inv;
            if (lane == 0) J.sigma[pos] = sc;
        }
        if (threadIdx.x == 0) {
            int cnt = 0;
            for (int q = 0; q < n; ++q) cnt += (sig[q] > J.eps);
            *J.count = cnt;
        }
    }
}

static int num_sms() {
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
constexpr int kClusterDynSmem = 120 * 1024;

// returns false (and clears the error) when the cluster launch is refused
template <class T>
static bool launch_jacobi_cluster(const SVDJob* sj, const PreJob* pj, int njobs, int cs, cudaStream_t st) {
    auto kern = k_jacobi_cluster<T>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterDynSmem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(njobs * cs, 1, 1);
    cfg.blockDim = dim3(JT, 1, 1);
    cfg.dynamicSmemBytes = kClusterDynSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, sj, pj);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

void launch_svd(const SVDJob* jobs, int njobs, int max_n, cudaStream_t st) {
    if (max_n > JMAXN) throw Error(H2_ERR_UNSUPPORTED, "SVD wider than 2048 columns");
    if (njobs <= 0) return;
    int cs = jacobi_cluster_size(njobs);
    if (cs <= 1 || !launch_jacobi_cluster<double>(jobs, nullptr, njobs, cs, st)) k_svd<<<njobs, JT, 0, st>>>(jobs);
}

void launch_jacobi_pre(const PreJob* jobs, int njobs, size_t max_mn, cudaStream_t st) {
    if (njobs <= 0) return;
    int cs = jacobi_cluster_size(njobs);
    if (cs <= 1 || !launch_jacobi_cluster<float>(nullptr, jobs, njobs, cs, st)) {
        static bool attr_set[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            cudaFuncSetAttribute(k_jacobi_pre, cudaFuncAttributeMaxDynamicSharedMemorySize, kPreSmem);
            attr_set[dev] = true;
        }
        const int smem = (max_mn * sizeof(float) <= (size_t)kPreSmem) ? (int)(max_mn * sizeof(float)) : 0;
        k_jacobi_pre<<<njobs, JT, smem, st>>>(jobs, smem);
    }
}

// ------------------------------------------------------------------ pivoted Cholesky
// Symmetric pivoting on the largest remaining diagonal entry (Higham,
// "Accuracy and Stability of Numerical Algorithms", Sec. 10.3), stopped when
// the pivot falls below rel_tol times the largest initial diagonal entry.
constexpr int CT = 256;
constexpr int CMAXK = 1024;

__global__ void __launch_bounds__(CT) k_pchol(const CholJob* __restrict__ jobs) {
    __shared__ int perm[CMAXK];
    __shared__ double rv[CT / 32];
    __shared__ int ri[CT / 32];
    __shared__ int piv;
    __shared__ double pval;
    const CholJob J = jobs[blockIdx.x];
    const int k = J.k;
    double* W = J.W;
    for (int e = threadIdx.x; e < k * k; e += CT) W[e] = J.G[(e % k) + (size_t)(e / k) * J.ldg];
    for (int i = threadIdx.x; i < k; i += CT) perm[i] = i;
    for (int e = threadIdx.x; e < J.zrows * k; e += CT) J.Z[e] = 0.0;
    __syncthreads();
    // largest initial diagonal entry
    double md = 0.0;
    for (int i = threadIdx.x; i < k; i += CT) md = fmax(md, W[i + (size_t)i * k]);
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
        // pivot: argmax of the remaining diagonal (lowest index on ties)
        double best = -1.0;
        int bi = j;
        for (int i = j + threadIdx.x; i < k; i += CT) {
            double d = W[i + (size_t)i * k];
            if (d > best) { best = d; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = best; ri[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = rv[0];
            int i0 = ri[0];
            for (int w = 1; w < CT / 32; ++w)
                if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
            piv = i0;
            pval = b;
        }
        __syncthreads();
        if (!(pval > tol) || !(pval > 0.0)) {
            rank = j;
            break;
        }
        const int p = piv;
        if (p != j) {  // symmetric swap of rows and columns j and p
            for (int c = threadIdx.x; c < k; c += CT) {
                double t = W[j + (size_t)c * k];
                W[j + (size_t)c * k] = W[p + (size_t)c * k];
                W[p + (size_t)c * k] = t;
            }
            __syncthreads();
            for (int r = threadIdx.x; r < k; r += CT) {
                double t = W[r + (size_t)j * k];
                W[r + (size_t)j * k] = W[r + (size_t)p * k];
                W[r + (size_t)p * k] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[j];
                perm[j] = perm[p];
                perm[p] = t;
            }
            __syncthreads();
        }
        const double d = sqrt(W[j + (size_t)j * k]);
        const double inv = 1.0 / d;
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < k; i += CT) W[i + (size_t)j * k] *= inv;
        if (threadIdx.x == 0) W[j + (size_t)j * k] = d;
        __syncthreads();
        // trailing update of the whole trailing square (kept symmetric for the swaps)
        const int rem = k - j - 1;
        for (int64_t e = threadIdx.x; e < (int64_t)rem * rem; e += CT) {
            int i = j + 1 + (int)(e % rem), l = j + 1 + (int)(e / rem);
            W[i + (size_t)l * k] -= W[i + (size_t)j * k] * W[l + (size_t)j * k];
        }
        __syncthreads();
    }
    // Z = L^* P^*: Z[j, perm[i]] = L[i, j] for i >= j, j < rank
    for (int64_t e = threadIdx.x; e < (int64_t)k * rank; e += CT) {
        int i = (int)(e % k), j = (int)(e / k);
        if (i >= j) J.Z[j + (size_t)perm[i] * J.zrows] = W[i + (size_t)j * k];
    }
}

void launch_pchol(const CholJob* jobs, int njobs, cudaStream_t st) {
    if (njobs > 0) k_pchol<<<njobs, CT, 0, st>>>(jobs);
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

__device__ double lagrange(double a, double b, int m, int i, double x) {
    double xi = cheb_node(a, b, i, m), v = 1.0;
    for (int j = 0; j < m; ++j)
        if (j != i) {
            double xj = cheb_node(a, b, j, m);
            v *= (x - xj) / (xi - xj);
        }
    return v;
}

__device__ double kernel_eval(int kernel, const double* x, const double* y) {
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

// leaf bases: one thread per (point, nu)
__global__ void k_interp_leaf(const double* pts, const int64_t* perm, const int64_t* off, const int64_t* size,
                              const double* lo, const double* hi, double* const* leafp, int first_leaf, int m) {
    const int leaf = first_leaf + blockIdx.y;
    const int k = m * m * m;
    const int64_t cnt = size[leaf];
    double* out = leafp[leaf];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt * k; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % cnt;
        int nu = (int)(e / cnt);
        int ix = nu % m, iy = (nu / m) % m, iz = nu / (m * m);
        const double* x = pts + 3 * perm[off[leaf] + i];
        const double* l = lo + 3 * leaf;
        const double* h = hi + 3 * leaf;
        out[i + (size_t)nu * cnt] = lagrange(l[0], h[0], m, ix, x[0]) * lagrange(l[1], h[1], m, iy, x[1]) *
                                    lagrange(l[2], h[2], m, iz, x[2]);
    }
}

void launch_interp_leaf(const double* pts, const int64_t* perm, const int64_t* off, const int64_t* size,
                        const double* lo, const double* hi, double* const* leafp, int first_leaf, int nleaves, int m,
                        int64_t max_size, cudaStream_t st) {
    int k = m * m * m;
    int gx = (int)std::min<int64_t>(ceil_div(max_size * k, 128), 1024);
    dim3 grid(gx, nleaves);
    if (nleaves > 0) k_interp_leaf<<<grid, 128, 0, st>>>(pts, perm, off, size, lo, hi, leafp, first_leaf, m);
}

// transfers: E_c[nu', nu] = l_{parent, nu}(xi_{c, nu'}), one block per cluster c >= 1
__global__ void k_interp_transfer(const double* lo, const double* hi, double* const* trp, int m) {
    const int c = blockIdx.x + 1, p = (c - 1) / 2;
    const int k = m * m * m;
    const double *lc = lo + 3 * c, *hc = hi + 3 * c, *lp = lo + 3 * p, *hp = hi + 3 * p;
    double* out = trp[c];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        int nu1 = e % k, nu = e / k;
        int a0 = nu1 % m, a1 = (nu1 / m) % m, a2 = nu1 / (m * m);
        int b0 = nu % m, b1 = (nu / m) % m, b2 = nu / (m * m);
        double x0 = cheb_node(lc[0], hc[0], a0, m), x1 = cheb_node(lc[1], hc[1], a1, m),
               x2 = cheb_node(lc[2], hc[2], a2, m);
        out[nu1 + (size_t)nu * k] =
            lagrange(lp[0], hp[0], m, b0, x0) * lagrange(lp[1], hp[1], m, b1, x1) * lagrange(lp[2], hp[2], m, b2, x2);
    }
}

void launch_interp_transfer(const double* lo, const double* hi, double* const* trp, int nc, int m, cudaStream_t st) {
    if (nc > 1) k_interp_transfer<<<nc - 1, 256, 0, st>>>(lo, hi, trp, m);
}

// couplings: S_ts[nu, mu] = g(xi_{t,nu}, xi_{s,mu}), one block per admissible block
__global__ void k_interp_coupling(const double* lo, const double* hi, const int* bt, const int* bs,
                                  double* const* bp, int m, int kernel) {
    const int b = blockIdx.x, t = bt[b], s = bs[b];
    const int k = m * m * m;
    const double *lt = lo + 3 * t, *ht = hi + 3 * t, *ls = lo + 3 * s, *hs = hi + 3 * s;
    double* out = bp[b];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        int nu = e % k, mu = e / k;
        double x[3] = {cheb_node(lt[0], ht[0], nu % m, m), cheb_node(lt[1], ht[1], (nu / m) % m, m),
                       cheb_node(lt[2], ht[2], nu / (m * m), m)};
        double y[3] = {cheb_node(ls[0], hs[0], mu % m, m), cheb_node(ls[1], hs[1], (mu / m) % m, m),
                       cheb_node(ls[2], hs[2], mu / (m * m), m)};
        out[nu + (size_t)mu * k] = kernel_eval(kernel, x, y);
    }
}

void launch_interp_coupling(const double* lo, const double* hi, const int* bt, const int* bs, double* const* bp,
                            int nblocks, int m, int kernel, cudaStream_t st) {
    if (nblocks > 0) k_interp_coupling<<<nblocks, 256, 0, st>>>(lo, hi, bt, bs, bp, m, kernel);
}

// dense blocks: N_ts[i, j] = g(x_i, x_j)
__global__ void k_interp_dense(const double* pts, const int64_t* perm, const int64_t* off, const int64_t* size,
                               const int* bt, const int* bs, double* const* bp, int kernel) {
    const int b = blockIdx.x, t = bt[b], s = bs[b];
    const int64_t mt = size[t], ms = size[s];
    double* out = bp[b];
    for (int64_t e = threadIdx.x; e < mt * ms; e += blockDim.x) {
        int64_t i = e % mt, j = e / mt;
        out[e] = kernel_eval(kernel, pts + 3 * perm[off[t] + i], pts + 3 * perm[off[s] + j]);
    }
}

void launch_interp_dense(const double* pts, const int64_t* perm, const int64_t* off, const int64_t* size,
                         const int* bt, const int* bs, double* const* bp, int nblocks, int kernel, cudaStream_t st) {
    if (nblocks > 0) k_interp_dense<<<nblocks, 256, 0, st>>>(pts, perm, off, size, bt, bs, bp, kernel);
}

// ------------------------------------------------------------------ block norms
__global__ void k_sumsq(const SumSqJob* __restrict__ jobs, double* out) {
    __shared__ double red[256 / 32];
    const SumSqJob J = jobs[blockIdx.x];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)J.rows * J.cols; e += 256) {
        double v = J.A[(e % J.rows) + (size_t)(e / J.rows) * J.lda];
        s += v * v;
    }
    s = block_sum<256>(s, red);
    if (threadIdx.x == 0) atomicAdd(out + J.slot, s);
}

void launch_sumsq(const SumSqJob* jobs, int njobs, double* out, cudaStream_t st) {
    if (njobs > 0) k_sumsq<<<njobs, 256, 0, st>>>(jobs, out);
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
