/*
 * h2mul.h -- C-ABI of the GB300 (sm_103a) adaptive H^2-matrix product.
 *
 * The library computes Z <- Z + X Y for H^2-matrices X, Y, Z (S. Boerm,
 * "Adaptive fast multiplication of H^2-matrices", arXiv 2309.09061, Sec. 1:
 * the product in the general form Z <- Z + XY).  It first builds compressed
 * induced row and column bases and the product on the refined block tree
 * T^XY (Sec. 4-5), then coarsens that representation to Z's block tree with
 * new adaptive, nested, isometric cluster bases (Sec. 6).
 *
 * Conventions for every entry point:
 *   - Return value 0 (H2_OK) on success, a negative H2_ERR_* code on failure;
 *     h2_error_string() names the code.  No entry point aborts the process.
 *   - Dense matrices are column-major doubles with a leading dimension.
 *   - A handle (h2_matrix*) owns all of its device buffers; h2_free releases
 *     them.  Handles live on the CUDA device that was current when they were
 *     created; every call must be made with that device current.
 *   - `opts` may be NULL (defaults: eps = 1e-6, H2_FP64, legacy default
 *     stream, no statistics).  Work is issued on opts->stream; every entry
 *     point returns after that stream has finished the call's work.
 */
#ifndef H2MUL_H
#define H2MUL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define H2_API __attribute__((visibility("default")))
#else
#define H2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define H2_OK 0
#define H2_ERR_ARG (-1)         /* invalid argument (NULL pointer, bad size, bad enum) */
#define H2_ERR_SHAPE (-2)       /* operands do not share one cluster tree / block tree */
#define H2_ERR_OOM (-3)         /* device or host allocation failed */
#define H2_ERR_NUMERIC (-4)     /* NaN or Inf met in an input or an intermediate */
#define H2_ERR_TIMEOUT (-5)     /* an iterative device routine ran out of its bounded sweeps */
#define H2_ERR_UNSUPPORTED (-6) /* a case outside the supported operand relations */
#define H2_ERR_CUDA (-7)        /* a CUDA runtime call failed */

/* Kernel functions g(x, y) for h2_build_interp (Sec. 7 and the workloads):
 *   H2_K_LAPLACE  1 / (4 pi |x - y|), 0 on coinciding points
 *   H2_K_YUKAWA   exp(-|x - y|) / |x - y|, 0 on coinciding points
 *   H2_K_POLY2    (1 + x.y)^2      (degree 2 per coordinate: interpolated exactly for order >= 3)
 *   H2_K_CONST    1                (the all-ones matrix)
 *   H2_K_DELTA    1 if x == y else 0 (the identity matrix for distinct points)
 *   H2_K_DLP      <n(y), x - y> / (4 pi |x - y|^3), 0 on coinciding points: the
 *                 double-layer potential of the Laplace kernel (the second operator
 *                 of Sec. 7, as point collocation); needs a normal n(y) per point
 *                 (h2_build_interp_normals), and gives V != W. */
#define H2_K_LAPLACE 0
#define H2_K_YUKAWA 1
#define H2_K_POLY2 2
#define H2_K_CONST 3
#define H2_K_DELTA 4
#define H2_K_DLP 5

/* Precision of the contractions (products of coupling, transfer, basis and
 * auxiliary matrices).  QR factorisations, singular value decompositions and
 * the choice of ranks always run in FP64.
 *   H2_FP64    every product in FP64 (the plain FP64 GPU form)
 *   H2_MIXED   products in FP32 with FP32 accumulation on the CUDA cores
 *   H2_TF32X3  products on the tensor cores (tcgen05.mma kind::tf32): each FP32
 *              operand split as a0 + a1 into two TF32 pieces, three products
 *              a0 b0 + a0 b1 + a1 b0 accumulated in FP32 in TMEM (about FP32
 *              accuracy); H2_TC is the same value
 *   H2_TF32    one TF32 product a0 b0 per pair (operand rounding 2^-12: the
 *              products are off by about 5e-4 relative; for eps >= 1e-3)
 *   H2_BF16X3  tensor cores with BF16 pieces (tcgen05.mma kind::f16): a0 + a1
 *              with 8 significant bits each, three products (about 2^-17 on
 *              the whole, single blocks up to 3e-5; for eps >= 1e-4)
 *   H2_AUTO    chosen by eps: H2_TF32 for eps >= 1e-3, H2_BF16X3 for
 *              1e-4 <= eps < 1e-3, H2_TF32X3 below 1e-4 (three-term products
 *              wherever eps < 1e-5), H2_FP64 for eps < 1e-7 (exact mode
 *              included)
 * In every mode but H2_FP64 the wide-to-square reduction ahead of each SVD
 * runs in FP32 and FP32 sweeps precondition the FP64 Jacobi sweeps; the
 * weights' Gram matrices and the other products that must be FP64-accurate
 * run in double-float FP32 arithmetic, and the pivoted Cholesky, the final
 * sweeps and every rank decision stay FP64.  With the default schedules
 * (h2_opts.autotune = 0) a product gives the same bits on every run: no
 * reduction depends on the order in which CTAs finish. */
#define H2_FP64 0
#define H2_MIXED 1
#define H2_TF32X3 2
#define H2_TC H2_TF32X3
#define H2_TF32 3
#define H2_BF16X3 4
#define H2_AUTO 5

typedef struct h2_matrix h2_matrix;

/* Per-call statistics, filled when opts->stats is not NULL. Times are device
 * times between CUDA events on opts->stream, in milliseconds. */
typedef struct {
    double t_prep_ms;      /* basis products, basis weights, total weights */
    double t_rows_a_ms;    /* compressed induced row basis (Fig. 4) */
    double t_cols_a_ms;    /* compressed induced column basis */
    double t_mat_a_ms;     /* H^2-matrix on T^XY in the induced bases */
    double t_rows_b_ms;    /* coarsened row basis (Fig. 7) */
    double t_cols_b_ms;    /* coarsened column basis */
    double t_mat_b_ms;     /* final couplings on the target block tree */
    double t_total_ms;     /* the whole call, host synchronisations included */
    int64_t kernel_launches; /* kernels launched by the call */
    int64_t product_nodes;   /* nodes of T^XY */
    int64_t triples;         /* (t,s,r) contributions to T^XY couplings */
    int max_rank_a;          /* largest rank of the induced bases */
    int max_rank_b;          /* largest rank of the final bases */
    double bytes_moved;      /* algorithmic bytes of the contractions (model) */
    double flops;            /* algorithmic flops of the contractions (model) */
    /* Per kernel family (index H2_FAM_*): device time of all launches (sum of
     * CUDA-event intervals around each launch on opts->stream), number of
     * launches, algorithmic flops and bytes (every operand read once, every
     * output written once; counted on the host from the launch descriptors). */
    double fam_ms[12];
    int64_t fam_launches[12];
    double fam_flops[12];
    double fam_bytes[12];
} h2_stats;

/* Kernel families of h2_stats.fam_*. */
#define H2_FAM_GEMM64 0  /* batched segmented products, FP64 arithmetic */
#define H2_FAM_GEMM32 1  /* batched segmented products, FP32 arithmetic */
#define H2_FAM_QR64 2    /* Householder QR, FP64 */
#define H2_FAM_QR32 3    /* Householder QR, FP32 (wide-to-square reductions, mixed mode) */
#define H2_FAM_CHOL 4    /* pivoted Cholesky of weight Gram matrices */
#define H2_FAM_SVD 5     /* one-sided Jacobi SVD, FP64 sweeps */
#define H2_FAM_SVDPRE 6  /* one-sided Jacobi preconditioning, FP32 sweeps */
#define H2_FAM_NORM 7    /* spectral norms by power iteration */
#define H2_FAM_COPY 8    /* batched copies, scalings, transpositions */
#define H2_FAM_OTHER 9   /* block norms, finiteness checks */
#define H2_FAM_GEMMTC 10 /* batched segmented products on tcgen05 (H2_TC) */
#define H2_FAM_GEMMDF 11 /* FP64-accurate products of H2_MIXED / H2_TC in double-float FP32 arithmetic */

/* Device memory supplied by the caller.  alloc(bytes, stream, ctx) returns a
 * device pointer on the current device, aligned to at least 256 bytes, usable
 * by work issued on `stream` (or NULL when out of memory); free(ptr, bytes,
 * stream, ctx) returns it with stream-ordered semantics: work issued on
 * `stream` after the call may reuse the memory, and the library issues no
 * later work on it.  `stream` is the stream the buffer was allocated for: the
 * call's opts->stream, or one of the library's internal streams (the column
 * side of a product, the products of h2_mul_add_batched). */
typedef void* (*h2_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*h2_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct {
    double eps;       /* relative truncation tolerance; 0 keeps every nonzero singular value */
    int precision;    /* H2_FP64, H2_MIXED, H2_TF32X3 (= H2_TC), H2_TF32, H2_BF16X3 or H2_AUTO */
    void* stream;     /* cudaStream_t; NULL selects the legacy default stream */
    h2_stats* stats;  /* optional output, may be NULL */
    /* Device memory.  alloc == NULL: the library allocates (cudaMalloc for the
     * buffers of handles, its own stream-ordered pool for scratch).  Otherwise
     * every device buffer of the call -- scratch and the buffers of the handles
     * it creates or rebuilds -- comes from alloc and goes back through free
     * (both required).  A handle remembers the callbacks its buffers came from
     * and returns them through the same free in h2_free, or when a later call
     * replaces them; alloc_ctx must stay valid until then. */
    h2_alloc_fn alloc;
    h2_free_fn free;
    void* alloc_ctx;
    /* Nonzero: the library tunes its launch schedules online.  Each batch of
     * products is keyed by (kernel family, number of output tiles, K per
     * tile); the first batches of a key run the candidate schedules in turn
     * (for the FP32-class products the mode's kernel or the other one --
     * CUDA-core FP32 against the tensor cores, at least as accurate -- with
     * split-K by the default rule or off; for the others split-K by the
     * default rule, off, or over 2 or 4 slices), their device times are read
     * when the call ends, and later batches of the key run the fastest.  The
     * choices are kept per device for the life of the process.  Every
     * candidate computes the same products, so results agree to rounding.
     * Zero (the default schedules): in the tensor-core modes, a batch whose
     * jobs fit 64-row tiles runs on the CUDA-core FP32 kernel (faster there,
     * and at least as accurate), wider jobs on the tensor cores; split-K by
     * the default rule (when a batch would not fill the GPU). */
    int autotune;
} h2_opts;

/* Structure and sizes of a handle (h2_info). */
typedef struct {
    int64_t n;          /* number of points (rows = columns) */
    int depth;          /* depth L of the cluster tree; all leaves sit on level L */
    int nclusters;      /* 2^(L+1) - 1, numbered level by level (heap order) */
    int64_t nblocks;    /* nodes of the block tree */
    int64_t nadmissible;/* admissible leaves (coupling matrices) */
    int64_t ndense;     /* inadmissible leaves (dense blocks) */
    int leaf_size;
    int order;          /* Chebyshev order m of the input bases (rank m^3), 0 after a product */
    double eta;
    int max_row_rank;
    int max_col_rank;
    double device_bytes;/* device memory held by the handle */
} h2_info_t;

/* Build the H^2-matrix of g(x_i, x_j) by tensor Chebyshev interpolation of
 * order `cheb_order` (rank cheb_order^3), Sec. 2, Example "Integral operator"
 * (point evaluation in place of the Galerkin integrals):
 *   V_t[i, nu] = l_{t,nu}(x_i) on leaves, E_t'[nu', nu] = l_{t,nu}(xi_{t',nu'}),
 *   S_ts[nu, mu] = g(xi_{t,nu}, xi_{s,mu}), dense N_ts[i, j] = g(x_i, x_j).
 * The cluster tree is a median bisection along the longest box axis down to
 * the depth L where every cluster holds at most `leaf_size` points; the block
 * tree uses max(diam B_t, diam B_s) <= eta dist(B_t, B_s) (Def. "Block tree").
 *   points      n x 3, row-major (x0 y0 z0 x1 ...), in host memory or in
 *               device memory of the current device (the library tells them
 *               apart with cudaPointerGetAttributes); read only, copied to the
 *               host for the tree construction (it runs on the host); owned by
 *               the caller.
 *   n >= 1, 1 <= leaf_size, 1 <= cheb_order <= 8, eta >= 0, kernel H2_K_*.
 *   out         receives the new handle; untouched on error.
 * Errors: H2_ERR_ARG (H2_K_DLP needs h2_build_interp_normals), H2_ERR_NUMERIC
 * (non-finite point), H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_build_interp(const double* points, int64_t n, int kernel, int leaf_size, double eta,
                    int cheb_order, const h2_opts* opts, h2_matrix** out);

/* h2_build_interp with a unit normal per point (n x 3, row-major, same order
 * as `points`, host or device memory like `points`; read only, copied).  For H2_K_DLP the kernel is
 * interpolated as the normal derivative in y of 1 / (4 pi |x - y|): V is the
 * Lagrange basis, W the normal-derivative basis
 *   W_s[j, mu] = grad l_{s,mu}(y_j) . n(y_j) on leaves, with the Lagrange
 *   transfer matrices (differentiation is linear and the parent's polynomials
 *   are interpolated exactly),
 * S_ts = 1 / (4 pi |xi_{t,nu} - xi_{s,mu}|), dense N_ts[i, j] = g(x_i, x_j).
 * Other kernels ignore `normals` (it may be NULL for them).
 * Errors: as h2_build_interp; H2_ERR_ARG if H2_K_DLP and normals == NULL,
 * H2_ERR_NUMERIC for a non-finite normal. */
H2_API int h2_build_interp_normals(const double* points, const double* normals, int64_t n, int kernel,
                                   int leaf_size, double eta, int cheb_order, const h2_opts* opts,
                                   h2_matrix** out);

/* Z <- Z + X Y (Sec. 1), approximated to the block-relative tolerance
 * opts->eps in both phases (Sec. 5, Sec. 6, Sec. 7).  X, Y and Z must share
 * one cluster tree and block tree (built from the same points, leaf size and
 * eta); otherwise H2_ERR_SHAPE.  Z's bases are free: when Z's row basis is
 * not X's row basis (or Z's column basis not Y's column basis), for example
 * Z from an earlier product or of another Chebyshev order, it is preserved in
 * phase A beside V_X (W_Y), so that Z's couplings are represented in the new
 * bases.  The same handle may be passed as X, Y and Z.  On
 * success Z holds new adaptive bases and couplings on its own block tree; on
 * error Z is unchanged (the result is built aside and swapped in at the end).
 * X and Y are only read. */
H2_API int h2_mul_add(h2_matrix* Z, const h2_matrix* X, const h2_matrix* Y, const h2_opts* opts);

/* Z[i] <- Z[i] + X[i] Y[i] for count independent products (different sizes,
 * orders, geometries), each with the relations and semantics of h2_mul_add
 * and opts->eps / opts->precision.  The products run concurrently (up to 16
 * at a time, each on its own host thread and internal non-blocking stream)
 * after the work already issued on opts->stream; the call returns when all
 * of them are done.  With H2_BATCH_GROUPING=1 in the environment the
 * concurrent products' GEMM batches of the same kernel are grouped into
 * shared launches (up to 8 products at a time); results then agree with
 * those of single products to rounding, not bit for bit.  A Z handle may
 * not appear twice.  status (may be NULL) receives count per-product codes;
 * the return value is the first nonzero one (products that failed leave
 * their Z unchanged, the others are updated).  opts->stats receives sums over
 * the products (times are summed device times, not the elapsed time).
 * Errors: as h2_mul_add, plus H2_ERR_ARG when a Z handle appears twice or as
 * an operand of another product of the batch. */
H2_API int h2_mul_add_batched(h2_matrix* const* Z, const h2_matrix* const* X, const h2_matrix* const* Y, int count,
                              const h2_opts* opts, int* status);

/* Expand A into a dense n x n matrix in the ORIGINAL point order (row i and
 * column j belong to points i and j), column-major with leading dimension
 * ld >= n.  `out` is a host pointer if out_on_device == 0, else a device
 * pointer on the handle's device.  Meant for tests at small n (n^2 doubles).
 * Errors: H2_ERR_ARG, H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_to_dense(const h2_matrix* A, double* out, int64_t ld, int out_on_device, const h2_opts* opts);

/* y = A x (trans = 0) or y = A^* x (trans = 1) for nvec vectors: x and y are
 * device arrays of n x nvec doubles, column-major with leading dimension n,
 * rows in the ORIGINAL point order; x is read, y overwritten (no aliasing).
 * Forward transformation through the column basis, couplings, backward
 * transformation through the row basis and dense blocks (the O(nk)
 * H^2-matrix-vector product the paper relies on, Sec. 2).  Row i of A is
 * A^* e_i.  Errors: H2_ERR_ARG, H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_matvec(const h2_matrix* A, const double* x, double* y, int64_t nvec, int trans, const h2_opts* opts);

/* A <- A with adaptive isometric bases (recompression of an input, for
 * example a Chebyshev matrix whose rank m^3 exceeds what opts->eps needs).
 * The bases are orthogonalized (the QR factorisations of Fig. 1 with their
 * isometric factors kept: V = Q R), the couplings are moved into them
 * (S' = R_V,t S R_W,s^*), and the second phase of the product (Sec. 6:
 * coarsening, Fig. 7, and the final couplings) runs with A's own block tree
 * as the intermediate's tree, at the block-relative tolerance opts->eps
 * (0 keeps every nonzero singular value) and in opts->precision.  On error A
 * is unchanged.  Errors: H2_ERR_ARG, H2_ERR_NUMERIC, H2_ERR_TIMEOUT, H2_ERR_OOM,
 * H2_ERR_CUDA. */
H2_API int h2_recompress(h2_matrix* A, const h2_opts* opts);

/* Relative spectral error of a computed product (the eps_2 of Sec. 7):/* Relative spectral error of a computed product (the eps_2 of Sec. 7):
 *   *eps2 = ||Zr - (Z0 + X Y)||_2 / ||Z0 + X Y||_2,   *norm = ||Z0 + X Y||_2,
 * where Zr is the result of h2_mul_add on a copy of Z0 (for example a clone
 * taken before the call).  Each spectral norm is estimated by `steps` steps of
 * power iteration on the normal operator A^* A (Sec. 7 uses 20): x is
 * normalised, the estimate is ||A x|| of the last unit x, then x <- A^* A x.
 * Every application of A or A^* runs through h2_matvec of the four operands;
 * no dense matrix is formed.  x0 (host, n doubles in the ORIGINAL point order)
 * is the start vector; NULL selects x0_i = 1 + 0.37 i / n.  The estimates are
 * lower bounds that converge to the norms.  All four handles must share one
 * structure.  Errors: H2_ERR_ARG (NULL pointers, steps outside 1..100000),
 * H2_ERR_SHAPE (different structures), H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_product_error(const h2_matrix* Zr, const h2_matrix* Z0, const h2_matrix* X, const h2_matrix* Y,
                            const double* x0, int steps, const h2_opts* opts, double* eps2, double* norm);

/* Spectral norms of the blocks of A's block tree, computed on the device by
 * the power iteration that the product uses for its block weights (Sec. 5 and
 * Sec. 6: ranks are chosen relative to block norms).  For block b, 0 <= b <
 * nblocks (h2_info), in the order of the block tree:
 *   t[b], s[b]  its row and column clusters (indices as in h2_get_structure)
 *   kind[b]     0 admissible, 1 dense (inadmissible leaf), 2 split
 *   norm[b]     ||S_b||_2 of the coupling matrix of an admissible block
 *               (rank(t) x rank(s)), ||N_b||_2 of a dense block, 0 for a split
 *               block
 * opts->precision selects the iteration as in the product: H2_FP64 (or
 * H2_AUTO resolving to it) iterates in FP64 and stops when the estimate
 * changes by less than 1e-10 (relative), every other mode in FP32 and stops
 * at 1e-5; at most 60 steps from x_j = 1 + 0.37 j / n.  Each value is the
 * length of A_b x for the last unit vector x: a lower bound of the norm up to
 * rounding.  Any output pointer may be NULL (host arrays of nblocks entries).
 * Errors: H2_ERR_ARG, H2_ERR_UNSUPPORTED (a block wider than 2048),
 * H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_block_norms(const h2_matrix* A, const h2_opts* opts, int* t, int* s, int* kind, double* norm);

/* Sizes and structure of a handle.  Errors: H2_ERR_ARG. */
H2_API int h2_info(const h2_matrix* A, h2_info_t* info);

/* Copy structure arrays of a handle to host memory (any pointer may be NULL):
 *   perm        n entries: original index of the point at tree position p
 *   offsets     nclusters entries: first tree position of each cluster
 *   sizes       nclusters entries: number of points of each cluster
 *   row_ranks   nclusters entries: rank of the row basis per cluster
 *   col_ranks   nclusters entries: rank of the column basis per cluster
 * Errors: H2_ERR_ARG. */
H2_API int h2_get_structure(const h2_matrix* A, int64_t* perm, int64_t* offsets, int64_t* sizes,
                     int* row_ranks, int* col_ranks);

/* Deep copy of a handle (same structure, bases and blocks) on the same device;
 * the copy owns its own buffers.  Errors: H2_ERR_ARG, H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_clone(const h2_matrix* A, const h2_opts* opts, h2_matrix** out);

/* Host-only planning, no device call: the cluster tree and block tree that
 * h2_build_interp would build for these points (Def. "Cluster tree",
 * Def. "Block tree"), and the product block tree T^XY of a product of two
 * such matrices (Sec. 6).
 *   perm     n entries (may be NULL): original index at each tree position
 *   counts   8 entries (may be NULL): depth L, admissible, dense and split
 *            blocks of the block tree, admissible, dense and split nodes of
 *            T^XY, and the number of (t,s,r) triples contributing to T^XY.
 * Errors: H2_ERR_ARG (bad sizes), H2_ERR_NUMERIC (non-finite point). */
H2_API int h2_plan_structure(const double* points, int64_t n, int leaf_size, double eta, int64_t* perm,
                             int64_t* counts);

/* h2_to_dense without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while
 * they run -- for example code inside a stream whose memory is managed by
 * another allocator, or a real-time phase that forbids cudaMalloc/cudaFree --
 * but still need the dense expansion of a handle.
 * It writes the same result as h2_to_dense(A, out, ld, 1, ...): A expanded
 * into the n x n device matrix `out` (original point order, column-major,
 * ld >= n), issued on `stream` (a cudaStream_t, NULL for the legacy default
 * stream) and finished before the call returns.
 * Scratch: one fixed device array of 4 Mi doubles (32 MiB) in the library,
 * held on every GPU that loads the library until the process exits.  The
 * call needs n^2 + (the expanded cluster bases, about n x rank per level) +
 * (n x rank per admissible block row) doubles plus its descriptor arrays; it
 * measures them on the host first and rejects a matrix that does not fit with
 * H2_ERR_UNSUPPORTED before any device work is issued.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it (the lookup is
 * serialised between threads); make that first call before any stream
 * capture, and make no call on a device after a cudaDeviceReset of it.
 * Every call shares the array and it keeps the last call's contents (the
 * call clears what must start at zero), so calls that overlap on the GPU --
 * from several threads or streams -- race and must be serialised by the
 * caller.
 * Errors: H2_ERR_ARG, H2_ERR_UNSUPPORTED (too large), H2_ERR_CUDA. */
H2_API int h2_to_dense_noalloc(const h2_matrix* A, double* out, int64_t ld, void* stream);

/* Device memory the library holds from its own sources -- cudaMalloc for the
 * buffers of handles and its stream-ordered pool for scratch -- summed over
 * devices: the bytes held now and the most held at once since the library was
 * loaded or the peak was last reset (reset_peak != 0 sets it to the current
 * figure after reading it).  Memory from caller callbacks (h2_opts.alloc) is
 * not counted: with callbacks on every call, both figures stay at zero.  Any
 * pointer may be NULL.  Always H2_OK.  The paper has no counterpart; this is a
 * diagnostic of the allocation contract. */
H2_API int h2_library_memory(int64_t* current_bytes, int64_t* peak_bytes, int reset_peak);

/* Release a handle and its device memory; NULL is ignored.  Buffers from
 * caller callbacks (h2_opts.alloc) go back through the matching free; the
 * library's own buffers through cudaFree.  No wait is needed before: every
 * entry point returns after its work on the handle has finished. */
H2_API void h2_free(h2_matrix* A);

/* Static description of an error code. */
H2_API const char* h2_error_string(int code);

/* Message of the last failed call on the calling thread ("" if none); valid
 * until the next call on that thread. */
H2_API const char* h2_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* H2MUL_H */
