/*
 * lrspike.h -- C ABI of the GB300-native Low-Rank SPIKE (LR-SPIKE) solver.
 *
 * Solves banded systems A x = f (and A^T x = h) with the LR-SPIKE scheme of
 * Spring, Polizzi and Sameh, "Low-Rank SPIKE Framework for Solving Large Sparse
 * Linear Systems with Applications" (arXiv 2504.11167):
 *   - A is n x n with half-bandwidth k on both sides (section 2.1, "SPIKE
 *     partitioning": a matrix with unequal bandwidths uses the larger one);
 *   - it is split into p diagonal blocks A_i of roughly equal size n_i > k,
 *     coupled by k x k blocks B_i (last k rows of partition i, first k columns
 *     of partition i+1) and C_i (first k rows of partition i, last k columns of
 *     partition i-1) (section 2.1, block-tridiagonal partition);
 *   - factor: banded LU of every A_i, the spikes T_i = A_i^{-1}[0; B_i] and
 *     W_i = A_i^{-1}[C_i; 0] (section 2.1, eq. 'Veqn') compressed to rank r
 *     (the paper's n_svd, section 3.1), and the reduced system in the
 *     compressed unknowns (section 3.2);
 *   - solve: D-stage g = D^{-1} f, reduced solve, low-rank recovery
 *     (section 2.1 solve summary; section 3.3 table 'solver-list'), used as
 *     the preconditioner of an FP64 outer iteration.
 *
 * Every compute step runs in CUDA kernels of this library on one GPU.  No call
 * throws or aborts: each returns an lrspike_status, and lrspike_last_error()
 * gives a detail string.  A handle is not thread-safe; distinct handles are
 * independent.  All work of a handle is ordered on the CUDA stream given to
 * lrspike_create (NULL = the legacy default stream).
 *
 * Band storage (all entry points): diagonal-major, 2k+1 rows of length ld >= n,
 *   band[(k + i - j) * ld + j] = A[i][j]   for |i - j| <= k,
 * entries that fall outside the matrix are ignored.  Vectors are column-major
 * n x nrhs with leading dimension ld >= n, FP64.
 */
#ifndef LRSPIKE_H
#define LRSPIKE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrspike_ctx *lrspike_handle; /* opaque; owned by the library */

typedef enum {
    LRSPIKE_OK = 0,
    LRSPIKE_ERR_INVALID_ARG = 1,   /* bad option, size or pointer                 */
    LRSPIKE_ERR_STATE = 2,         /* e.g. solve before a successful factor        */
    LRSPIKE_ERR_OOM = 3,           /* device or pinned host allocation failed      */
    LRSPIKE_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed  */
    LRSPIKE_ERR_SINGULAR = 5,      /* zero or non-finite pivot (row in last_error) */
    LRSPIKE_ERR_NOT_CONVERGED = 6, /* outer iteration hit max_iter or stagnated    */
    LRSPIKE_ERR_UNSUPPORTED = 7    /* option combination not built                 */
} lrspike_status;

/* Working precision of the preconditioner (factors, spikes, D-stage,
 * retrieval).  The residual f - A x, the reduced system and the solution
 * update are always FP64 (the single-precision preconditioner inside a
 * double-precision solve of section 4).  MIXED_TF32: as MIXED_FP32 with the
 * block products of the band LU on the tensor cores (TF32 operands, FP32
 * accumulation; the triangular base blocks stay FP32); for k > 64 every block
 * product of the factorisation and the spike compression (tcgen05, FP32
 * accumulator).  MIXED_BF16 (k > 64 only): those block products take BF16
 * operands (rounded to nearest even from the FP32 values), FP32 accumulation;
 * the D-stage streams the BF16 copies of the factor tiles (half the bytes)
 * and accumulates in FP32. */
enum { LRSPIKE_FP64 = 0, LRSPIKE_MIXED_FP32 = 1, LRSPIKE_MIXED_TF32 = 2, LRSPIKE_MIXED_BF16 = 3 };
/* Compression of the spikes (section 3.1): SPIKE = truncated SVD of the
 * explicit spikes T_i, W_i (the paper's choice, optimal by Eckart-Young);
 * COUPLING = truncated SVD of B_i, C_i, then r-column solves (the cheaper
 * alternative the paper compares against). */
enum { LRSPIKE_COMPRESS_SPIKE = 0, LRSPIKE_COMPRESS_COUPLING = 1 };
/* Reduced system (section 3.3, table 'solver-list'): FULL = the low-rank
 * reduced system of LR-SPIKE-I, solved directly; TRUNCATED = its truncated
 * block-diagonal form S~~_r of LR-SPIKE-T (eq. 'red_sys_prec_mid_2');
 * OTF = LR-SPIKE-OTF (section 2.2 "SPIKE-on-the-fly", eqs. OTF-1/OTF-2;
 * section 3.3): the TRUE reduced system on the interface tips
 * [x_{i,b}; x_{i+1,t}] (2k per interface), solved by right-preconditioned
 * BiCGStab to otf_tol, its spike products formed on the fly by solves with
 * the partitions (one D-stage per product), preconditioned by S~~_r; then
 * x = g - D^{-1}[C_i x_{i-1,b}; 0; B_i x_{i+1,t}].  Each application of the
 * solver (the outer loop's correction) is one such solve, so one outer step
 * gives the solution to about otf_tol.  Factorised like TRUNCATED.  Built
 * without pivoting (k <= 1024; wide bands run every solve on the wide-band
 * factors), outer IR or NONE, not graph_safe;
 * solve_transpose uses the TRUNCATED preconditioner.  Extra device memory:
 * FP64 n x max_nrhs, working precision n x max_nrhs, 10 x 2k(p-1) x max_nrhs
 * FP64. */
enum { LRSPIKE_REDUCED_FULL = 0, LRSPIKE_REDUCED_TRUNCATED = 1, LRSPIKE_REDUCED_OTF = 2 };
/* Outer iteration: IR = iterative refinement x += M^{-1}(f - A x); with
 * k <= 64, no pivoting, not OTF, not graph_safe and every partition holding
 * >= 256 + 2k rows, the handle allocates one extra FP64 vector of n at create
 * and a one-RHS solve forms each correction's retrieval inside the next
 * residual kernel, the iterate alternating between x and that vector (x holds
 * the result on return; the arithmetic is that of the separate kernels);
 * BICGSTAB = right-preconditioned BiCGStab (the paper's outer solver, section
 * 4), FP64 vectors and scalars, one iteration = two applications of M^{-1};
 * each column stops when its residual meets tol, and convergence is confirmed
 * with the true residual f - A x (a column whose recurrence drifted is
 * restarted from it while iterations remain).  BiCGStab allocates 8 extra
 * FP64 vectors of n x max_nrhs at create;
 * NONE = one application x = M^{-1} f (the preconditioner alone). */
enum { LRSPIKE_OUTER_IR = 0, LRSPIKE_OUTER_BICGSTAB = 1, LRSPIKE_OUTER_NONE = 2 };

typedef struct {
    int64_t n;            /* matrix order, n >= 1                                    */
    int32_t k;            /* half-bandwidth, 0 <= k <= 1024 (k > 64: wide-band path) */
    int32_t p;            /* partitions, 1 <= p, every n_i > k when p > 1           */
    int32_t r;            /* compression rank n_svd, 0 <= r <= k                     */
    int32_t precision;    /* LRSPIKE_FP64 | LRSPIKE_MIXED_FP32 | _TF32 | _BF16       */
    int32_t pivoting;     /* 0 = none; 1 = partial pivoting inside each partition   */
    int32_t compress;     /* LRSPIKE_COMPRESS_*                                      */
    int32_t reduced;      /* LRSPIKE_REDUCED_*                                       */
    int32_t outer;        /* LRSPIKE_OUTER_*                                         */
    int32_t max_iter;     /* outer iteration limit (default 50)                      */
    double tol;           /* per-column ||f - A x||_2 / ||f||_2 target
                             (default 1e-12 for FP64, 1e-10 for mixed)               */
    double rank_tol;      /* singular values <= rank_tol * sigma_1 are dropped
                             (default 1e-13 FP64, 1e-6 mixed)                        */
    int32_t max_nrhs;     /* largest nrhs a solve may pass (default 16)              */
    int32_t profile;      /* 1 = time every kernel with CUDA events (see below)     */
    /* Wide bands (k > 64) truncate the spikes with the randomized SVD the paper
     * uses (section 3.1, Halko-Martinsson-Tropp proto-algorithm on the spike
     * T: Y = T Omega, orthonormal basis Q, power_iters passes Y = T (T^T Q),
     * SVD of Q^T T): ell = min(k, r + oversample) sketch columns (ell <= 64 in
     * FP64, <= 128 in the mixed modes), Gaussian sketches from SplitMix64 +
     * Box-Muller at counter a*ell + j with seed + 2 i + side (partition i,
     * side 0 = T_i, 1 = W_i); the basis by shifted CholeskyQR3.  Ignored for
     * k <= 64 (exact SVD). */
    int32_t oversample;   /* default r                                               */
    int32_t power_iters;  /* default 2                                               */
    uint64_t seed;        /* default 0x4C52535049                                    */
    /* graph_safe = 1: factor and solve only enqueue work on the handle's stream
     * (no host synchronisation, no host reads, no allocation), so a caller can
     * capture them in a CUDA graph and replay it.  The solve then enqueues
     * max_iter refinement steps (IR; NONE is one application) and leaves the
     * final residual on the device; lrspike_finish reports the outcome.  With
     * IR, the residual that meets tol for every column sets a device flag and
     * the kernels of the remaining enqueued steps return at entry (x and the
     * residual norms stay those of the converged step).
     * Requires device buffers, outer IR or NONE, profile 0, k <= 64. */
    int32_t graph_safe;
    /* block: the block size KB (8, 16, 32 or 64, >= the smallest block that
     * holds k; 0 = that smallest block).  A tuning knob for k <= 64. */
    int32_t block;
    /* reduced = OTF: relative residual target of the reduced BiCGStab in each
     * solve (default 1e-8, the paper's default) and its iteration limit
     * (default 100; the last iterate is used when it is reached). */
    double otf_tol;
    int32_t otf_max_iter;
} lrspike_options;

typedef struct {
    int32_t iterations;       /* outer iterations done (BiCGStab: full iterations)     */
    int32_t converged;        /* 1 if every column met tol                             */
    double max_rel_residual;  /* worst column's final ||f - A x|| / ||f||              */
    double *rel_residual;     /* caller-owned host array of >= nrhs entries, or NULL   */
    int32_t reduced_iterations; /* reduced = OTF: reduced BiCGStab iterations, all outer steps */
} lrspike_info;

/* Fills *opt with defaults for n, k, p, r (FP64, no pivoting, SPIKE
 * compression, FULL reduced system, IR).  Returns INVALID_ARG on NULL. */
lrspike_status lrspike_options_default(lrspike_options *opt, int64_t n, int32_t k, int32_t p,
                                       int32_t r);

/* Validates *opt, allocates every device workspace the handle needs (sized by
 * n, k, p, r, precision and max_nrhs) and returns the handle in *out.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream), borrowed.
 * k <= 64 uses blocks of KB in {8, 16, 32, 64} >= k and the hand-written
 * block kernels; 64 < k <= 1024 (wide bands) uses blocks of W = 64 ceil(k/64)
 * whose products are batched over the partitions: on the tensor cores
 * (tcgen05; TF32 or BF16 operands, FP32 accumulation) in the MIXED_TF32 and
 * MIXED_BF16 modes, as SIMT GEMMs in the working precision in the FP64 and
 * MIXED_FP32 modes; SPIKE compression, no pivoting, sketch width
 * min(k, r + oversample) <= 64 (FP64) or <= 128 (mixed modes).  r <= 32,
 * or r <= 64 for wide bands with the TRUNCATED reduced system.  The wide-band
 * D-stage runs one cluster of CTAs per partition (at most 8).
 * COUPLING compression with k <= 64, p > 1 and r > 0: the handle also owns a
 * second, non-blocking stream and two events; lrspike_factor runs the
 * coupling blocks' Gram matrices, eigenvectors and spike right-hand sides on
 * it beside the band LU, forked from and joined back into cuda_stream (work
 * after the factor call on cuda_stream sees all of it; under stream capture
 * the fork and join become graph edges).
 * Errors: INVALID_ARG (n < 1, k < 0 or k > 1024, r < 0 or r > k, p < 1,
 * n_i <= k with p > 1, max_nrhs < 1, unknown enum), UNSUPPORTED, OOM, CUDA. */
lrspike_status lrspike_create(const lrspike_options *opt, void *cuda_stream, lrspike_handle *out);

/* LR-SPIKE factorisation of the banded A.
 * band: (2k+1) x ld values as described above, FP64.  Device pointer: borrowed,
 * not copied -- the caller keeps it alive and unmodified until the next factor
 * or destroy, because every solve's FP64 residual reads it.  Host pointer
 * (pinned or pageable): copied into a device buffer owned by the handle; for
 * the unpivoted k <= 64 FP32 / FP64 factorisation with p >= 2 (and profile 0)
 * the copy runs on a further stream of the handle in min(p, 16) partition groups (the
 * columns around every interface first) and each group's band LU starts when
 * its columns have landed; the call returns after the factorisation, so the
 * host buffer may be reused at once.
 * Errors: INVALID_ARG (NULL, ld < n), SINGULAR (a zero or non-finite pivot in
 * some A_i; the global row is in lrspike_last_error), CUDA. */
lrspike_status lrspike_factor(lrspike_handle h, const double *band, int64_t ld);

/* Solves A x = f to the handle's tolerance with the chosen outer iteration.
 * f, x: n x nrhs column-major FP64 with leading dimension ld >= n, both on the
 * device or both on the host (host buffers are copied in and out); x must not
 * alias f.  1 <= nrhs <= max_nrhs.  info may be NULL.
 * Errors: STATE (no successful factor), INVALID_ARG, NOT_CONVERGED (x holds
 * the last iterate; IR: max_iter reached or the residual stagnated; BiCGStab:
 * max_iter reached or a breakdown, a zero or non-finite scalar), CUDA. */
lrspike_status lrspike_solve(lrspike_handle h, const double *f, double *x, int32_t nrhs,
                             int64_t ld, lrspike_info *info);

/* Solves A^T lambda = h with the same factors: the outer iteration uses the
 * transposed preconditioner M^{-T} = D^{-T}(I - V^T R^{-T} U^T), the
 * transpose of M^{-1} = (I - U R^{-1} V) D^{-1}.  Arguments as lrspike_solve. */
lrspike_status lrspike_solve_transpose(lrspike_handle hd, const double *h, double *lambda,
                                       int32_t nrhs, int64_t ld, lrspike_info *info);

/* For a graph_safe handle: waits for the handle's stream and reports the last
 * factorisation (SINGULAR as lrspike_factor would) and the last solve (info as
 * lrspike_solve fills it: iterations = the refinement steps that ran before
 * the residual met tol (max_iter if it never did; 1 for NONE), the per-column
 * relative residual of the final iterate; NOT_CONVERGED if a column is above
 * tol).
 * STATE if nothing was solved since the last factor. */
lrspike_status lrspike_finish(lrspike_handle h, lrspike_info *info);

/* Releases the handle and every buffer it owns.  NULL is accepted. */
lrspike_status lrspike_destroy(lrspike_handle h);

/* Detail string of the handle's last error ("" if none); owned by the handle,
 * valid until its next call.  With h == NULL: the last error of a call that
 * had no handle (create). */
const char *lrspike_last_error(lrspike_handle h);

/* ---- introspection (profiling and tests) ------------------------------ */

/* Number of kernel launches this handle has issued since create (all
 * kernels of the library; reset by lrspike_profile_reset). */
int64_t lrspike_launch_count(lrspike_handle h);

/* With opt.profile = 1 every kernel launch is bracketed by CUDA events on the
 * handle's stream.  lrspike_profile_get returns, for kernel id 0..count-1,
 * its name, its launches and the summed event time in ms (synchronises the
 * stream).  Returns INVALID_ARG past the last id. */
lrspike_status lrspike_profile_get(lrspike_handle h, int32_t id, const char **name,
                                   int64_t *launches, double *total_ms);
lrspike_status lrspike_profile_reset(lrspike_handle h);

/* Copies the device arrays of the compressed reduced system to host buffers
 * (any may be NULL): sigma (p x 2 x r singular values of T_i / W_i, zero where
 * dropped or absent) and R (2r(p-1) squared, row-major, the matrix that is
 * solved).  Used by the tests to compare the compression with the oracle. */
lrspike_status lrspike_get_reduced(lrspike_handle h, double *sigma, double *R);

/* ---- allocation-free band residual ----------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code running inside a latency-critical
 * serving loop, where a cudaMalloc would synchronise the whole device and
 * stall its other streams, or a host framework that owns all device memory
 * through its own pool and forbids stray allocations.  It needs no handle
 * (creating one allocates) and calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Computes r = f - A x in FP64 from the band (layout as above) and the 2-norm
 * of every column of r, with the same kernel and the same deterministic
 * reduction order that lrspike_solve uses for its convergence test.
 *   band  (2k+1) x ld_band, device; f, x: n x nrhs column-major with leading
 *   dimension ld >= n, device; r: device, n x nrhs column-major with leading
 *   dimension n (column q at r + q*n); norms: device, nrhs doubles.
 *   1 <= nrhs <= 16.  Enqueued on cuda_stream (NULL = legacy default stream);
 *   the call returns without waiting for the GPU.
 * Its scratch (one partial sum per 256 rows and column, and a counter) is a
 * fixed static device array of LRSPIKE_NOALLOC_MAX_PARTIALS doubles that every
 * GPU loading the library holds until the process exits: sizes with
 * ceil(n/256) * nrhs > LRSPIKE_NOALLOC_MAX_PARTIALS are rejected with
 * INVALID_ARG.  The first call on each device looks up that device's address of
 * the array (with the device current); make that first call before any stream
 * capture.  All calls on a device share the array, so calls that overlap on the
 * GPU (other streams or host threads) race and must be serialised by the
 * caller.  Errors (INVALID_ARG for NULL, host or oversized arguments, CUDA) are
 * described by lrspike_last_error(NULL). */
#define LRSPIKE_NOALLOC_MAX_PARTIALS 65536
lrspike_status lrspike_residual_noalloc(const double *band, int64_t ld_band, int64_t n, int32_t k,
                                        const double *f, const double *x, double *r, int32_t nrhs,
                                        int64_t ld, double *norms, void *cuda_stream);

/* ---- gradient of the band ------------------------------------------------
 * For x = A^{-1} f and a loss L(x), the adjoint solve A^T lambda = dL/dx
 * (lrspike_solve_transpose with the stored factors) gives dL/df = lambda and
 * dL/dA = -lambda x^T; only the entries inside the band are parameters of A.
 * This entry point writes that band-restricted outer product:
 *   grad_band[(k + i - j) ld_band + j] = alpha * sum_q lam_q[i] x_q[j]
 * for every |i - j| <= k inside the matrix (alpha = -1 gives dL/dA), and 0 at
 * the band positions outside the matrix.  lam, x: device, n x nrhs
 * column-major, leading dimension ld >= n; grad_band: device, (2k+1) x
 * ld_band, ld_band >= n.  1 <= nrhs <= 16, 0 <= k <= 1024.  Enqueued on
 * cuda_stream (NULL = legacy default stream); no allocation, no handle.
 * Errors (INVALID_ARG for NULL, host pointers or bad sizes, CUDA) are
 * described by lrspike_last_error(NULL). */
lrspike_status lrspike_band_outer(const double *lam, const double *x, int32_t nrhs, int64_t ld, int64_t n,
                                  int32_t k, double alpha, double *grad_band, int64_t ld_band,
                                  void *cuda_stream);

/* ---- FP64 rate of the current GPU ------------------------------------------
 * The paper has no counterpart to this entry point; it measures what bounds
 * the FP64 residual r = f - A x (one FMA per band entry) on GPUs whose FP64
 * units are scarce.  One kernel of independent FMA chains on every SM, iters
 * iterations of 16 chains per thread, timed with CUDA events on cuda_stream
 * (NULL = legacy default stream); the call waits for it.  *tflops receives
 * 2 x FMAs / elapsed time in TFLOP/s.  Errors (INVALID_ARG for iters < 1 or
 * a NULL output, CUDA) are described by lrspike_last_error(NULL). */
lrspike_status lrspike_fp64_fma_probe(int64_t iters, double *tflops, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LRSPIKE_H */
