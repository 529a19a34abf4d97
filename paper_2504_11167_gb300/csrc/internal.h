// Internal state and launcher declarations of the LR-SPIKE CUDA library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lrspike.h"

namespace lrs {

enum KernelId {
    KID_LU = 0,
    KID_SPIKE_RHS,
    KID_SWEEP,
    KID_GRAM,
    KID_GRAM_REDUCE,
    KID_COUPLING_GRAM,
    KID_JACOBI,
    KID_MAKE_U,
    KID_RED_BUILD,
    KID_RED_FACTOR,
    KID_NORM,
    KID_RESIDUAL,
    KID_DSTAGE,
    KID_RED_SOLVE,
    KID_RETRIEVE,
    KID_PROJECT_T,
    KID_DSTAGE_T,
    KID_VEC,
    KID_MATVEC,
    KID_WIDE_GATHER,
    KID_WIDE_GEMM,
    KID_WIDE_LU64,
    KID_WIDE_VEC,
    KID_WIDE_TC,
    KID_WIDE_CHOLQR,
    KID_WIDE_DSTAGE,
    KID_DIAGS,
    KID_LU_INV,
    KID_OTF,
    KID_COUNT
};

extern const char *const kKernelNames[KID_COUNT];

struct Pending {
    int kid;
    cudaEvent_t a, b;
};

// One handle.  Device arrays typed void* hold the working precision T
// (double in FP64 mode, float in the mixed modes).
// Early exit of a graph-safe refinement (a fixed number of enqueued steps):
// the residual whose column norms all meet |r_j| <= tol |f_j| raises flag[0];
// while it is up every later kernel of the loop returns at entry.  flag[1]
// counts the residuals of the loop that found the tolerance unmet (= the
// preconditioner applications that ran).  flag == nullptr: no rule.
struct StopRule {
    int *flag = nullptr;
    const double *fnrm = nullptr;
    double tol = 0.0;
    int count = 0;  // 1: a miss adds one step to flag[1]
};

struct Ctx {
    lrspike_options opt{};
    cudaStream_t stream = nullptr;
    // coupling compression: second stream (non-blocking) on which the
    // coupling-block Gram matrices, their eigenvectors and the spike
    // right-hand sides run beside the band LU; fork / join events
    cudaStream_t side = nullptr;
    // second iterate buffer (n doubles) for the fused retrieval + residual of
    // the IR loop; allocated when every partition holds >= 256 + 2k rows
    double *xalt = nullptr;
    // set by run_sweep when the spike sweep wrote the COUPLING-mode u-factors
    // into Ucat itself (run_make_u then has nothing to do)
    bool u_by_sweep = false;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // factorisation of a host band (k <= 64, band LU by the column kernel):
    // the upload runs on its own stream in partition groups (the columns
    // around every interface first, for the coupling branch), and each
    // group's band LU starts on its own stream as soon as its columns land
    cudaStream_t up = nullptr;
    std::vector<cudaStream_t> grp_streams;
    std::vector<cudaEvent_t> grp_ev;  // [2g]: group g uploaded, [2g+1]: its LU done
    cudaEvent_t ev_up = nullptr, ev_strips = nullptr;
    int lu_g0 = 0, lu_g1 = -1;        // partitions [lu_g0, lu_g1) of the next band LU (lu_g1 < 0: all)
    int device = 0;
    int KB = 8;          // block size (>= k, power of two in 8..64)
    bool fp64 = true;    // working precision is double
    size_t tsize = 8;    // sizeof(T)
    int64_t n = 0, NB = 0, maxni = 0;
    int k = 0, p = 1, r = 0;
    int m = 0;           // spike columns: 2*KB (SPIKE) or 2*r (COUPLING)
    std::vector<int64_t> off_h, boff_h;
    int64_t *off_d = nullptr, *boff_d = nullptr;

    // factors: LT/UT tiles [NB][KB][KB], DI [NB][KB]
    void *LT = nullptr, *UT = nullptr, *DI = nullptr;
    void *X = nullptr;        // spike columns [NB][KB][m]
    // pivoted factors (pivoting = 1) instead of LT/UT/DI: per block
    // [L_JJ^{-1}, L_{J+1,J}, U_JJ^{-1}, U_{J,J+1}, U_{J,J+2}] and the gather
    // permutation of the 2KB stacked rows
    void *PF = nullptr;
    unsigned char *PIVP = nullptr;
    void *Ucat = nullptr;     // low-rank columns [n][2r]: u_T then u_W
    void *PQ = nullptr;       // projections [p][2][r][KB]: P_i (T~_i), Q_i (W~_i)
    double *Gram = nullptr;   // [p][2][KB][KB]
    double *Gpart = nullptr;  // [p][chunks][2][KB][KB]
    int gram_chunks = 1;
    double *sigma = nullptr;  // [p][2][r]
    // reduced system, interfaces i = 0..p-2, blocks of 2r x 2r (row-major)
    double *E = nullptr, *F = nullptr, *Gs = nullptr;   // diagonal, super, sub blocks
    double *Rinv = nullptr;   // TRUNCATED: E_i^{-1}
    // FULL: block cyclic reduction of R (set 0) and of R^T (set 1): working
    // copies of the blocks (reduced in place level by level), the inverses of
    // the blocks each level eliminates, and the level multipliers
    // alpha = G E^{-1}, beta = F E^{-1} of the equations it keeps
    struct BcrSet {
        double *E = nullptr, *F = nullptr, *G = nullptr, *Einv = nullptr, *al = nullptr, *be = nullptr;
    } bcr[2];
    bool bcr_t_ready = false;  // bcr[1] (R^T) reduced since the last factorisation

    // solve scratch (max_nrhs columns)
    double *rv = nullptr;     // FP64 residual / work vector, n x max_nrhs
    void *Yv = nullptr;       // T, n x max_nrhs: forward-sweep results
    void *Gv = nullptr;       // T, n x max_nrhs: D-stage result g
    double *psi = nullptr;    // [p-1][2r][max_nrhs]
    double *zr = nullptr;     // [p-1][2r][max_nrhs]
    double *wr = nullptr;     // FULL solve work, same size
    double *nrm = nullptr;    // [4][max_nrhs]: |f|, |r|, 1/|r|, spare
    double *partial = nullptr;
    int64_t npartial = 0;
    unsigned int *counter = nullptr;
    int64_t *status = nullptr; // first singular global row (INT64_MAX = none)
    int *stopf = nullptr;       // graph-safe early exit: [0] converged, [1] steps applied
    StopRule stop;              // rule the residual applies during a graph-safe solve
    const int *skip = nullptr;  // refinement kernels return at entry while *skip != 0
    double *host = nullptr;    // pinned host scratch
    // BiCGStab vectors (FP64, n x max_nrhs each: r, shadow r, p, v, s, t,
    // M^{-1}p, M^{-1}s), per-column scalars and reduction partials
    double *bv[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double *dots = nullptr;
    double *bpartial = nullptr;

    // wide bands (k > 64): blocks of W = 64 ceil(k/64); every partition padded
    // to NBW blocks (PS = NBW W rows).  Block products run on the tensor cores
    // (gpath 1: TF32, 2: BF16 operands) or as SIMT GEMMs (gpath 0: FP64 and
    // FP32 modes).  Each matrix that enters products is kept in the layouts
    // they read (WMat in wide.cu): working precision column-major / row-major,
    // operand type column-major / row-major.
    bool wide = false;
    int W = 0, NBW = 0, ell = 0, lp = 0;
    int64_t PS = 0;
    int gpath = 0;
    size_t osize = 8;        // operand element size of the block products
    int dcs = 0;             // CTAs per partition (cluster size) of the last D-stage launch
    // factor tiles, kinds 0..3 = L_JJ^{-1}, U_JJ^{-1}, Z_J = U_{J,J+1}, Y_J = L_{J+1,J},
    // each [p][NBW][W x W]; layouts f, fr, oc, orow
    void *WF[4] = {}, *WFr[4] = {}, *WFoc[4] = {}, *WFor[4] = {};
    // block-step work [p][W x W] (layouts f, fr, oc, orow): Schur complement,
    // A_{J,J+1}, A_{J+1,J}, recursion temporary
    void *WSm[4] = {}, *WBm[4] = {}, *WCm[4] = {}, *WTm[4] = {};
    // randomized truncation without explicit spikes: the range finder's
    // products T X = A_i^{-1}[0; B_i X] and T^T Q = [0; B_i]^T A_i^{-T} Q are
    // block solves on panels of 2 lp columns (T side, W side)
    void *WCpl[4] = {};                     // coupling tiles B_i / C_i [2p][W x W] (layouts f, fr, oc, orow)
    void *WP1 = nullptr, *WP2 = nullptr;    // solve panels [p][PS x 2lp], working precision
    void *WP1c = nullptr, *WP2c = nullptr;  // their operand-type copies (BF16 only)
    void *WTip = nullptr, *WTipc = nullptr; // panel tips [2p][W x lp] (working / operand BF16)
    void *WOm = nullptr;                    // sketches [2p][W x lp] (operand type)
    void *WQk = nullptr;                    // [2p][PS x lp]: orthonormal range basis (working)
    void *WZk = nullptr, *WZc = nullptr;    // [2p][W x lp]: T^T Q (working / operand BF16)
    void *WG = nullptr;                     // [2p][lp x lp] Gram (working)
    void *WGp = nullptr;                    // [2p][gram chunks of PS][lp x lp] partial Grams over row chunks
    double *WGd = nullptr;                  // [2p][lp x lp] FP64 Gram
    void *WRi = nullptr;                    // [2p][lp x lp] R^{-1} of the CholeskyQR pass
    void *WE = nullptr;                     // [2p][r][lp] leading eigenvectors
    void *WV1 = nullptr, *WV2 = nullptr;    // vector panels [p][PS x 16]
    int *gemm_err = nullptr;                // tensor-core GEMM wait-limit flag
    // the device work of a wide-band factorisation, captured once into a CUDA
    // graph (on a private stream) and replayed while the band's address and
    // leading dimension stay the same; not used when profiling
    cudaStream_t wcap = nullptr;
    cudaGraphExec_t wgraph = nullptr;
    const double *wgraph_band = nullptr;
    int64_t wgraph_ld = 0, wgraph_launches = 0;
    bool wgraph_failed = false;  // capture refused: launches run eagerly
    int *diag_list = nullptr;              // band rows holding a nonzero (residual), or NULL
    int ndiag = 0;

    const double *band = nullptr;
    int64_t ld = 0;
    double *band_own = nullptr;
    size_t band_own_bytes = 0;
    double *io_f = nullptr, *io_x = nullptr;  // device copies for host-pointer solves
    size_t io_bytes = 0;
    bool factored = false;
    int last_nrhs = 0;        // graph_safe: columns of the last enqueued solve
    // LR-SPIKE-OTF (reduced = OTF; the factorisation is the TRUNCATED one)
    bool otf = false;
    int otf_iters = 0;        // reduced BiCGStab iterations of the last solve
    double *ocv = nullptr;    // FP64 n x max_nrhs: coupling right-hand side c(y)
    void *og = nullptr;       // T, n x max_nrhs: g = D^{-1} f kept for the recovery
    double *orv = nullptr;    // kOtfVecs reduced vectors [p-1][2k] x max_nrhs
    double *osc = nullptr;    // reduced BiCGStab scalars
    double *oone = nullptr;   // max_nrhs ones (unscaled D-stage input)

    std::string err;
    int64_t launches = 0;
    bool profile = false;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    int64_t kcount[KID_COUNT] = {};
    double kms[KID_COUNT] = {};
};

// Records a kernel launch: counts it and, when profiling, brackets it with
// events on the handle's stream.  Returns false (with c->err set) when the
// launch failed.
bool begin_launch(Ctx *c, int kid, cudaEvent_t *ev_end);
bool end_launch(Ctx *c, int kid, cudaEvent_t ev_end);

template <typename F>
inline bool launch(Ctx *c, int kid, F &&f) {
    cudaEvent_t e = nullptr;
    if (!begin_launch(c, kid, &e)) return false;
    f();
    return end_launch(c, kid, e);
}

// ---- launchers (each dispatches on the working precision and KB) --------
bool run_band_lu(Ctx *c);
// column-by-column band LU + per-block triangular inverses (same tiles)
bool run_band_lu_col(Ctx *c);
bool run_spike_rhs(Ctx *c);
bool run_sweep(Ctx *c);
bool run_gram(Ctx *c);
bool run_coupling_gram(Ctx *c);
bool run_jacobi(Ctx *c);
bool run_make_u(Ctx *c);
bool run_reduced_build(Ctx *c);
bool run_reduced_factor(Ctx *c);

// solve-phase pieces; nrhs columns, ld = leading dimension of f / x
bool run_norms(Ctx *c, const double *v, int64_t ld, int nrhs, double *out);
bool run_residual(Ctx *c, const double *f, const double *x, int64_t ld, int nrhs, bool trans,
                  bool x_zero);
bool run_dstage(Ctx *c, const double *rin, int64_t ld, int nrhs);
// the same with the column scale factors of the input given explicitly
bool run_dstage_inv(Ctx *c, const double *rin, int nrhs, const double *inv);
bool run_reduced_solve(Ctx *c, int nrhs, bool trans);
bool run_retrieve(Ctx *c, double *x, int64_t ld, int nrhs, bool accumulate);
bool run_project_t(Ctx *c, const double *hin, int64_t ld, int nrhs);
bool run_dstage_t(Ctx *c, const double *hin, int64_t ldh, double *x, int64_t ldx, int nrhs, bool accumulate);
// wide bands (wide.cu)
bool wide_setup(Ctx *c);
void wide_free(Ctx *c);
bool run_wide_factor(Ctx *c);
bool run_wide_dstage(Ctx *c, const double *rin, int nrhs);
bool run_wide_dstage_inv(Ctx *c, const double *rin, int nrhs, const double *inv);
bool run_wide_dstage_t(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, bool accumulate);
bool run_lu_inv64(Ctx *c, void *A, int lda, int64_t sA, void *Li, void *Ui, int ldo, int64_t sO, int64_t row0);
bool run_jacobi_batch(Ctx *c, int n, const double *G, int nmat, int rout, double rank_tol, void *out,
                      double *sigma);
bool run_reduced_build_ld(Ctx *c, int ldpq);
// partial pivoting inside the partitions (pivot.cu)
bool run_band_lu_piv(Ctx *c);
bool run_sweep_piv(Ctx *c);
bool run_dstage_piv(Ctx *c, const double *rin, int nrhs);
bool run_dstage_t_piv(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, bool accumulate);
bool launch_residual_raw(const double *band, int64_t ldb, int k, int64_t n, const double *f,
                         const double *x, int64_t ld, int nrhs, double *r, double *partial,
                         unsigned *counter, double *nrm, cudaStream_t st);
// Block products of the wide-band path on the tensor cores (tc_gemm.cu):
// C_b = alpha A'_b B'_b^T + beta C_b with K-contiguous operands, element
// (m, k) of A'_b at p + b s + m ld + k (FP32 values read as TF32, or BF16).
struct GemmOperand {
    const void *p;
    int64_t ld, s;
};
// Outputs (each nullable): f, FP32 column-major f[m + n ldf + b sf] (beta
// reads it); row, operand type, row-major row[(n % rsplit) + (n / rsplit) rss
// + m ldr + b sr] (rsplit 0 = no split); frow, FP32 with the same row-major
// map; col, operand type, column-major.
struct GemmOutput {
    float *f = nullptr;
    int64_t ldf = 0, sf = 0;
    void *row = nullptr;
    int64_t ldr = 0, sr = 0;
    int rsplit = 0;
    int64_t rss = 0;
    void *col = nullptr;
    int64_t ldc = 0, sc = 0;
    float *frow = nullptr;
};
// A tiled TMA tensor map (no swizzle, zero fill out of range) through the
// driver's encoder; false with *err set when the encoder refuses it.
bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                       const cuuint64_t *strides, const cuuint32_t *box, const cuuint32_t *estr, std::string *err);
bool tc_gemm(cudaStream_t st, bool bf16, int M, int N, int K, int batch, float alpha, const GemmOperand &A,
             const GemmOperand &B, float beta, const GemmOutput &C, int *err_dev, std::string *err);
// error text returned by lrspike_last_error(NULL)
void set_handleless_error(const std::string &msg);
// M^{-1} (or M^{-T}) applied to the FP64 vector in (n x nrhs, leading
// dimension n) whose column norms |in| and 1/|in| are at nrm + max_nrhs and
// nrm + 2 max_nrhs: out (+)= |in| * M^{-1}(in/|in|).  Used by the outer loops.
bool apply_precond(Ctx *c, const double *in, double *out, int64_t ldo, int nrhs, bool trans, bool accumulate);
// The outer IR loop may defer the retrieval of an application into the next
// residual: apply_precond_deferred leaves g (Gv) and z (zr) for
// run_residual_retrieve, which forms x_out = x_in + |r| (g - U z) and
// r = f - A x_out in one kernel (x_out != x_in).  Only where
// fused_retrieve_ok holds.
bool fused_retrieve_ok(const Ctx *c, int nrhs, bool trans);
bool apply_precond_deferred(Ctx *c, const double *in, int nrhs);
bool run_residual_retrieve(Ctx *c, const double *f, const double *x_in, double *x_out);
// LR-SPIKE-OTF (otf.cu): out (+)= |in| * (OTF solve of in/|in|)
constexpr int kOtfVecs = 10;
bool otf_alloc(Ctx *c);
bool apply_otf(Ctx *c, const double *in, double *out, int64_t ldo, int nrhs, bool accumulate);

// BiCGStab outer iteration (right-preconditioned, FP64 vectors).
struct BicgResult {
    int iterations = 0;
    bool breakdown = false;   // a column hit a zero or non-finite scalar
    std::vector<double> rel;  // final |f - A x| / |f| per column (true residual)
};
bool bicgstab_alloc(Ctx *c);
bool run_bicgstab(Ctx *c, const double *f, double *x, int64_t ldx, int nrhs, bool trans, BicgResult &res);

}  // namespace lrs
