// Wide bands, 64 < k <= 1024 (the 2-D convection-diffusion systems of
// section 4, half-bandwidth = grid width).
//
// Every partition A_i is cut into blocks of W = 64 ceil(k/64) >= k rows, so it
// is block tridiagonal with W x W blocks; partitions are padded to NBW blocks
// with identity rows.  The block operations are dense contractions of order
// W (up to 1024), run as batched GEMMs over the p partitions (cuBLAS; FP64,
// FP32, or TF32 tensor cores with FP32 accumulation for LRSPIKE_MIXED_TF32):
//
//   factor, block step J (all partitions at once):
//     S_J = A_JJ - Y_{J-1} Z_{J-1};  S_J = L U with L^{-1}, U^{-1} by
//     recursive halving (64 x 64 base blocks in k_lu_inv64);
//     Z_J = L_JJ^{-1} A_{J,J+1} (= U_{J,J+1}),  Y_J = A_{J+1,J} U_JJ^{-1} (= L_{J+1,J})
//   spikes [T_i | W_i] = A_i^{-1} [[0; B_i] | [C_i; 0]] (eq. 'Veqn') by the
//     forward and backward block recurrences on a 2W-column panel
//   compression: the randomized SVD the paper uses for wide bands (section
//     3.1, Halko-Martinsson-Tropp proto-algorithm), on the right singular
//     subspace through G = T^T T: Y = G Omega, power passes with
//     re-orthonormalisation, Rayleigh-Ritz on Q^T G Q; u = T V_r, P = V_r^T
//   D-stage and its transpose: the same block recurrences on nrhs columns.
//
// Layouts: column-major W x W tiles; factor tiles [p][NBW][W x W]; panels
// [p][PS x cols] with PS = NBW W rows (leading dimension PS).
#include <cublas_v2.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrs {

namespace {

constexpr int VP = 16;  // columns of the vector panels (max nrhs)

// ---------------------------------------------------------------------------
// A_JJ (S), A_{J,J+1} (B), A_{J+1,J} (C) of every partition, W x W column-major.
// One CTA per 32 x 32 tile: it reads the tile along band diagonals (consecutive
// columns are consecutive band addresses) and writes it column by column.
template <typename T>
__global__ void __launch_bounds__(256)
    k_wide_gather(const double *__restrict__ band, int64_t ld, int k, Parts P, int W, int J, T *__restrict__ S,
                  T *__restrict__ B, T *__restrict__ C) {
    __shared__ T tile[32][33];
    const int which = blockIdx.z % 3, part = blockIdx.z / 3;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int64_t rb = (which == 2) ? (int64_t)(J + 1) * W : (int64_t)J * W;  // first local row
    const int64_t cb = (which == 1) ? (int64_t)(J + 1) * W : (int64_t)J * W;  // first local column
    for (int e = threadIdx.x; e < 63 * 32; e += 256) {
        const int dd = e / 32 - 31, b = e % 32, a = b + dd;
        if (a < 0 || a >= 32) continue;
        const int64_t lr = rb + a0 + a, lc = cb + b0 + b;
        T v = T(0);
        if (lr < ni && lc < ni) {
            const int64_t d = k + lr - lc;
            if (d >= 0 && d <= 2 * k) v = (T)band[d * ld + s + lc];
        } else if (which == 0 && lr == lc) {
            v = T(1);  // padding rows carry the identity
        }
        tile[a][b] = v;
    }
    __syncthreads();
    T *out = (which == 0 ? S : which == 1 ? B : C) + (int64_t)part * W * W;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int b = ty; b < 32; b += 8) out[(int64_t)(b0 + b) * W + a0 + tx] = tile[tx][b];
}

// Spike right-hand sides on the zeroed panel X [PS x 2W]: [0; B_i] in columns
// 0..k-1 (rows n_i-k..n_i-1) and [C_i; 0] in columns W..W+k-1 (rows 0..k-1).
template <typename T>
__global__ void k_wide_spike_rhs(const double *__restrict__ band, int64_t ld, int k, Parts P, int W, int64_t PS,
                                 T *__restrict__ X) {
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    T *x = X + (int64_t)part * PS * 2 * W;
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int a = (int)(e % k), b = (int)(e / k);
        if (part < P.p - 1) {  // B_i[a][b] = A[s+n_i-k+a][s+n_i+b], nonzero for b <= a
            const int64_t sn = s + ni;
            x[(int64_t)b * PS + ni - k + a] = (b <= a) ? (T)band[(int64_t)(a - b) * ld + sn + b] : T(0);
        }
        if (part > 0)  // C_i[a][b] = A[s+a][s-k+b], nonzero for a <= b
            x[(int64_t)(W + b) * PS + a] = (a <= b) ? (T)band[(int64_t)(2 * k + a - b) * ld + s - k + b] : T(0);
    }
}

// SplitMix64 (Steele, Lea, Flood 2014): output i of the generator started at seed.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Gaussian sketches Omega_b (W x lp, column-major), b = 2 i + side: entry
// (a, j), a < k, j < ell, is the Box-Muller normal of SplitMix64 outputs 2c,
// 2c+1 at c = a ell + j with seed + b; zero elsewhere.
template <typename T>
__global__ void k_wide_sketch(T *__restrict__ Om, int W, int k, int ell, int lp, unsigned long long seed,
                              int nmat) {
    const int64_t per = (int64_t)W * lp, total = per * nmat;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const int64_t rem = e % per;
        const int j = (int)(rem / W), a = (int)(rem % W);
        T v = T(0);
        if (a < k && j < ell) {
            const unsigned long long cidx = (unsigned long long)a * ell + j, sd = seed + (unsigned long long)b;
            const double u1 = ((double)(splitmix64(sd, 2 * cidx) >> 11) + 0.5) * 0x1p-53;
            const double u2 = (double)(splitmix64(sd, 2 * cidx + 1) >> 11) * 0x1p-53;
            v = (T)(sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2));
        }
        Om[e] = v;
    }
}

template <typename T>
__global__ void k_to_f64(const T *__restrict__ in, double *__restrict__ out, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (double)in[e];
}

// Columns c of E_b (lp x lp, column-major) scaled by 1 / sigma_{b,c} (0 where sigma is 0).
template <typename T>
__global__ void k_scale_cols(T *__restrict__ E, const double *__restrict__ sg, int lp, int nmat) {
    const int64_t total = (int64_t)nmat * lp * lp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / ((int64_t)lp * lp);
        const int c = (int)((e % ((int64_t)lp * lp)) / lp);
        const double sv = sg[b * lp + c];
        E[e] = (sv > 0.0) ? (T)((double)E[e] / sv) : T(0);
    }
}

// Vector panels: V[part][c][row] (leading dimension PS) <- r / |r|.
template <typename T>
__global__ void k_wide_pack(const double *__restrict__ rin, const double *__restrict__ inv, int64_t n, Parts P,
                            int64_t PS, int nrhs, T *__restrict__ V) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= PS) return;
    for (int c = 0; c < nrhs; ++c)
        V[((int64_t)part * VP + c) * PS + row] = (row < ni) ? (T)(rin[c * n + s + row] * inv[c]) : T(0);
}

// Transposed D-stage input: h / |h| minus V^T w at the partition tips
// (top rows: P_{i-1}^T w_zeta(i-1); bottom rows: Q_{i+1}^T w_omega(i)).
template <typename T>
__global__ void k_wide_pack_t(const double *__restrict__ hin, const double *__restrict__ inv,
                              const double *__restrict__ zr, const T *__restrict__ PQ, int W, Parts P, int k, int r,
                              int64_t n, int64_t PS, int nrhs, T *__restrict__ V) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= PS) return;
    const int n2 = 2 * r;
    for (int c = 0; c < nrhs; ++c) {
        double v = 0.0;
        if (row < ni) {
            v = hin[c * n + s + row] * inv[c];
            if (r > 0 && row < k && part >= 1) {
                const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * W;
                for (int j = 0; j < r; ++j)
                    v -= (double)Pm[(int64_t)j * W + row] * zr[((int64_t)(part - 1) * n2 + j) * nrhs + c];
            }
            if (r > 0 && row >= ni - k && part <= P.p - 2) {
                const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * W;
                const int64_t q = row - (ni - k);
                for (int j = 0; j < r; ++j)
                    v -= (double)Qm[(int64_t)j * W + q] * zr[((int64_t)part * n2 + r + j) * nrhs + c];
            }
        }
        V[((int64_t)part * VP + c) * PS + row] = (T)v;
    }
}

// g (n x nrhs, leading dimension n) <- the D-stage panel
template <typename T>
__global__ void k_wide_unpack(const T *__restrict__ V, int64_t n, Parts P, int64_t PS, int nrhs, T *__restrict__ Gv) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= ni) return;
    for (int c = 0; c < nrhs; ++c) Gv[c * n + s + row] = V[((int64_t)part * VP + c) * PS + row];
}

// x (+)= |h| * the transposed D-stage panel
template <typename T>
__global__ void k_wide_unpack_t(const T *__restrict__ V, const double *__restrict__ nrm, Parts P, int64_t PS,
                                int nrhs, double *__restrict__ x, int64_t ldx, int accumulate) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= ni) return;
    for (int c = 0; c < nrhs; ++c) {
        const double upd = nrm[c] * (double)V[((int64_t)part * VP + c) * PS + row];
        const int64_t xi = c * ldx + s + row;
        x[xi] = accumulate ? x[xi] + upd : upd;
    }
}

// psi_{i-1}[0:r] = P_{i-1} g_t,  psi_i[r:2r] = Q_{i+1} g_b  (FP64)
template <typename T>
__global__ void k_wide_psi(const T *__restrict__ Gv, const T *__restrict__ PQ, int W, Parts P, int k, int r,
                           int64_t n, int nrhs, double *__restrict__ psi) {
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int n2 = 2 * r;
    for (int o = threadIdx.x; o < 2 * r * nrhs; o += blockDim.x) {
        const int side = o / (r * nrhs), rem = o % (r * nrhs), j = rem / nrhs, c = rem % nrhs;
        if (side == 0 && part >= 1) {
            const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * W + (int64_t)j * W;
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += (double)Pm[q] * (double)Gv[c * n + s + q];
            psi[((int64_t)(part - 1) * n2 + j) * nrhs + c] = acc;
        } else if (side == 1 && part <= P.p - 2) {
            const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * W + (int64_t)j * W;
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += (double)Qm[q] * (double)Gv[c * n + s + ni - k + q];
            psi[((int64_t)part * n2 + r + j) * nrhs + c] = acc;
        }
    }
}

// flag[d] = 1 when band row d holds a nonzero entry inside the matrix
__global__ void k_nonzero_diags(const double *__restrict__ band, int64_t ld, int64_t n, int k, int *__restrict__ flag) {
    const int d = blockIdx.y;
    const int64_t lo = std::max<int64_t>(0, k - d), hi = std::min<int64_t>(n, n + k - d);  // columns j with 0 <= j+d-k < n
    bool any = false;
    for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi; j += (int64_t)gridDim.x * blockDim.x)
        any = any || band[(int64_t)d * ld + j] != 0.0;
    if (__syncthreads_or(any) && threadIdx.x == 0) flag[d] = 1;
}

// ---------------------------------------------------------------------------
inline char *at(void *base, int64_t elems, int tsz) { return static_cast<char *>(base) + elems * tsz; }

bool gemm(Ctx *c, bool ta, bool tb, int m, int n, int kk, double alpha, const void *A, int lda, int64_t sA,
          const void *B, int ldb, int64_t sB, double beta, void *C, int ldc, int64_t sC, int batch) {
    cublasHandle_t h = static_cast<cublasHandle_t>(c->blas);
    const cudaDataType dt = c->fp64 ? CUDA_R_64F : CUDA_R_32F;
    const cublasComputeType_t ct = c->fp64 ? CUBLAS_COMPUTE_64F
                                   : (c->opt.precision == LRSPIKE_MIXED_TF32) ? CUBLAS_COMPUTE_32F_FAST_TF32
                                                                               : CUBLAS_COMPUTE_32F;
    const float af = (float)alpha, bf = (float)beta;
    const void *pa = c->fp64 ? static_cast<const void *>(&alpha) : static_cast<const void *>(&af);
    const void *pb = c->fp64 ? static_cast<const void *>(&beta) : static_cast<const void *>(&bf);
    cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
    const bool ok = launch(c, KID_WIDE_GEMM, [&] {
        st = cublasGemmStridedBatchedEx(h, ta ? CUBLAS_OP_T : CUBLAS_OP_N, tb ? CUBLAS_OP_T : CUBLAS_OP_N, m, n, kk,
                                        pa, A, dt, lda, sA, B, dt, ldb, sB, pb, C, dt, ldc, sC, batch, ct,
                                        CUBLAS_GEMM_DEFAULT);
    });
    if (st != CUBLAS_STATUS_SUCCESS) {
        c->err = "cuBLAS batched GEMM failed with status " + std::to_string((int)st);
        return false;
    }
    return ok;
}

// In-place recursive LU with both inverses of the n x n leading view of A
// (column-major, leading dimension W, one matrix per partition at stride sA):
// Li = L^{-1}, Ui = U^{-1} (views at stride sO), Tm is workspace (stride sT).
// Halves: A11 = L11 U11; U12 = L11^{-1} A12; L21 = A21 U11^{-1};
// A22 -= L21 U12 = L22 U22; (L^{-1})_21 = -L22^{-1} L21 L11^{-1},
// (U^{-1})_12 = -U11^{-1} U12 U22^{-1}.  The zero triangles of Li, Ui must be
// zero on entry.
bool luinv(Ctx *c, void *A, void *Li, void *Ui, void *Tm, int n, int64_t sA, int64_t sO, int64_t sT, int64_t row0) {
    const int W = c->W, tz = c->tsize, p = c->p;
    if (n == 64) return run_lu_inv64(c, A, W, sA, Li, Ui, W, sO, row0);
    const int h = n / 2;
    auto q12 = [&](void *b) { return at(b, (int64_t)h * W, tz); };
    auto q21 = [&](void *b) { return at(b, h, tz); };
    auto q22 = [&](void *b) { return at(b, (int64_t)h * W + h, tz); };
    if (!luinv(c, A, Li, Ui, Tm, h, sA, sO, sT, row0)) return false;
    return gemm(c, false, false, h, h, h, 1.0, Li, W, sO, q12(A), W, sA, 0.0, q12(Tm), W, sT, p) &&      // U12
           gemm(c, false, false, h, h, h, 1.0, q21(A), W, sA, Ui, W, sO, 0.0, q21(Tm), W, sT, p) &&      // L21
           gemm(c, false, false, h, h, h, -1.0, q21(Tm), W, sT, q12(Tm), W, sT, 1.0, q22(A), W, sA, p) &&  // A22 -= L21 U12
           luinv(c, q22(A), q22(Li), q22(Ui), q22(Tm), h, sA, sO, sT, row0 + h) &&
           gemm(c, false, false, h, h, h, 1.0, q21(Tm), W, sT, Li, W, sO, 0.0, q21(A), W, sA, p) &&      // L21 L11^{-1}
           gemm(c, false, false, h, h, h, -1.0, q22(Li), W, sO, q21(A), W, sA, 0.0, q21(Li), W, sO, p) &&
           gemm(c, false, false, h, h, h, 1.0, q12(Tm), W, sT, q22(Ui), W, sO, 0.0, q12(A), W, sA, p) &&  // U12 U22^{-1}
           gemm(c, false, false, h, h, h, -1.0, Ui, W, sO, q12(A), W, sA, 0.0, q12(Ui), W, sO, p);
}

template <typename T>
bool wide_factor_t(Ctx *c) {
    const int W = c->W, NB = c->NBW, p = c->p, tz = c->tsize;
    const int64_t WW = (int64_t)W * W, sF = NB * WW, PS = c->PS;
    Parts P{c->off_d, c->boff_d, p};
    const size_t tiles = (size_t)p * sF * tz;
    if (cudaMemsetAsync(c->WLi, 0, tiles, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->WUi, 0, tiles, c->stream) != cudaSuccess) {
        c->err = "cudaMemsetAsync failed";
        return false;
    }
    for (int J = 0; J < NB; ++J) {
        if (!launch(c, KID_WIDE_GATHER, [&] {
                k_wide_gather<T><<<dim3(W / 32, W / 32, 3 * p), 256, 0, c->stream>>>(
                    c->band, c->ld, c->k, P, W, J, (T *)c->WS, (T *)c->WB, (T *)c->WC);
            }))
            return false;
        void *Li = at(c->WLi, J * WW, tz), *Ui = at(c->WUi, J * WW, tz);
        void *Z = at(c->WZ, J * WW, tz), *Y = at(c->WY, J * WW, tz);
        if (J > 0 && !gemm(c, false, false, W, W, W, -1.0, at(c->WY, (J - 1) * WW, tz), W, sF,
                           at(c->WZ, (J - 1) * WW, tz), W, sF, 1.0, c->WS, W, WW, p))
            return false;
        if (!luinv(c, c->WS, Li, Ui, c->WT, W, WW, sF, WW, (int64_t)J * W)) return false;
        if (!gemm(c, false, false, W, W, W, 1.0, Li, W, sF, c->WB, W, WW, 0.0, Z, W, sF, p) ||
            !gemm(c, false, false, W, W, W, 1.0, c->WC, W, WW, Ui, W, sF, 0.0, Y, W, sF, p))
            return false;
    }
    if (p < 2 || c->r == 0) return true;

    // spikes [T | W] on the panel X1 (forward results in X2, solution back in X1)
    const int64_t sX = PS * 2 * W;
    const size_t panel = (size_t)p * sX * tz;
    if (cudaMemsetAsync(c->WX1, 0, panel, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->WX2, 0, panel, c->stream) != cudaSuccess) {
        c->err = "cudaMemsetAsync failed";
        return false;
    }
    if (!launch(c, KID_SPIKE_RHS, [&] {
            k_wide_spike_rhs<T><<<p, 256, 0, c->stream>>>(c->band, c->ld, c->k, P, W, PS, (T *)c->WX1);
        }))
        return false;
    // the T columns are zero above the block holding the first row of B_i
    int64_t jt0 = NB;
    for (int i = 0; i < p; ++i) jt0 = std::min<int64_t>(jt0, (c->off_h[i + 1] - c->off_h[i] - c->k) / W);
    for (int J = 0; J < NB; ++J) {
        const int c0 = (J < jt0) ? W : 0, nc = 2 * W - c0;
        void *x1 = at(c->WX1, (int64_t)c0 * PS + (int64_t)J * W, tz);
        void *x2 = at(c->WX2, (int64_t)c0 * PS + (int64_t)J * W, tz);
        if (J > 0 && !gemm(c, false, false, W, nc, W, -1.0, at(c->WY, (J - 1) * WW, tz), W, sF,
                           at(c->WX2, (int64_t)c0 * PS + (int64_t)(J - 1) * W, tz), (int)PS, sX, 1.0, x1, (int)PS,
                           sX, p))
            return false;
        if (!gemm(c, false, false, W, nc, W, 1.0, at(c->WLi, J * WW, tz), W, sF, x1, (int)PS, sX, 0.0, x2, (int)PS,
                  sX, p))
            return false;
    }
    for (int J = NB - 1; J >= 0; --J) {
        void *x1 = at(c->WX1, (int64_t)J * W, tz), *x2 = at(c->WX2, (int64_t)J * W, tz);
        if (J < NB - 1 && !gemm(c, false, false, W, 2 * W, W, -1.0, at(c->WZ, J * WW, tz), W, sF,
                                at(c->WX1, (int64_t)(J + 1) * W, tz), (int)PS, sX, 1.0, x2, (int)PS, sX, p))
            return false;
        if (!gemm(c, false, false, W, 2 * W, W, 1.0, at(c->WUi, J * WW, tz), W, sF, x2, (int)PS, sX, 0.0, x1, (int)PS,
                  sX, p))
            return false;
    }

    // Gram matrices: G_{2i} = T_i^T T_i, G_{2i+1} = W_i^T W_i
    for (int side = 0; side < 2; ++side) {
        void *xs = at(c->WX1, (int64_t)side * W * PS, tz);
        if (!gemm(c, true, false, W, W, (int)PS, 1.0, xs, (int)PS, sX, xs, (int)PS, sX, 0.0, at(c->WG, side * WW, tz), W,
                  2 * WW, p))
            return false;
    }

    // randomized subspace iteration on every Gram matrix (2p of them)
    const int nm = 2 * p, lp = c->lp, ell = c->ell, r = c->r;
    const int64_t sY = (int64_t)W * lp, sH = (int64_t)lp * lp;
    const double orth_tol = c->fp64 ? 1e-7 : 1e-3;
    if (!launch(c, KID_WIDE_VEC, [&] {
            k_wide_sketch<T><<<1024, 256, 0, c->stream>>>((T *)c->WOm, W, c->k, ell, lp, c->opt.seed, nm);
        }))
        return false;
    auto orth = [&](void *Y, void *Q) {  // Q = Y V Lambda^{-1/2} from Y^T Y = V Lambda V^T
        return gemm(c, true, false, lp, lp, W, 1.0, Y, W, sY, Y, W, sY, 0.0, c->WH, lp, sH, nm) &&
               launch(c, KID_WIDE_VEC, [&] {
                   k_to_f64<T><<<64, 256, 0, c->stream>>>((const T *)c->WH, c->WHd, nm * sH);
               }) &&
               run_jacobi_batch(c, lp, c->WHd, nm, lp, orth_tol, c->WE, c->Wsg) &&
               launch(c, KID_WIDE_VEC, [&] {
                   k_scale_cols<T><<<64, 256, 0, c->stream>>>((T *)c->WE, c->Wsg, lp, nm);
               }) &&
               gemm(c, false, false, W, lp, lp, 1.0, Y, W, sY, c->WE, lp, sH, 0.0, Q, W, sY, nm);
    };
    if (!gemm(c, false, false, W, lp, W, 1.0, c->WG, W, WW, c->WOm, W, sY, 0.0, c->WYk, W, sY, nm)) return false;
    for (int it = 0; it < c->opt.power_iters; ++it)
        if (!orth(c->WYk, c->WQk) ||
            !gemm(c, false, false, W, lp, W, 1.0, c->WG, W, WW, c->WQk, W, sY, 0.0, c->WYk, W, sY, nm))
            return false;
    if (!orth(c->WYk, c->WQk) ||
        !gemm(c, false, false, W, lp, W, 1.0, c->WG, W, WW, c->WQk, W, sY, 0.0, c->WTk, W, sY, nm) ||
        !gemm(c, true, false, lp, lp, W, 1.0, c->WQk, W, sY, c->WTk, W, sY, 0.0, c->WH, lp, sH, nm) ||
        !launch(c, KID_WIDE_VEC, [&] {
            k_to_f64<T><<<64, 256, 0, c->stream>>>((const T *)c->WH, c->WHd, nm * sH);
        }) ||
        !run_jacobi_batch(c, lp, c->WHd, nm, r, c->opt.rank_tol, c->WE, c->sigma))
        return false;
    // P^T = V_r = Q E_r (W x r, leading dimension W): PQ holds P row-major r x W;
    // E_r of matrix b (r eigenvectors of length lp) starts at b r lp
    if (!gemm(c, false, false, W, r, lp, 1.0, c->WQk, W, sY, c->WE, lp, (int64_t)r * lp, 0.0, c->PQ, W,
              (int64_t)r * W, nm))
        return false;

    // u = X V_r into Ucat (row-major n x 2r): u^T (r x n_i, leading dimension 2r)
    // = V_r^T X^T, partitions grouped by n_i for pointer-array batches
    std::vector<std::pair<int64_t, std::vector<int>>> groups;
    for (int i = 0; i < p; ++i) {
        const int64_t ni = c->off_h[i + 1] - c->off_h[i];
        auto g = std::find_if(groups.begin(), groups.end(), [&](const auto &x) { return x.first == ni; });
        if (g == groups.end()) groups.push_back({ni, {i}});
        else g->second.push_back(i);
    }
    // per (group, side): [A pointers][B pointers][C pointers]
    std::vector<const void *> hp;
    for (auto &g : groups)
        for (int side = 0; side < 2; ++side) {
            for (int i : g.second) hp.push_back(at(c->PQ, (int64_t)(2 * i + side) * r * W, tz));
            for (int i : g.second) hp.push_back(at(c->WX1, (int64_t)i * sX + (int64_t)side * W * PS, tz));
            for (int i : g.second) hp.push_back(at(c->Ucat, c->off_h[i] * 2 * r + side * r, tz));
        }
    // the pointer arrays are read by the GEMMs of this factorisation only
    if (cudaMemcpyAsync(c->Wptr, hp.data(), hp.size() * sizeof(void *), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess) {
        c->err = "pointer array copy failed";
        return false;
    }
    cublasHandle_t hb = static_cast<cublasHandle_t>(c->blas);
    const cudaDataType dt = c->fp64 ? CUDA_R_64F : CUDA_R_32F;
    const cublasComputeType_t ct = c->fp64 ? CUBLAS_COMPUTE_64F
                                   : (c->opt.precision == LRSPIKE_MIXED_TF32) ? CUBLAS_COMPUTE_32F_FAST_TF32
                                                                               : CUBLAS_COMPUTE_32F;
    const double one = 1.0, zero = 0.0;
    const float onef = 1.0f, zerof = 0.0f;
    size_t off = 0;
    for (auto &g : groups)
        for (int side = 0; side < 2; ++side) {
            const int cnt = (int)g.second.size();
            void **base = c->Wptr + off;
            cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
            const bool ok = launch(c, KID_WIDE_GEMM, [&] {
                st = cublasGemmBatchedEx(hb, CUBLAS_OP_T, CUBLAS_OP_T, r, (int)g.first, W,
                                         c->fp64 ? (const void *)&one : (const void *)&onef, base, dt, W, base + cnt,
                                         dt, (int)PS, c->fp64 ? (const void *)&zero : (const void *)&zerof,
                                         base + 2 * cnt, dt, 2 * r, cnt, ct, CUBLAS_GEMM_DEFAULT);
            });
            if (!ok || st != CUBLAS_STATUS_SUCCESS) {
                if (c->err.empty()) c->err = "cuBLAS batched GEMM (u-factors) failed";
                return false;
            }
            off += 3 * (size_t)cnt;
        }
    return true;
}

}  // namespace

bool wide_setup(Ctx *c) {
    const int k = c->k, p = c->p, r = c->r;
    c->W = 64 * ((k + 63) / 64);
    int64_t nbw = 0;
    for (int i = 0; i < p; ++i) nbw = std::max<int64_t>(nbw, (c->off_h[i + 1] - c->off_h[i] + c->W - 1) / c->W);
    c->NBW = (int)nbw;
    c->PS = nbw * c->W;
    c->ell = std::min(k, r + c->opt.oversample);
    c->lp = c->ell <= 16 ? 16 : c->ell <= 32 ? 32 : 64;
    const size_t tz = c->tsize, W = c->W, WW = W * W, NB = c->NBW, PS = c->PS, lp = c->lp;
    auto al = [&](void **ptr, size_t bytes) { return cudaMalloc(ptr, bytes) == cudaSuccess; };
    bool ok = al(&c->WLi, p * NB * WW * tz) && al(&c->WUi, p * NB * WW * tz) && al(&c->WZ, p * NB * WW * tz) &&
              al(&c->WY, p * NB * WW * tz) && al(&c->WS, p * WW * tz) && al(&c->WB, p * WW * tz) &&
              al(&c->WC, p * WW * tz) && al(&c->WT, p * WW * tz) && al(&c->WV1, p * PS * VP * tz) &&
              al(&c->WV2, p * PS * VP * tz) && al((void **)&c->diag_list, (2 * k + 1) * sizeof(int));
    if (ok && p > 1 && r > 0)
        ok = al(&c->WX1, p * PS * 2 * W * tz) && al(&c->WX2, p * PS * 2 * W * tz) && al(&c->WG, 2 * p * WW * tz) &&
             al(&c->WOm, 2 * p * W * lp * tz) && al(&c->WYk, 2 * p * W * lp * tz) &&
             al(&c->WQk, 2 * p * W * lp * tz) && al(&c->WTk, 2 * p * W * lp * tz) &&
             al(&c->WH, 2 * p * lp * lp * tz) && al(&c->WE, 2 * p * lp * lp * tz) &&
             al((void **)&c->WHd, 2 * p * lp * lp * 8) && al((void **)&c->Wsg, 2 * p * lp * 8) &&
             al((void **)&c->Wptr, 6 * (size_t)p * sizeof(void *));
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return false;
    c->blas = h;
    return cublasSetStream(h, c->stream) == CUBLAS_STATUS_SUCCESS;
}

void wide_free(Ctx *c) {
    void *ptrs[] = {c->WLi, c->WUi, c->WZ,  c->WY,  c->WS,  c->WB,   c->WC,  c->WT,    c->WX1,
                    c->WX2, c->WG,  c->WOm, c->WYk, c->WQk, c->WTk,  c->WH,  c->WE,    c->WHd,
                    c->Wsg, c->WV1, c->WV2, c->Wptr, c->diag_list};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (c->blas) cublasDestroy(static_cast<cublasHandle_t>(c->blas));
    c->blas = nullptr;
}

bool run_wide_factor(Ctx *c) {
    const bool ok = c->fp64 ? wide_factor_t<double>(c) : wide_factor_t<float>(c);
    if (!ok) return false;
    if (c->p > 1 && c->r > 0 && !(run_reduced_build_ld(c, c->W) && run_reduced_factor(c))) return false;
    // band rows with a nonzero entry: the FP64 residual visits only those
    const int nd = 2 * c->k + 1;
    if (cudaMemsetAsync(c->diag_list, 0, nd * sizeof(int), c->stream) != cudaSuccess) return false;
    if (!launch(c, KID_DIAGS, [&] {
            k_nonzero_diags<<<dim3(64, nd), 256, 0, c->stream>>>(c->band, c->ld, c->n, c->k, c->diag_list);
        }))
        return false;
    std::vector<int> flag(nd), list;
    if (cudaMemcpyAsync(flag.data(), c->diag_list, nd * sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return false;
    for (int d = 0; d < nd; ++d)
        if (flag[d]) list.push_back(d);
    if (list.empty()) list.push_back(c->k);
    c->ndiag = (int)list.size();
    return cudaMemcpyAsync(c->diag_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice,
                           c->stream) == cudaSuccess &&
           cudaStreamSynchronize(c->stream) == cudaSuccess;
}

template <typename T>
static bool wide_dstage_t(Ctx *c, const double *rin, int nrhs, bool trans, double *x, int64_t ldx, bool acc) {
    const int W = c->W, NB = c->NBW, p = c->p, tz = c->tsize;
    const int64_t WW = (int64_t)W * W, sF = NB * WW, PS = c->PS, sV = PS * VP;
    Parts P{c->off_d, c->boff_d, p};
    const dim3 grid((unsigned)((PS + 255) / 256), p);
    const double *inv = c->nrm + 2 * c->opt.max_nrhs;
    if (!launch(c, KID_WIDE_VEC, [&] {
            if (trans)
                k_wide_pack_t<T><<<grid, 256, 0, c->stream>>>(rin, inv, c->zr, (const T *)c->PQ, W, P, c->k, c->r,
                                                              c->n, PS, nrhs, (T *)c->WV1);
            else
                k_wide_pack<T><<<grid, 256, 0, c->stream>>>(rin, inv, c->n, P, PS, nrhs, (T *)c->WV1);
        }))
        return false;
    auto v1 = [&](int J) { return at(c->WV1, (int64_t)J * W, tz); };
    auto v2 = [&](int J) { return at(c->WV2, (int64_t)J * W, tz); };
    auto tile = [&](void *base, int J) { return at(base, J * WW, tz); };
    // forward: y_J = L_JJ^{-1}(b_J - L_{J,J-1} y_{J-1})   (transposed: U^T)
    void *Lo = trans ? c->WZ : c->WY, *Di = trans ? c->WUi : c->WLi;
    for (int J = 0; J < NB; ++J) {
        if (J > 0 && !gemm(c, trans, false, W, nrhs, W, -1.0, tile(Lo, J - 1), W, sF, v2(J - 1), (int)PS, sV, 1.0,
                           v1(J), (int)PS, sV, p))
            return false;
        if (!gemm(c, trans, false, W, nrhs, W, 1.0, tile(Di, J), W, sF, v1(J), (int)PS, sV, 0.0, v2(J), (int)PS, sV, p))
            return false;
    }
    // backward: x_J = U_JJ^{-1}(y_J - U_{J,J+1} x_{J+1})   (transposed: L^T)
    void *Up = trans ? c->WY : c->WZ, *Dj = trans ? c->WLi : c->WUi;
    for (int J = NB - 1; J >= 0; --J) {
        if (J < NB - 1 && !gemm(c, trans, false, W, nrhs, W, -1.0, tile(Up, J), W, sF, v1(J + 1), (int)PS, sV, 1.0,
                                v2(J), (int)PS, sV, p))
            return false;
        if (!gemm(c, trans, false, W, nrhs, W, 1.0, tile(Dj, J), W, sF, v2(J), (int)PS, sV, 0.0, v1(J), (int)PS, sV, p))
            return false;
    }
    if (trans)
        return launch(c, KID_WIDE_VEC, [&] {
            k_wide_unpack_t<T><<<grid, 256, 0, c->stream>>>((const T *)c->WV1, c->nrm + c->opt.max_nrhs, P, PS, nrhs,
                                                            x, ldx, acc ? 1 : 0);
        });
    if (!launch(c, KID_WIDE_VEC, [&] {
            k_wide_unpack<T><<<grid, 256, 0, c->stream>>>((const T *)c->WV1, c->n, P, PS, nrhs, (T *)c->Gv);
        }))
        return false;
    if (p < 2 || c->r == 0) return true;
    return launch(c, KID_WIDE_VEC, [&] {
        k_wide_psi<T><<<p, 256, 0, c->stream>>>((const T *)c->Gv, (const T *)c->PQ, W, P, c->k, c->r, c->n, nrhs,
                                                 c->psi);
    });
}

bool run_wide_dstage(Ctx *c, const double *rin, int nrhs) {
    return c->fp64 ? wide_dstage_t<double>(c, rin, nrhs, false, nullptr, 0, false)
                   : wide_dstage_t<float>(c, rin, nrhs, false, nullptr, 0, false);
}

bool run_wide_dstage_t(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, bool accumulate) {
    return c->fp64 ? wide_dstage_t<double>(c, hin, nrhs, true, x, ldx, accumulate)
                   : wide_dstage_t<float>(c, hin, nrhs, true, x, ldx, accumulate);
}

}  // namespace lrs
