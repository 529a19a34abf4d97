// The reduced system of the low-rank spike matrix (paper section 3.2), FP64.
//
// Unknowns per interface i = 0..p-2 (between partitions i and i+1):
//   z_i = [zeta_i ; omega_{i+1}],  zeta_i = P_i x_{i+1,t},  omega_{i+1} = Q_{i+1} x_{i,b}
// (the r-vectors that the paper exchanges instead of k-row tips).  With
// x_j = g_j - u_{T,j} zeta_j - u_{W,j} omega_j (low-rank recovery) the
// reduced matrix R = I + V U is block tridiagonal with 2r x 2r blocks
//   E_i = [[I, P_i u_{W,i+1}^t], [Q_{i+1} u_{T,i}^b, I]]      (diagonal)
//   F_i = [[P_i u_{T,i+1}^t, 0], [0, 0]]                      (couples z_{i+1})
//   G_i = [[0, 0], [0, Q_{i+1} u_{W,i}^b]]                    (couples z_{i-1})
// TRUNCATED (LR-SPIKE-T, S~~_r of eq. 'red_sys_prec_mid_2') keeps E_i only:
// the paper drops the top tip of T~ and the bottom tip of W~, which are
// exactly F and G here.  FULL keeps all blocks (the reduced system of
// LR-SPIKE-I, here solved directly by block cyclic reduction, below).
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrs {

template <typename T>
__global__ void k_red_build(const T *__restrict__ PQ, int KB, const T *__restrict__ Ucat, Parts P, int k,
                            int r, double *__restrict__ E, double *__restrict__ F,
                            double *__restrict__ Gs) {
    const int i = blockIdx.x;
    const int n2 = 2 * r;
    const int64_t sn = P.off[i + 1];
    const T *Pi = PQ + ((int64_t)i * 2 + 0) * r * KB;          // P_i
    const T *Qn = PQ + ((int64_t)(i + 1) * 2 + 1) * r * KB;    // Q_{i+1}
    double *e = E + (int64_t)i * n2 * n2, *f = F + (int64_t)i * n2 * n2, *g = Gs + (int64_t)i * n2 * n2;
    const bool hasF = (i + 1 <= P.p - 2), hasG = (i >= 1);
    for (int t = threadIdx.x; t < n2 * n2; t += blockDim.x) {
        const int a = t / n2, b = t % n2;
        double ev = (a == b) ? 1.0 : 0.0, fv = 0.0, gv = 0.0;
        if (a < r && b >= r) {            // P_i u_{W,i+1}^t
            for (int q = 0; q < k; ++q) ev += (double)Pi[a * KB + q] * (double)Ucat[(sn + q) * n2 + b];
        } else if (a >= r && b < r) {     // Q_{i+1} u_{T,i}^b
            for (int q = 0; q < k; ++q)
                ev += (double)Qn[(a - r) * KB + q] * (double)Ucat[(sn - k + q) * n2 + b];
        }
        if (hasF && a < r && b < r)       // P_i u_{T,i+1}^t
            for (int q = 0; q < k; ++q) fv += (double)Pi[a * KB + q] * (double)Ucat[(sn + q) * n2 + b];
        if (hasG && a >= r && b >= r)     // Q_{i+1} u_{W,i}^b
            for (int q = 0; q < k; ++q)
                gv += (double)Qn[(a - r) * KB + q] * (double)Ucat[(sn - k + q) * n2 + b];
        e[t] = ev;
        f[t] = fv;
        g[t] = gv;
    }
}

// The same blocks with the operands staged in shared memory first (P_i,
// Q_{i+1}, the top k rows of u of partition i+1 and the bottom k rows of
// partition i, as doubles): every entry sums the same terms in the same order
// as k_red_build, but reads shared memory instead of strided global loads.
template <typename T>
__global__ void k_red_build_s(const T *__restrict__ PQ, int KB, const T *__restrict__ Ucat, Parts P, int k,
                              int r, double *__restrict__ E, double *__restrict__ F,
                              double *__restrict__ Gs) {
    extern __shared__ double sb[];
    const int i = blockIdx.x;
    const int n2 = 2 * r;
    const int64_t sn = P.off[i + 1];
    double *Ps = sb, *Qs = Ps + r * k, *Ut = Qs + r * k, *Ub = Ut + k * n2;  // [r][k] [r][k] [k][n2] [k][n2]
    const T *Pi = PQ + ((int64_t)i * 2 + 0) * r * KB;
    const T *Qn = PQ + ((int64_t)(i + 1) * 2 + 1) * r * KB;
    for (int e = threadIdx.x; e < r * k; e += blockDim.x) {
        const int a = e / k, q = e % k;
        Ps[e] = (double)Pi[a * KB + q];
        Qs[e] = (double)Qn[a * KB + q];
    }
    for (int e = threadIdx.x; e < k * n2; e += blockDim.x) {
        const int q = e / n2, b = e % n2;
        Ut[e] = (double)Ucat[(sn + q) * n2 + b];
        Ub[e] = (double)Ucat[(sn - k + q) * n2 + b];
    }
    __syncthreads();
    double *e_ = E + (int64_t)i * n2 * n2, *f = F + (int64_t)i * n2 * n2, *g = Gs + (int64_t)i * n2 * n2;
    const bool hasF = (i + 1 <= P.p - 2), hasG = (i >= 1);
    for (int t = threadIdx.x; t < n2 * n2; t += blockDim.x) {
        const int a = t / n2, b = t % n2;
        double ev = (a == b) ? 1.0 : 0.0, fv = 0.0, gv = 0.0;
        if (a < r && b >= r) {            // P_i u_{W,i+1}^t
            for (int q = 0; q < k; ++q) ev += Ps[a * k + q] * Ut[q * n2 + b];
        } else if (a >= r && b < r) {     // Q_{i+1} u_{T,i}^b
            for (int q = 0; q < k; ++q) ev += Qs[(a - r) * k + q] * Ub[q * n2 + b];
        }
        if (hasF && a < r && b < r)       // P_i u_{T,i+1}^t
            for (int q = 0; q < k; ++q) fv += Ps[a * k + q] * Ut[q * n2 + b];
        if (hasG && a >= r && b >= r)     // Q_{i+1} u_{W,i}^b
            for (int q = 0; q < k; ++q) gv += Qs[(a - r) * k + q] * Ub[q * n2 + b];
        e_[t] = ev;
        f[t] = fv;
        g[t] = gv;
    }
}

// In-place inverse of the n x n matrix in Ms (row stride n) by Gauss-Jordan
// elimination with partial pivoting on [M | I]; aug has room for n x 2n.
// Returns false (to thread 0) on a zero pivot.
__device__ bool gj_inverse(double *aug, int n, double *fac, int *pivrow) {
    const int w = 2 * n;
    bool ok = true;
    for (int c = 0; c < n; ++c) {
        if (threadIdx.x == 0) {
            int best = c;
            for (int i = c + 1; i < n; ++i)
                if (fabs(aug[i * w + c]) > fabs(aug[best * w + c])) best = i;
            *pivrow = best;
        }
        __syncthreads();
        const int pr = *pivrow;
        if (pr != c)
            for (int j = threadIdx.x; j < w; j += blockDim.x) {
                const double t = aug[c * w + j];
                aug[c * w + j] = aug[pr * w + j];
                aug[pr * w + j] = t;
            }
        __syncthreads();
        const double piv = aug[c * w + c];
        if (piv == 0.0 || !isfinite(piv)) ok = false;
        const double pinv = (piv == 0.0) ? 1.0 : 1.0 / piv;
        for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = aug[i * w + c];
        __syncthreads();
        for (int j = threadIdx.x; j < w; j += blockDim.x) aug[c * w + j] *= pinv;
        __syncthreads();
        for (int t = threadIdx.x; t < n * w; t += blockDim.x) {
            const int i = t / w, j = t % w;
            if (i != c) aug[t] -= fac[i] * aug[c * w + j];
        }
        __syncthreads();
    }
    return ok;
}

__device__ void load_aug(double *aug, const double *M, int n) {
    const int w = 2 * n;
    for (int t = threadIdx.x; t < n * w; t += blockDim.x) {
        const int i = t / w, j = t % w;
        aug[t] = (j < n) ? M[i * n + j] : ((j - n == i) ? 1.0 : 0.0);
    }
    __syncthreads();
}

__device__ void store_inv(const double *aug, double *out, int n) {
    const int w = 2 * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) out[t] = aug[(t / n) * w + n + t % n];
}

__global__ void k_red_factor_trunc(const double *__restrict__ E, int n2, double *__restrict__ Rinv,
                                   int64_t *status) {
    extern __shared__ double sm[];
    double *aug = sm, *fac = aug + 2 * n2 * n2;
    __shared__ int pivrow;
    const int i = blockIdx.x;
    load_aug(aug, E + (int64_t)i * n2 * n2, n2);
    const bool ok = gj_inverse(aug, n2, fac, &pivrow);
    if (!ok && threadIdx.x == 0) atomicMin((unsigned long long *)status, 0x7ffffffffffffffeULL);
    store_inv(aug, Rinv + (int64_t)i * n2 * n2, n2);
}

// The same inverse for blocks too large for [E | I] in shared memory (2r >
// 64): Gauss-Jordan in place with partial pivoting.  Step c exchanges rows c
// and the pivot row, scales row c (its diagonal becomes 1 / pivot) and
// eliminates column c from every other row (column c then holds the
// multiples of the eliminated identity column); the row exchanges are undone
// at the end as column exchanges in reverse order.  Shared memory: n2^2 + n2
// doubles (129 KB at 2r = 128).
__global__ void k_red_factor_trunc_ip(const double *__restrict__ E, int n2, double *__restrict__ Rinv,
                                      int64_t *status) {
    extern __shared__ double sm[];
    double *a = sm, *fac = a + n2 * n2;
    __shared__ int perm[128];
    __shared__ int pivrow;
    const int blk = blockIdx.x;
    const double *e = E + (int64_t)blk * n2 * n2;
    for (int t = threadIdx.x; t < n2 * n2; t += blockDim.x) a[t] = e[t];
    __syncthreads();
    bool ok = true;
    for (int c = 0; c < n2; ++c) {
        if (threadIdx.x == 0) {
            int best = c;
            for (int i = c + 1; i < n2; ++i)
                if (fabs(a[i * n2 + c]) > fabs(a[best * n2 + c])) best = i;
            pivrow = best;
            perm[c] = best;
        }
        __syncthreads();
        const int pr = pivrow;
        if (pr != c)
            for (int j = threadIdx.x; j < n2; j += blockDim.x) {
                const double t = a[c * n2 + j];
                a[c * n2 + j] = a[pr * n2 + j];
                a[pr * n2 + j] = t;
            }
        __syncthreads();
        const double piv = a[c * n2 + c];
        if (piv == 0.0 || !isfinite(piv)) ok = false;
        const double pinv = (piv == 0.0) ? 1.0 : 1.0 / piv;
        for (int i = threadIdx.x; i < n2; i += blockDim.x) fac[i] = a[i * n2 + c];
        __syncthreads();
        for (int j = threadIdx.x; j < n2; j += blockDim.x) a[c * n2 + j] = (j == c) ? pinv : a[c * n2 + j] * pinv;
        __syncthreads();
        for (int t = threadIdx.x; t < n2 * n2; t += blockDim.x) {
            const int i = t / n2, j = t % n2;
            if (i == c) continue;
            a[t] = (j == c) ? -fac[i] * pinv : a[t] - fac[i] * a[c * n2 + j];
        }
        __syncthreads();
    }
    for (int c = n2 - 1; c >= 0; --c) {
        const int pc = perm[c];
        if (pc != c)
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const double t = a[i * n2 + c];
                a[i * n2 + c] = a[i * n2 + pc];
                a[i * n2 + pc] = t;
            }
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) atomicMin((unsigned long long *)status, 0x7ffffffffffffffeULL);
    double *out = Rinv + (int64_t)blk * n2 * n2;
    for (int t = threadIdx.x; t < n2 * n2; t += blockDim.x) out[t] = a[t];
}

// z = R^{-1} psi (or R^{-T} psi), TRUNCATED: per interface.
__global__ void k_red_solve_trunc(const double *__restrict__ Rinv, const double *__restrict__ psi,
                                  double *__restrict__ z, int n2, int nrhs, int trans) {
    const int i = blockIdx.x;
    const double *M = Rinv + (int64_t)i * n2 * n2;
    const double *v = psi + (int64_t)i * n2 * nrhs;
    double *o = z + (int64_t)i * n2 * nrhs;
    for (int t = threadIdx.x; t < n2 * nrhs; t += blockDim.x) {
        const int a = t / nrhs, c = t % nrhs;
        double acc = 0.0;
        for (int q = 0; q < n2; ++q) acc += (trans ? M[q * n2 + a] : M[a * n2 + q]) * v[q * nrhs + c];
        o[t] = acc;
    }
}

// ---------------------------------------------------------------------------
// FULL reduced system by block cyclic reduction (log2(p) levels instead of a
// chain over the p-1 interfaces).  At level l (h = 2^l) the equations
// i = 2h(j+1) - 1 are kept and their neighbours i -+ h eliminated:
//   alpha_i = G_i E_{i-h}^{-1},  beta_i = F_i E_{i+h}^{-1}
//   E_i <- E_i - alpha_i F_{i-h} - beta_i G_{i+h}
//   G_i <- -alpha_i G_{i-h},  F_i <- -beta_i F_{i+h}   (now coupling i -+ 2h)
// until one equation (i = 2^L - 1) is left.  The solve reduces the right-hand
// side the same way (w_i -= alpha_i w_{i-h} + beta_i w_{i+h}), solves the last
// equation, and back-substitutes level by level
//   z_i = E_i^{-1} (w_i - G_i z_{i-h} - F_i z_{i+h})   for the eliminated i.
// R^T is reduced the same way from its own blocks (diagonal E_i^T, super
// G_{i+1}^T, sub F_{i-1}^T).  Blocks row-major n2 x n2, FP64.

// working copies of the blocks of R (trans = 0) or R^T (trans = 1)
__global__ void k_bcr_copy(const double *__restrict__ E, const double *__restrict__ F,
                           const double *__restrict__ Gs, int m, int n2, int trans, double *__restrict__ oE,
                           double *__restrict__ oF, double *__restrict__ oG) {
    const int i = blockIdx.x, nn = n2 * n2;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int a = t / n2, b = t % n2, tt = b * n2 + a;
        if (!trans) {
            oE[(int64_t)i * nn + t] = E[(int64_t)i * nn + t];
            oF[(int64_t)i * nn + t] = F[(int64_t)i * nn + t];
            oG[(int64_t)i * nn + t] = Gs[(int64_t)i * nn + t];
        } else {
            oE[(int64_t)i * nn + t] = E[(int64_t)i * nn + tt];
            oF[(int64_t)i * nn + t] = (i + 1 < m) ? Gs[(int64_t)(i + 1) * nn + tt] : 0.0;
            oG[(int64_t)i * nn + t] = (i >= 1) ? F[(int64_t)(i - 1) * nn + tt] : 0.0;
        }
    }
}

// Einv_i = E_i^{-1} for i = first + j stride, j < count (Gauss-Jordan in
// shared memory with partial pivoting)
__global__ void k_bcr_invert(const double *__restrict__ E, double *__restrict__ Einv, int n2, int first, int stride,
                             int64_t *status) {
    extern __shared__ double sm[];
    double *aug = sm, *fac = aug + 2 * n2 * n2;
    __shared__ int pivrow;
    const int i = first + blockIdx.x * stride, nn = n2 * n2;
    load_aug(aug, E + (int64_t)i * nn, n2);
    const bool ok = gj_inverse(aug, n2, fac, &pivrow);
    if (!ok && threadIdx.x == 0) atomicMin((unsigned long long *)status, 0x7ffffffffffffffeULL);
    store_inv(aug, Einv + (int64_t)i * nn, n2);
}

// one level of the reduction for the kept equation i = 2h(j+1) - 1: CTA
// (j, y) forms rows [y RB, y RB + RB) of alpha_i, beta_i and of the new E_i,
// G_i, F_i (each row of the update needs only that row of alpha and beta)
constexpr int BCR_RB = 8;
__global__ void k_bcr_reduce(double *__restrict__ E, double *__restrict__ F, double *__restrict__ G,
                             const double *__restrict__ Einv, double *__restrict__ al, double *__restrict__ be,
                             int m, int n2, int h) {
    extern __shared__ double sm[];
    const int j = blockIdx.x, i = 2 * h * (j + 1) - 1, lo = i - h, hi = i + h, nn = n2 * n2;
    const int r0 = blockIdx.y * BCR_RB, nr = min(BCR_RB, n2 - r0);
    const bool has_hi = hi < m;
    double *A = sm, *B = sm + BCR_RB * n2;  // rows r0.. of alpha, beta
    for (int t = threadIdx.x; t < nr * n2; t += blockDim.x) {
        const int a = r0 + t / n2, b = t % n2;
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < n2; ++q) {
            sa += G[(int64_t)i * nn + a * n2 + q] * Einv[(int64_t)lo * nn + q * n2 + b];
            if (has_hi) sb += F[(int64_t)i * nn + a * n2 + q] * Einv[(int64_t)hi * nn + q * n2 + b];
        }
        A[t] = sa;
        B[t] = sb;
        al[(int64_t)j * nn + a * n2 + b] = sa;
        be[(int64_t)j * nn + a * n2 + b] = sb;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * n2; t += blockDim.x) {
        const int ra = t / n2, a = r0 + ra, b = t % n2;
        double e = E[(int64_t)i * nn + a * n2 + b], g = 0.0, f = 0.0;
        for (int q = 0; q < n2; ++q) {
            e -= A[ra * n2 + q] * F[(int64_t)lo * nn + q * n2 + b];
            g -= A[ra * n2 + q] * G[(int64_t)lo * nn + q * n2 + b];
            if (has_hi) {
                e -= B[ra * n2 + q] * G[(int64_t)hi * nn + q * n2 + b];
                f -= B[ra * n2 + q] * F[(int64_t)hi * nn + q * n2 + b];
            }
        }
        E[(int64_t)i * nn + a * n2 + b] = e;
        G[(int64_t)i * nn + a * n2 + b] = g;
        F[(int64_t)i * nn + a * n2 + b] = f;
    }
}

// w_i -= alpha_i w_{i-h} + beta_i w_{i+h} for the kept i = 2h(j+1) - 1 (CTA j);
// w in the psi layout [m][n2][nrhs]
__global__ void k_bcr_fwd(const double *__restrict__ al, const double *__restrict__ be, double *__restrict__ w,
                          int m, int n2, int h, int nrhs) {
    const int j = blockIdx.x, i = 2 * h * (j + 1) - 1, lo = i - h, hi = i + h, nn = n2 * n2, nv = n2 * nrhs;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const int a = t / nrhs, c = t % nrhs;
        double acc = w[(int64_t)i * nv + t];
        for (int q = 0; q < n2; ++q) {
            acc -= al[(int64_t)j * nn + a * n2 + q] * w[(int64_t)lo * nv + q * nrhs + c];
            if (hi < m) acc -= be[(int64_t)j * nn + a * n2 + q] * w[(int64_t)hi * nv + q * nrhs + c];
        }
        w[(int64_t)i * nv + t] = acc;
    }
}

// z_i = E_i^{-1} (w_i - G_i z_{i-h} - F_i z_{i+h}) for the eliminated
// i = h (2j+1) - 1 (CTA j); the last equation (h = 0 marks it) has no neighbours
__global__ void k_bcr_bwd(const double *__restrict__ Einv, const double *__restrict__ F,
                          const double *__restrict__ G, const double *__restrict__ w, double *__restrict__ z, int m,
                          int n2, int h, int top, int nrhs) {
    extern __shared__ double tv[];  // [n2][nrhs]
    const int j = blockIdx.x, i = h ? h * (2 * j + 1) - 1 : top, nn = n2 * n2, nv = n2 * nrhs;
    const int lo = i - h, hi = i + h;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const int a = t / nrhs, c = t % nrhs;
        double acc = w[(int64_t)i * nv + t];
        if (h)
            for (int q = 0; q < n2; ++q) {
                if (lo >= 0) acc -= G[(int64_t)i * nn + a * n2 + q] * z[(int64_t)lo * nv + q * nrhs + c];
                if (hi < m) acc -= F[(int64_t)i * nn + a * n2 + q] * z[(int64_t)hi * nv + q * nrhs + c];
            }
        tv[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const int a = t / nrhs, c = t % nrhs;
        double acc = 0.0;
        for (int q = 0; q < n2; ++q) acc += Einv[(int64_t)i * nn + a * n2 + q] * tv[q * nrhs + c];
        z[(int64_t)i * nv + t] = acc;
    }
}

// levels of the reduction of m equations: kept and eliminated counts
struct BcrLevels {
    std::vector<int> kept, elim;
    int top = 0;
};
static BcrLevels bcr_levels(int m) {
    BcrLevels L;
    int h = 1;
    while (m / h > 1) {
        L.kept.push_back(m / (2 * h));
        int e = 0;
        for (int64_t i = h - 1; i < m; i += 2 * h) ++e;
        L.elim.push_back(e);
        h *= 2;
    }
    L.top = h - 1;
    return L;
}

// set 0 reduces R, set 1 R^T
static bool bcr_factor(Ctx *c, int t) {
    const int n2 = 2 * c->r, m = c->p - 1;
    const size_t nn = (size_t)n2 * n2;
    const BcrLevels L = bcr_levels(m);
    const size_t inv_smem = (2 * nn + n2) * sizeof(double), red_smem = 2 * BCR_RB * n2 * sizeof(double);
    cudaFuncSetAttribute(k_bcr_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem);
    {
        auto &b = c->bcr[t];
        if (!launch(c, KID_RED_FACTOR, [&] {
                k_bcr_copy<<<m, 256, 0, c->stream>>>(c->E, c->F, c->Gs, m, n2, t, b.E, b.F, b.G);
            }))
            return false;
        size_t off = 0;
        for (size_t l = 0; l < L.kept.size(); ++l) {
            const int h = 1 << l;
            if (!launch(c, KID_RED_FACTOR, [&] {
                    k_bcr_invert<<<L.elim[l], 256, inv_smem, c->stream>>>(b.E, b.Einv, n2, h - 1, 2 * h, c->status);
                }))
                return false;
            if (L.kept[l] > 0 && !launch(c, KID_RED_FACTOR, [&] {
                    k_bcr_reduce<<<dim3(L.kept[l], (n2 + BCR_RB - 1) / BCR_RB), 256, red_smem, c->stream>>>(
                        b.E, b.F, b.G, b.Einv, b.al + off * nn, b.be + off * nn, m, n2, h);
                }))
                return false;
            off += L.kept[l];
        }
        if (!launch(c, KID_RED_FACTOR, [&] {
                k_bcr_invert<<<1, 256, inv_smem, c->stream>>>(b.E, b.Einv, n2, L.top, 1, c->status);
            }))
            return false;
    }
    return true;
}

static bool bcr_solve(Ctx *c, int nrhs, bool trans) {
    const int n2 = 2 * c->r, m = c->p - 1;
    const size_t nn = (size_t)n2 * n2, nv = (size_t)n2 * nrhs;
    const BcrLevels L = bcr_levels(m);
    // R^T is reduced the first time a transposed solve needs it
    if (trans && !c->bcr_t_ready) {
        if (!bcr_factor(c, 1)) return false;
        c->bcr_t_ready = true;
    }
    auto &b = c->bcr[trans ? 1 : 0];
    if (cudaMemcpyAsync(c->wr, c->psi, (size_t)m * nv * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        c->err = "reduced right-hand side copy failed";
        return false;
    }
    size_t off = 0;
    std::vector<size_t> offs;
    for (size_t l = 0; l < L.kept.size(); ++l) {
        offs.push_back(off);
        if (L.kept[l] > 0 && !launch(c, KID_RED_SOLVE, [&] {
                k_bcr_fwd<<<L.kept[l], 128, 0, c->stream>>>(b.al + off * nn, b.be + off * nn, c->wr, m, n2, 1 << l,
                                                          nrhs);
            }))
            return false;
        off += L.kept[l];
    }
    const size_t smem = nv * sizeof(double);
    if (!launch(c, KID_RED_SOLVE, [&] {
            k_bcr_bwd<<<1, 128, smem, c->stream>>>(b.Einv, b.F, b.G, c->wr, c->zr, m, n2, 0, L.top, nrhs);
        }))
        return false;
    for (int l = (int)L.kept.size() - 1; l >= 0; --l)
        if (!launch(c, KID_RED_SOLVE, [&] {
                k_bcr_bwd<<<L.elim[l], 128, smem, c->stream>>>(b.Einv, b.F, b.G, c->wr, c->zr, m, n2, 1 << l, 0,
                                                               nrhs);
            }))
            return false;
    return true;
}

// ldpq: row stride of the projections P_i, Q_i (the block size)
template <typename T>
static bool build_impl(Ctx *c, int ldpq) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (size_t)(2 * c->r * c->k + 4 * c->k * c->r) * sizeof(double);
    if (smem <= 96 * 1024) {
        cudaFuncSetAttribute(k_red_build_s<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch(c, KID_RED_BUILD, [&] {
            k_red_build_s<T><<<c->p - 1, 256, smem, c->stream>>>((const T *)c->PQ, ldpq, (const T *)c->Ucat, P,
                                                                 c->k, c->r, c->E, c->F, c->Gs);
        });
    }
    return launch(c, KID_RED_BUILD, [&] {
        k_red_build<T><<<c->p - 1, 256, 0, c->stream>>>((const T *)c->PQ, ldpq, (const T *)c->Ucat, P, c->k,
                                                        c->r, c->E, c->F, c->Gs);
    });
}

bool run_reduced_build_ld(Ctx *c, int ldpq) {
    if (c->p < 2 || c->r == 0) return true;
    return c->fp64 ? build_impl<double>(c, ldpq) : build_impl<float>(c, ldpq);
}

bool run_reduced_build(Ctx *c) { return run_reduced_build_ld(c, c->KB); }

bool run_reduced_factor(Ctx *c) {
    if (c->p < 2 || c->r == 0) return true;
    const int n2 = 2 * c->r, ni = c->p - 1;
    if (c->opt.reduced == LRSPIKE_REDUCED_TRUNCATED && n2 > 64) {
        const size_t smem = (size_t)(n2 * n2 + n2) * sizeof(double);
        cudaFuncSetAttribute(k_red_factor_trunc_ip, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch(c, KID_RED_FACTOR, [&] {
            k_red_factor_trunc_ip<<<ni, 256, smem, c->stream>>>(c->E, n2, c->Rinv, c->status);
        });
    }
    if (c->opt.reduced == LRSPIKE_REDUCED_TRUNCATED) {
        const size_t smem = (2 * n2 * n2 + n2) * sizeof(double);
        cudaFuncSetAttribute(k_red_factor_trunc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch(c, KID_RED_FACTOR, [&] {
            k_red_factor_trunc<<<ni, 256, smem, c->stream>>>(c->E, n2, c->Rinv, c->status);
        });
    }
    (void)ni;
    // a graph-safe handle reduces both now (a captured transposed solve must
    // not depend on host state); others reduce R^T on first use
    c->bcr_t_ready = c->opt.graph_safe != 0;
    return bcr_factor(c, 0) && (!c->opt.graph_safe || bcr_factor(c, 1));
}

bool run_reduced_solve(Ctx *c, int nrhs, bool trans) {
    if (c->p < 2 || c->r == 0) return true;
    const int n2 = 2 * c->r, ni = c->p - 1;
    if (c->opt.reduced == LRSPIKE_REDUCED_TRUNCATED)
        return launch(c, KID_RED_SOLVE, [&] {
            k_red_solve_trunc<<<ni, 128, 0, c->stream>>>(c->Rinv, c->psi, c->zr, n2, nrhs, trans);
        });
    return bcr_solve(c, nrhs, trans);
}

}  // namespace lrs
