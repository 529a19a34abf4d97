// Right-preconditioned BiCGStab outer iteration (van der Vorst), FP64 vectors,
// with the LR-SPIKE operator M^{-1} (or M^{-T}) as the preconditioner
// (paper section 4: the preconditioned Krylov solver around LR-SPIKE; one
// iteration applies the preconditioner twice).
//
// All nrhs columns iterate together, each with its own scalars.  The scalars
// live on the device and are formed by the kernels that need them, so an
// iteration needs one host synchronisation (the convergence test).  A column
// that has converged is frozen by a mask: its x and r are no longer written.
//
// Per iteration (column q, tilde r the fixed shadow residual):
//   beta  = (rho_new / rho) (alpha / omega)
//   p     = r + beta (p - omega v)                       k_bicg_p
//   ph    = M^{-1} p                                     preconditioner
//   v     = A ph,  rhv = tilde r . v                     k_bicg_mv<0>
//   alpha = rho_new / rhv;  s = r - alpha v              k_bicg_s
//   sh    = M^{-1} s                                     preconditioner
//   t     = A sh,  t.s,  t.t                             k_bicg_mv<1>
//   omega = t.s / t.t  (0 once |s| <= tol |f|: the early exit x += alpha ph)
//   x    += alpha ph + omega sh;  r = s - omega t;  rho = rho_new;
//   rho_new = tilde r . r,  |r|^2                        k_bicg_update
// Every sum over rows is reduced deterministically: per-CTA partials, added in
// CTA order by the last CTA of the launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrs {

namespace {

constexpr int VBS = 256;          // threads per CTA
constexpr int kMaxCtas = 152 * 8;  // grid-stride cap: 8 CTAs on each of the 152 SMs

// rows of the device scalar array (each row holds max_nrhs doubles)
enum Scalar { S_RHO = 0, S_ALPHA, S_OMEGA, S_RHO_NEW, S_RHV, S_TS, S_TT, S_SS, S_RR, S_BB, S_ACTIVE, S_RESTART,
              S_ROWS };

inline unsigned vgrid(int64_t n) {
    return (unsigned)std::min<int64_t>((n + VBS - 1) / VBS, kMaxCtas);
}

// Adds the first nv of NV per-thread values over the whole grid (nv <= 32).  Returns true in the last CTA
// to finish (all of its threads), with the totals in tot[]; other CTAs get
// false.  Partials are added in CTA order, so the sums are reproducible.
template <int NV>
__device__ __forceinline__ bool grid_sums(const double (&v)[NV], int nv, double *partial, unsigned *counter, double *tot) {
    __shared__ double red[NV][VBS / 32];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double s = warp_sum(v[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double t = 0.0;
        for (int w = 0; w < VBS / 32; ++w) t += red[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * nv + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // thread (q, g) adds the partials of CTAs g, g + G, ... for quantity q;
    // then the G group sums of each q are added in order by one thread
    __shared__ double grp[VBS];
    const int G = VBS / nv;  // nv <= 32, so G >= 8
    const int q = threadIdx.x % nv, g = threadIdx.x / nv;
    double t = 0.0;
    if (g < G)
        for (unsigned b = g; b < gridDim.x; b += G) t += __ldcg(&partial[(int64_t)b * nv + q]);
    grp[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int j = 0; j < G; ++j) s += grp[j * nv + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
    __syncthreads();
    return true;
}

__device__ __forceinline__ double safe_div(double a, double b) { return (b != 0.0) ? a / b : 0.0; }

// r = r0, tilde r = r0, p = v = 0 for the columns flagged in S_RESTART;
// rho = alpha = omega = 1, rho_new = |r0|^2, |r|^2 for those columns.
template <int NR>
__global__ void __launch_bounds__(VBS)
    k_bicg_restart(const double *__restrict__ r0, int64_t n, int nrhs, int mx, double *__restrict__ r,
                   double *__restrict__ rh, double *__restrict__ pv, double *__restrict__ vv, double *sc,
                   double *partial, unsigned *counter) {
    double ss[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) ss[q] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)VBS + threadIdx.x; i < n; i += (int64_t)gridDim.x * VBS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            if (q >= nrhs || sc[S_RESTART * mx + q] == 0.0) continue;
            const double a = r0[q * n + i];
            r[q * n + i] = a;
            rh[q * n + i] = a;
            pv[q * n + i] = 0.0;
            vv[q * n + i] = 0.0;
            ss[q] += a * a;
        }
    }
    __shared__ double tot[NR];
    if (grid_sums<NR>(ss, nrhs, partial, counter, tot) && threadIdx.x < nrhs) {
        const int q = threadIdx.x;
        if (sc[S_RESTART * mx + q] != 0.0) {
            sc[S_RHO * mx + q] = 1.0;
            sc[S_ALPHA * mx + q] = 1.0;
            sc[S_OMEGA * mx + q] = 1.0;
            sc[S_RHO_NEW * mx + q] = tot[q];
            sc[S_RR * mx + q] = tot[q];
        }
    }
}

// p = r + beta (p - omega v); |p| and 1/|p| into nrm (the preconditioner's
// input scale).  Frozen columns get p = 0.
template <int NR>
__global__ void __launch_bounds__(VBS)
    k_bicg_p(const double *__restrict__ r, const double *__restrict__ vv, double *__restrict__ pv, int64_t n,
             int nrhs, int mx, const double *__restrict__ sc, double *nrm, double *inv, double *partial,
             unsigned *counter) {
    double beta[NR], om[NR], act[NR], ss[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        ss[q] = 0.0;
        act[q] = 0.0;
        beta[q] = om[q] = 0.0;
        if (q < nrhs) {
            act[q] = sc[S_ACTIVE * mx + q];
            om[q] = sc[S_OMEGA * mx + q];
            beta[q] = safe_div(sc[S_RHO_NEW * mx + q], sc[S_RHO * mx + q]) * safe_div(sc[S_ALPHA * mx + q], om[q]);
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)VBS + threadIdx.x; i < n; i += (int64_t)gridDim.x * VBS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            if (q >= nrhs) continue;
            const int64_t e = q * n + i;
            const double a = (act[q] != 0.0) ? r[e] + beta[q] * (pv[e] - om[q] * vv[e]) : 0.0;
            pv[e] = a;
            ss[q] += a * a;
        }
    }
    __shared__ double tot[NR];
    if (grid_sums<NR>(ss, nrhs, partial, counter, tot) && threadIdx.x < nrhs) {
        const double nv = sqrt(tot[threadIdx.x]);
        nrm[threadIdx.x] = nv;
        inv[threadIdx.x] = (nv > 0.0) ? 1.0 / nv : 0.0;
    }
}

// y = A u (or A^T u) from the FP64 band, with MODE 0: tilde r . y -> S_RHV;
// MODE 1: y . s -> S_TS and y . y -> S_TT.
template <int NR, int MODE>
__global__ void __launch_bounds__(VBS)
    k_bicg_mv(const double *__restrict__ band, int64_t ldb, int k, int64_t n, int trans,
              const double *__restrict__ u, double *__restrict__ y, const double *__restrict__ w, int nrhs,
              int mx, double *sc, double *partial, unsigned *counter, const int *__restrict__ dlist, int ndl) {
    constexpr int NV = (MODE == 0) ? NR : 2 * NR;
    double dv[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) dv[q] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)VBS + threadIdx.x; i < n; i += (int64_t)gridDim.x * VBS) {
        double acc[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = 0.0;
        const int t0 = (int)max((int64_t)0, k - i), t1 = (int)min((int64_t)2 * k, n - 1 - i + k);
        // with a list of the band rows that hold nonzeros only those are visited
        const int nt = dlist ? ndl : t1 - t0 + 1;
        for (int it = 0; it < nt; ++it) {
            const int t = dlist ? (trans ? dlist[it] : 2 * k - dlist[it]) : t0 + it;
            if (t < t0 || t > t1) continue;
            const int64_t j = i - k + t;
            // A[i][j] = band[(k+i-j) ldb + j];  A^T[i][j] = A[j][i] = band[(k+j-i) ldb + i]
            const double a = trans ? band[(int64_t)t * ldb + i] : band[(int64_t)(2 * k - t) * ldb + j];
#pragma unroll
            for (int q = 0; q < NR; ++q)
                if (q < nrhs) acc[q] += a * u[q * n + j];
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            if (q >= nrhs) continue;
            y[q * n + i] = acc[q];
            const double wq = w[q * n + i];
            if (MODE == 0) {
                dv[q] += wq * acc[q];
            } else {
                dv[q] += acc[q] * wq;
                dv[NR + q] += acc[q] * acc[q];
            }
        }
    }
    // quantity slots: q for t.s (or tilde r . y), NR + q for t.t; unused slots stay 0
    __shared__ double tot[NV];
    const int nv = (MODE == 0) ? nrhs : NV;
    if (grid_sums<NV>(dv, nv, partial, counter, tot) && threadIdx.x < nrhs) {
        const int q = threadIdx.x;
        if (MODE == 0) {
            sc[S_RHV * mx + q] = tot[q];
        } else {
            sc[S_TS * mx + q] = tot[q];
            sc[S_TT * mx + q] = tot[NR + q];
        }
    }
}

// alpha = rho_new / rhv;  s = r - alpha v;  |s|, 1/|s| into nrm; |s|^2 -> S_SS.
template <int NR>
__global__ void __launch_bounds__(VBS)
    k_bicg_s(const double *__restrict__ r, const double *__restrict__ vv, double *__restrict__ sv, int64_t n,
             int nrhs, int mx, double *sc, double *nrm, double *inv, double *partial, unsigned *counter) {
    double al[NR], act[NR], ss[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        ss[q] = 0.0;
        al[q] = act[q] = 0.0;
        if (q < nrhs) {
            act[q] = sc[S_ACTIVE * mx + q];
            al[q] = safe_div(sc[S_RHO_NEW * mx + q], sc[S_RHV * mx + q]);
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)VBS + threadIdx.x; i < n; i += (int64_t)gridDim.x * VBS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            if (q >= nrhs) continue;
            const int64_t e = q * n + i;
            const double a = (act[q] != 0.0) ? r[e] - al[q] * vv[e] : 0.0;
            sv[e] = a;
            ss[q] += a * a;
        }
    }
    __shared__ double tot[NR];
    if (grid_sums<NR>(ss, nrhs, partial, counter, tot) && threadIdx.x < nrhs) {
        const int q = threadIdx.x;
        const double nv = sqrt(tot[q]);
        nrm[q] = nv;
        inv[q] = (nv > 0.0) ? 1.0 / nv : 0.0;
        sc[S_SS * mx + q] = tot[q];
        sc[S_ALPHA * mx + q] = safe_div(sc[S_RHO_NEW * mx + q], sc[S_RHV * mx + q]);
    }
}

// omega; x += alpha ph + omega sh;  r = s - omega t;  rho = rho_new;
// rho_new = tilde r . r;  |r|^2 -> S_RR.
template <int NR>
__global__ void __launch_bounds__(VBS)
    k_bicg_update(const double *__restrict__ ph, const double *__restrict__ sh, const double *__restrict__ sv,
                  const double *__restrict__ tv, const double *__restrict__ rh, double *__restrict__ r,
                  double *__restrict__ x, int64_t ldx, int64_t n, int nrhs, int mx, double tol, double *sc,
                  double *partial, unsigned *counter) {
    constexpr int NV = 2 * NR;
    double al[NR], om[NR], act[NR], dv[NV];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        dv[q] = dv[NR + q] = 0.0;
        al[q] = om[q] = act[q] = 0.0;
        if (q < nrhs) {
            act[q] = sc[S_ACTIVE * mx + q];
            al[q] = sc[S_ALPHA * mx + q];
            const bool done = sqrt(sc[S_SS * mx + q]) <= tol * sqrt(sc[S_BB * mx + q]);
            om[q] = done ? 0.0 : safe_div(sc[S_TS * mx + q], sc[S_TT * mx + q]);
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)VBS + threadIdx.x; i < n; i += (int64_t)gridDim.x * VBS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            if (q >= nrhs) continue;
            const int64_t e = q * n + i;
            double rn = r[e];
            if (act[q] != 0.0) {
                x[q * ldx + i] += al[q] * ph[e] + om[q] * sh[e];
                rn = sv[e] - om[q] * tv[e];
                r[e] = rn;
            }
            dv[q] += rn * rn;
            dv[NR + q] += rh[e] * rn;
        }
    }
    __shared__ double tot[NV];
    if (grid_sums<NV>(dv, NV, partial, counter, tot) && threadIdx.x < nrhs) {
        const int q = threadIdx.x;
        if (sc[S_ACTIVE * mx + q] != 0.0) {
            const bool done = sqrt(sc[S_SS * mx + q]) <= tol * sqrt(sc[S_BB * mx + q]);
            sc[S_RHO * mx + q] = sc[S_RHO_NEW * mx + q];
            sc[S_OMEGA * mx + q] = done ? 0.0 : safe_div(sc[S_TS * mx + q], sc[S_TT * mx + q]);
            sc[S_RHO_NEW * mx + q] = tot[NR + q];
        }
        sc[S_RR * mx + q] = tot[q];
    }
}


template <int NR>
static bool bicg_kernels_restart(Ctx *c, unsigned g, const double *r0, int nrhs, double **bv, double *part) {
    const int mx = c->opt.max_nrhs;
    return launch(c, KID_VEC, [&] {
        k_bicg_restart<NR><<<g, VBS, 0, c->stream>>>(r0, c->n, nrhs, mx, bv[0], bv[1], bv[2], bv[3], c->dots, part,
                                                    c->counter);
    });
}

// One BiCGStab iteration for every column (frozen columns pass through).
template <int NR>
static bool bicg_iteration(Ctx *c, unsigned g, int nrhs, bool trans, double *xd, int64_t ldd, double **bv,
                           double *part) {
    const int mx = c->opt.max_nrhs;
    const int64_t n = c->n;
    double *r = bv[0], *rh = bv[1], *pv = bv[2], *vv = bv[3], *sv = bv[4], *tv = bv[5], *ph = bv[6], *sh = bv[7];
    double *sc = c->dots, *nrm = c->nrm + mx, *inv = c->nrm + 2 * mx;
    const int tr = trans ? 1 : 0;
    if (!launch(c, KID_VEC, [&] {
            k_bicg_p<NR><<<g, VBS, 0, c->stream>>>(r, vv, pv, n, nrhs, mx, sc, nrm, inv, part, c->counter);
        }))
        return false;
    if (!apply_precond(c, pv, ph, n, nrhs, trans, false)) return false;
    if (!launch(c, KID_MATVEC, [&] {
            k_bicg_mv<NR, 0><<<g, VBS, 0, c->stream>>>(c->band, c->ld, c->k, n, tr, ph, vv, rh, nrhs, mx, sc, part,
                                                       c->counter, c->diag_list, c->ndiag);
        }))
        return false;
    if (!launch(c, KID_VEC, [&] {
            k_bicg_s<NR><<<g, VBS, 0, c->stream>>>(r, vv, sv, n, nrhs, mx, sc, nrm, inv, part, c->counter);
        }))
        return false;
    if (!apply_precond(c, sv, sh, n, nrhs, trans, false)) return false;
    if (!launch(c, KID_MATVEC, [&] {
            k_bicg_mv<NR, 1><<<g, VBS, 0, c->stream>>>(c->band, c->ld, c->k, n, tr, sh, tv, sv, nrhs, mx, sc, part,
                                                       c->counter, c->diag_list, c->ndiag);
        }))
        return false;
    return launch(c, KID_VEC, [&] {
        k_bicg_update<NR><<<g, VBS, 0, c->stream>>>(ph, sh, sv, tv, rh, r, xd, ldd, n, nrhs, mx, c->opt.tol, sc,
                                                    part, c->counter);
    });
}

template <int NR>
static bool bicg_solve(Ctx *c, const double *fd, double *xd, int64_t ldd, int nrhs, bool trans, BicgResult &res) {
    const int mx = c->opt.max_nrhs;
    const unsigned g = vgrid(c->n);
    double **bv = c->bv, *part = c->bpartial;
    double *hf = c->host;              // |f| per column (read by the caller's norm pass)
    double *hr = c->host + mx;         // |r| read back
    double *hs = c->host + 2 * mx;     // [S_BB | S_ACTIVE | S_RESTART] rows uploaded together
    double *hrr = c->host + 5 * mx;    // S_RR read back
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return false;
    std::vector<char> active(nrhs), broke(nrhs, 0);
    for (int q = 0; q < mx; ++q) {
        const bool on = q < nrhs && hf[q] > 0.0;
        hs[q] = q < nrhs ? hf[q] * hf[q] : 0.0;
        hs[mx + q] = on ? 1.0 : 0.0;
        hs[2 * mx + q] = on ? 1.0 : 0.0;
        if (q < nrhs) active[q] = on;
    }
    auto upload = [&] {
        return cudaMemcpyAsync(c->dots + S_BB * mx, hs, 3 * mx * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream) == cudaSuccess;
    };
    auto true_residual = [&]() -> bool {
        if (!run_residual(c, fd, xd, ldd, nrhs, trans, false)) return false;
        if (cudaMemcpyAsync(hr, c->nrm + mx, nrhs * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return false;
        for (int q = 0; q < nrhs; ++q) res.rel[q] = (hf[q] > 0.0) ? hr[q] / hf[q] : 0.0;
        return true;
    };
    res.iterations = 0;
    res.breakdown = false;
    // x = 0, so the first residual is f itself
    if (!upload() || !run_residual(c, fd, xd, ldd, nrhs, trans, true) ||
        !bicg_kernels_restart<NR>(c, g, c->rv, nrhs, bv, part))
        return false;
    int it = 0;
    for (;;) {
        bool any = false;
        for (int q = 0; q < nrhs; ++q) any = any || active[q];
        if (any && it < c->opt.max_iter) {
            ++it;
            if (!bicg_iteration<NR>(c, g, nrhs, trans, xd, ldd, bv, part)) return false;
            if (cudaMemcpyAsync(hrr, c->dots + S_RR * mx, nrhs * 8, cudaMemcpyDeviceToHost, c->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return false;
            bool changed = false;
            for (int q = 0; q < nrhs; ++q) {
                if (!active[q]) continue;
                const double rel = std::sqrt(hrr[q]) / hf[q];
                if (!(rel == rel) || std::isinf(rel)) broke[q] = 1;
                if (broke[q] || rel <= c->opt.tol) {
                    active[q] = 0;
                    hs[mx + q] = 0.0;
                    changed = true;
                }
            }
            for (int q = 0; q < mx; ++q) hs[2 * mx + q] = 0.0;
            if (changed && !upload()) return false;
            continue;
        }
        // every column stopped (or the iteration limit): confirm with the true residual
        if (!true_residual()) return false;
        bool restart = false;
        for (int q = 0; q < nrhs; ++q) {
            const bool bad = !(res.rel[q] <= c->opt.tol);
            hs[2 * mx + q] = 0.0;
            if (bad && !broke[q] && it < c->opt.max_iter) {
                // the recursive residual drifted from f - A x: restart from the true one
                active[q] = 1;
                hs[mx + q] = 1.0;
                hs[2 * mx + q] = 1.0;
                restart = true;
            }
        }
        if (!restart) break;
        if (!upload() || !bicg_kernels_restart<NR>(c, g, c->rv, nrhs, bv, part)) return false;
    }
    res.iterations = it;
    for (int q = 0; q < nrhs; ++q) res.breakdown = res.breakdown || broke[q];
    return true;
}

}  // namespace

bool bicgstab_alloc(Ctx *c) {
    const size_t vec = (size_t)c->n * c->opt.max_nrhs * sizeof(double);
    for (double *&p : c->bv)  // zeroed: frozen columns are read but never restarted
        if (cudaMalloc((void **)&p, vec) != cudaSuccess || cudaMemset(p, 0, vec) != cudaSuccess) return false;
    if (cudaMalloc((void **)&c->dots, (size_t)S_ROWS * c->opt.max_nrhs * sizeof(double)) != cudaSuccess) return false;
    if (cudaMalloc((void **)&c->bpartial, (size_t)kMaxCtas * 32 * sizeof(double)) != cudaSuccess)
        return false;
    return cudaMemset(c->dots, 0, (size_t)S_ROWS * c->opt.max_nrhs * sizeof(double)) == cudaSuccess;
}

bool run_bicgstab(Ctx *c, const double *fd, double *xd, int64_t ldd, int nrhs, bool trans, BicgResult &res) {
    if (nrhs <= 1) return bicg_solve<1>(c, fd, xd, ldd, nrhs, trans, res);
    if (nrhs <= 2) return bicg_solve<2>(c, fd, xd, ldd, nrhs, trans, res);
    if (nrhs <= 4) return bicg_solve<4>(c, fd, xd, ldd, nrhs, trans, res);
    if (nrhs <= 8) return bicg_solve<8>(c, fd, xd, ldd, nrhs, trans, res);
    return bicg_solve<16>(c, fd, xd, ldd, nrhs, trans, res);
}

}  // namespace lrs
