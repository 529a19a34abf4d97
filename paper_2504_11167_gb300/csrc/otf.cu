// LR-SPIKE-OTF (paper section 2.2, "SPIKE-on-the-fly", eqs. OTF-1 / OTF-2;
// section 3.3: the truncated low-rank reduced system S~~_r as its
// preconditioner).  The TRUE reduced system of the spike matrix S = D^{-1} A is
// solved iteratively on the interface tips.  Per interface i = 1..p-1 the
// unknowns are y_i = [x_{i,b} ; x_{i+1,t}] (2k values).  Spike products are
// never formed: by linearity both spikes of partition i act through one solve
// with A_i on
//     c_i = [C_i x_{i-1,b} ; 0 ; B_i x_{i+1,t}],
// so  S_red y = y + tips(D^{-1} c(y))  costs one D-stage (all partitions at
// once).  Preconditioner, per interface, by Woodbury:
//     [[I, T~_{i,b}], [W~_{i+1,t}, I]]^{-1} y = y - [u_T^(b) ; u_W^(t)] E_i^{-1} [P_i y_t ; Q_{i+1} y_b]
// with the truncated reduced factors E_i^{-1} of the factorisation.
// One OTF solve:
//   1. g = D^{-1} f;
//   2. right-preconditioned BiCGStab on S_red y = tips(g), to a reduced
//      tolerance (1e-8 by default);
//   3. x = g - D^{-1} c(y).
// The outer refinement calls it for every correction.
//
// Reduced vectors are FP64, column-major by right-hand side, [p-1][2k] per
// column.  The reduced BiCGStab runs one CTA per column, so its dot products
// are block reductions in a fixed order (reproducible), and its scalars stay
// on the device.  The host reads the residual norms once per iteration (the
// convergence test).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrs {

namespace {

constexpr int OBS = 1024;  // threads per CTA of the reduced-vector kernels

enum OScalar { O_RHO = 0, O_ALPHA, O_OMEGA, O_RHO_NEW, O_BB, O_RR, O_ACTIVE, O_ROWS };

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[OBS / 32];
    __shared__ double tot;
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < OBS / 32; ++w) t += red[w];
        tot = t;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

// c (FP64, n x nrhs, only tip rows written): the top k rows of partition i
// get C_i x_{i-1,b}, the bottom k rows get B_i x_{i+1,t}; rows in both tips
// (partitions shorter than 2k) get both terms.
__global__ void __launch_bounds__(256)
    k_otf_rhs(const double *__restrict__ band, int64_t ldb, int k, Parts P, const double *__restrict__ y,
              int nrhs, int64_t n, double *__restrict__ cvec) {
    const int i = blockIdx.x, p = P.p;
    const int64_t s = P.off[i], ni = P.off[i + 1] - s, nrc = (int64_t)(p - 1) * 2 * k;
    for (int e = threadIdx.x; e < 2 * k * nrhs; e += blockDim.x) {
        const int c = e / (2 * k), sl = e % (2 * k);
        const int64_t rho = sl < k ? sl : ni - 2 * k + sl;  // top rows, then bottom rows
        if (sl >= k && rho < k) continue;                    // already handled as a top row
        const int64_t row = s + rho;
        double acc = 0.0;
        if (i > 0 && rho < k) {  // C_i x_{i-1,b}: columns s-k .. s-1
            const double *yy = y + c * nrc + (int64_t)(i - 1) * 2 * k;
            for (int l = 0; l < k; ++l) {
                const int64_t col = s - k + l, d = k + row - col;
                if (d <= 2 * k) acc += band[d * ldb + col] * yy[l];
            }
        }
        if (i < p - 1 && rho >= ni - k) {  // B_i x_{i+1,t}: columns s+ni .. s+ni+k-1
            const double *yy = y + c * nrc + (int64_t)i * 2 * k + k;
            for (int l = 0; l < k; ++l) {
                const int64_t col = s + ni + l, d = k + row - col;
                if (d >= 0) acc += band[d * ldb + col] * yy[l];
            }
        }
        cvec[c * n + row] = acc;
    }
}

// yout = (yin or 0) + tips(g); g is the D-stage output (T, n x nrhs)
template <typename T>
__global__ void __launch_bounds__(256)
    k_otf_tips(const T *__restrict__ g, int64_t n, int k, Parts P, const double *__restrict__ yin,
               double *__restrict__ yout, int nrhs) {
    const int64_t nrc = (int64_t)(P.p - 1) * 2 * k, tot = nrc * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / nrc, rem = e % nrc;
        const int i = (int)(rem / (2 * k)), j = (int)(rem % (2 * k));
        const int64_t sb = P.off[i + 1];
        const int64_t row = j < k ? sb - k + j : sb + (j - k);
        yout[e] = (yin ? yin[e] : 0.0) + (double)g[c * n + row];
    }
}

// psi_i = [P_i y_{i,t-part} ; Q_{i+1} y_{i,b-part}]  (psi layout [p-1][2r][nrhs])
template <typename T>
__global__ void __launch_bounds__(256)
    k_otf_psi(const T *__restrict__ PQ, int KB, int r, int k, int p, const double *__restrict__ y, int nrhs,
              double *__restrict__ psi) {
    const int64_t nrc = (int64_t)(p - 1) * 2 * k;
    const int tot = (p - 1) * 2 * r * nrhs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        const int c = e % nrhs, ij = e / nrhs, i = ij / (2 * r), j = ij % (2 * r);
        const double *yy = y + c * nrc + (int64_t)i * 2 * k;
        double acc = 0.0;
        if (j < r) {
            const T *Pm = PQ + ((int64_t)i * 2 + 0) * r * KB + (int64_t)j * KB;
            for (int q = 0; q < k; ++q) acc += (double)Pm[q] * yy[k + q];
        } else {
            const T *Qm = PQ + ((int64_t)(i + 1) * 2 + 1) * r * KB + (int64_t)(j - r) * KB;
            for (int q = 0; q < k; ++q) acc += (double)Qm[q] * yy[q];
        }
        psi[e] = acc;
    }
}

// yout_i = yin_i - [u_T^(b) z_i[0:r] ; u_W^(t) z_i[r:2r]]  (z in the psi layout)
template <typename T>
__global__ void __launch_bounds__(256)
    k_otf_unpsi(const T *__restrict__ Ucat, Parts P, int r, int k, const double *__restrict__ yin,
                const double *__restrict__ zr, double *__restrict__ yout, int nrhs) {
    const int p = P.p, n2 = 2 * r;
    const int64_t nrc = (int64_t)(p - 1) * 2 * k, tot = nrc * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / nrc, rem = e % nrc;
        const int i = (int)(rem / (2 * k)), j = (int)(rem % (2 * k));
        const int64_t sb = P.off[i + 1];
        double acc = 0.0;
        if (j < k) {  // u_T of partition i, row sb-k+j
            const T *u = Ucat + (sb - k + j) * n2;
            for (int q = 0; q < r; ++q) acc += (double)u[q] * zr[((int64_t)i * n2 + q) * nrhs + c];
        } else {      // u_W of partition i+1, row sb+j-k
            const T *u = Ucat + (sb + j - k) * n2 + r;
            for (int q = 0; q < r; ++q) acc += (double)u[q] * zr[((int64_t)i * n2 + r + q) * nrhs + c];
        }
        yout[e] = yin[e] - acc;
    }
}

// out (+)= |in| (g0 - g1), row-major over the n x nrhs vectors
template <typename T>
__global__ void __launch_bounds__(256)
    k_otf_update(const T *__restrict__ g0, const T *__restrict__ g1, int64_t n, const double *__restrict__ nrm,
                 double *__restrict__ out, int64_t ldo, int nrhs, int accumulate) {
    const int64_t tot = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, row = e % n;
        const double d = nrm[c] * ((double)g0[e] - (double)g1[e]);
        out[c * ldo + row] = accumulate ? out[c * ldo + row] + d : d;
    }
}

// ---- reduced BiCGStab vector steps: one CTA per column ----------------------
// sc: [O_ROWS][ldsc] device scalars
__global__ void __launch_bounds__(OBS)
    k_ob_init(const double *__restrict__ b, double *y, double *r, double *rt, double *pv, double *v, int64_t nrc,
              double *sc, int ldsc) {
    const int c = blockIdx.x;
    const double *bb = b + c * nrc;
    double *yy = y + c * nrc, *rr = r + c * nrc, *tt = rt + c * nrc, *pp = pv + c * nrc, *vv = v + c * nrc;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) {
        const double x = bb[e];
        yy[e] = 0.0; rr[e] = x; tt[e] = x; pp[e] = 0.0; vv[e] = 0.0;
        s += x * x;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) {
        sc[O_RHO * ldsc + c] = 1.0;
        sc[O_ALPHA * ldsc + c] = 1.0;
        sc[O_OMEGA * ldsc + c] = 1.0;
        sc[O_BB * ldsc + c] = s;
        sc[O_RR * ldsc + c] = s;
        sc[O_ACTIVE * ldsc + c] = (s > 0.0) ? 1.0 : 0.0;
    }
}

// rho_new = rt . r;  beta = (rho_new / rho)(alpha / omega);  p = r + beta (p - omega v)
__global__ void __launch_bounds__(OBS)
    k_ob_p(const double *r, const double *rt, double *pv, const double *v, int64_t nrc, double *sc, int ldsc) {
    const int c = blockIdx.x;
    if (sc[O_ACTIVE * ldsc + c] == 0.0) return;
    const double *rr = r + c * nrc, *tt = rt + c * nrc, *vv = v + c * nrc;
    double *pp = pv + c * nrc;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) s += tt[e] * rr[e];
    const double rho_new = block_sum(s);
    const double rho = sc[O_RHO * ldsc + c], alpha = sc[O_ALPHA * ldsc + c], omega = sc[O_OMEGA * ldsc + c];
    const bool ok = rho != 0.0 && omega != 0.0 && isfinite(rho_new);
    const double beta = ok ? (rho_new / rho) * (alpha / omega) : 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) pp[e] = rr[e] + beta * (pp[e] - omega * vv[e]);
    if (threadIdx.x == 0) {
        sc[O_RHO_NEW * ldsc + c] = rho_new;
        if (!ok || rho_new == 0.0) sc[O_ACTIVE * ldsc + c] = 0.0;  // breakdown: keep the current iterate
    }
}

// alpha = rho_new / (rt . v);  s = r - alpha v  (s written over r's buffer copy sv)
__global__ void __launch_bounds__(OBS)
    k_ob_s(const double *r, const double *rt, const double *v, double *sv, int64_t nrc, double *sc, int ldsc) {
    const int c = blockIdx.x;
    if (sc[O_ACTIVE * ldsc + c] == 0.0) return;
    const double *rr = r + c * nrc, *tt = rt + c * nrc, *vv = v + c * nrc;
    double *ss = sv + c * nrc;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) s += tt[e] * vv[e];
    const double rv = block_sum(s);
    const double rho_new = sc[O_RHO_NEW * ldsc + c];
    const bool ok = rv != 0.0 && isfinite(rv);
    const double alpha = ok ? rho_new / rv : 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) ss[e] = rr[e] - alpha * vv[e];
    if (threadIdx.x == 0) {
        sc[O_ALPHA * ldsc + c] = alpha;
        if (!ok) sc[O_ACTIVE * ldsc + c] = 0.0;
    }
}

// omega = (t . s)/(t . t);  y += alpha ph + omega sh;  r = s - omega t;  |r|^2;  rho = rho_new
__global__ void __launch_bounds__(OBS)
    k_ob_update(double *y, double *r, const double *sv, const double *t, const double *ph, const double *sh,
                int64_t nrc, double *sc, int ldsc) {
    const int c = blockIdx.x;
    if (sc[O_ACTIVE * ldsc + c] == 0.0) return;
    const double *ss = sv + c * nrc, *tt = t + c * nrc, *pp = ph + c * nrc, *qq = sh + c * nrc;
    double *yy = y + c * nrc, *rr = r + c * nrc;
    double a = 0.0, b = 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) {
        a += tt[e] * ss[e];
        b += tt[e] * tt[e];
    }
    const double ts = block_sum(a), tt2 = block_sum(b);
    const double omega = (tt2 > 0.0 && isfinite(tt2)) ? ts / tt2 : 0.0;
    const double alpha = sc[O_ALPHA * ldsc + c];
    double s2 = 0.0;
    for (int64_t e = threadIdx.x; e < nrc; e += OBS) {
        yy[e] += alpha * pp[e] + omega * qq[e];
        const double x = ss[e] - omega * tt[e];
        rr[e] = x;
        s2 += x * x;
    }
    s2 = block_sum(s2);
    if (threadIdx.x == 0) {
        sc[O_OMEGA * ldsc + c] = omega;
        sc[O_RR * ldsc + c] = s2;
        sc[O_RHO * ldsc + c] = sc[O_RHO_NEW * ldsc + c];
        if (omega == 0.0) sc[O_ACTIVE * ldsc + c] = 0.0;  // s was already the answer or breakdown
    }
}

__global__ void k_ob_deactivate(double *sc, int ldsc, int c) { sc[O_ACTIVE * ldsc + c] = 0.0; }

inline unsigned ogrid(int64_t tot) { return (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 8); }

}  // namespace

template <typename P>
static bool oalloc(P **ptr, size_t bytes) {
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) return false;
    *ptr = (P *)q;
    return true;
}

bool otf_alloc(Ctx *c) {
    const int mx = c->opt.max_nrhs;
    const int64_t nrc = (int64_t)(c->p - 1) * 2 * c->k;
    const size_t ts = c->fp64 ? 8 : 4;
    if (!oalloc(&c->ocv, (size_t)c->n * mx * 8)) return false;
    if (!oalloc(&c->og, (size_t)c->n * mx * ts)) return false;
    if (!oalloc(&c->orv, (size_t)kOtfVecs * nrc * mx * 8)) return false;
    if (!oalloc(&c->osc, (size_t)O_ROWS * mx * 8)) return false;
    if (!oalloc(&c->oone, (size_t)mx * 8)) return false;
    std::vector<double> ones(mx, 1.0);
    return cudaMemcpy(c->oone, ones.data(), mx * 8, cudaMemcpyHostToDevice) == cudaSuccess;
}

template <typename T>
static bool otf_impl(Ctx *c, const double *in, double *out, int64_t ldo, int nrhs, bool accumulate) {
    const int k = c->k, mx = c->opt.max_nrhs, p = c->p;
    const int64_t n = c->n, nrc = (int64_t)(p - 1) * 2 * k;
    Parts P{c->off_d, c->boff_d, c->p};
    double *V[kOtfVecs];
    for (int q = 0; q < kOtfVecs; ++q) V[q] = c->orv + (int64_t)q * nrc * mx;
    double *b = V[0], *y = V[1], *r = V[2], *rt = V[3], *pv = V[4], *v = V[5], *ph = V[6], *sv = V[7],
           *sh = V[8], *t = V[9];
    // 1. g = D^{-1}(in / |in|)
    if (!run_dstage(c, in, n, nrhs)) return false;
    if (cudaMemcpyAsync(c->og, c->Gv, (size_t)n * nrhs * sizeof(T), cudaMemcpyDeviceToDevice, c->stream) !=
        cudaSuccess) {
        c->err = "OTF copy of g failed";
        return false;
    }
    if (cudaMemsetAsync(c->ocv, 0, (size_t)n * nrhs * 8, c->stream) != cudaSuccess) {
        c->err = "OTF reset of the coupling vector failed";
        return false;
    }
    const unsigned g1 = ogrid(nrc * nrhs), gp = ogrid((int64_t)(p - 1) * 2 * c->r * nrhs);
    if (!launch(c, KID_OTF, [&] {
            k_otf_tips<T><<<g1, 256, 0, c->stream>>>((const T *)c->og, n, k, P, nullptr, b, nrhs);
        }))
        return false;
    // S_red applied to x: out = x + tips(D^{-1} c(x))
    auto apply_S = [&](const double *x, double *o) {
        return launch(c, KID_OTF, [&] {
                   k_otf_rhs<<<p, 256, 0, c->stream>>>(c->band, c->ld, k, P, x, nrhs, n, c->ocv);
               }) &&
               run_dstage_inv(c, c->ocv, nrhs, c->oone) && launch(c, KID_OTF, [&] {
                   k_otf_tips<T><<<g1, 256, 0, c->stream>>>((const T *)c->Gv, n, k, P, x, o, nrhs);
               });
    };
    // the truncated low-rank reduced system, inverted per interface (Woodbury)
    auto apply_M = [&](const double *x, double *o) {
        return launch(c, KID_OTF, [&] {
                   k_otf_psi<T><<<gp, 256, 0, c->stream>>>((const T *)c->PQ, c->KB, c->r, k, p, x, nrhs, c->psi);
               }) &&
               run_reduced_solve(c, nrhs, false) && launch(c, KID_OTF, [&] {
                   k_otf_unpsi<T><<<g1, 256, 0, c->stream>>>((const T *)c->Ucat, P, c->r, k, x, c->zr, o, nrhs);
               });
    };
    // 2. reduced BiCGStab on S_red y = b
    if (!launch(c, KID_OTF, [&] { k_ob_init<<<nrhs, OBS, 0, c->stream>>>(b, y, r, rt, pv, v, nrc, c->osc, mx); }))
        return false;
    std::vector<double> hs((size_t)O_ROWS * mx);
    int it = 0;
    for (; it < c->opt.otf_max_iter; ++it) {
        if (!launch(c, KID_OTF, [&] { k_ob_p<<<nrhs, OBS, 0, c->stream>>>(r, rt, pv, v, nrc, c->osc, mx); }) ||
            !apply_M(pv, ph) || !apply_S(ph, v) ||
            !launch(c, KID_OTF, [&] { k_ob_s<<<nrhs, OBS, 0, c->stream>>>(r, rt, v, sv, nrc, c->osc, mx); }) ||
            !apply_M(sv, sh) || !apply_S(sh, t) ||
            !launch(c, KID_OTF, [&] {
                k_ob_update<<<nrhs, OBS, 0, c->stream>>>(y, r, sv, t, ph, sh, nrc, c->osc, mx);
            }))
            return false;
        if (cudaMemcpyAsync(hs.data(), c->osc, hs.size() * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            c->err = "OTF reduced iteration failed";
            return false;
        }
        bool any = false;
        for (int q = 0; q < nrhs; ++q) {
            if (hs[(size_t)O_ACTIVE * mx + q] == 0.0) continue;
            const double bb = hs[(size_t)O_BB * mx + q], rr = hs[(size_t)O_RR * mx + q];
            if (!(rr > c->opt.otf_tol * c->opt.otf_tol * bb)) {
                if (!launch(c, KID_OTF, [&] { k_ob_deactivate<<<1, 1, 0, c->stream>>>(c->osc, mx, q); }))
                    return false;
            } else {
                any = true;
            }
        }
        if (!any) {
            ++it;
            break;
        }
    }
    c->otf_iters += it;
    // 3. x = g - D^{-1} c(y), scaled back by |in|
    if (!launch(c, KID_OTF, [&] { k_otf_rhs<<<p, 256, 0, c->stream>>>(c->band, c->ld, k, P, y, nrhs, n, c->ocv); }) ||
        !run_dstage_inv(c, c->ocv, nrhs, c->oone))
        return false;
    return launch(c, KID_OTF, [&] {
        k_otf_update<T><<<ogrid(n * nrhs), 256, 0, c->stream>>>((const T *)c->og, (const T *)c->Gv, n,
                                                               c->nrm + mx, out, ldo, nrhs, accumulate);
    });
}

bool apply_otf(Ctx *c, const double *in, double *out, int64_t ldo, int nrhs, bool accumulate) {
    return c->fp64 ? otf_impl<double>(c, in, out, ldo, nrhs, accumulate)
                   : otf_impl<float>(c, in, out, ldo, nrhs, accumulate);
}

}  // namespace lrs
