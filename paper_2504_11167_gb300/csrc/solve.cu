// Solve-phase kernels of one preconditioner application and of the FP64 outer
// iteration (paper section 2.1 solve summary, eqs. 'D-stage-in-summary' ..
// 'recovery-stage-in-summary'; section 3.3 low-rank recovery).
//
//   k_residual  r = f - A x (or f - A^T x) in FP64 from the band, with the
//               per-column sum of squares reduced deterministically (fixed
//               per-CTA partials, summed in order by the last CTA to finish)
//   k_sumsq     the same reduction for a plain vector (||f||)
//   k_dstage    g_i = A_i^{-1} (r_i / ||r||) per partition in the working
//               precision: forward and backward block chains; epilogue forms
//               psi = V g at both ends of the partition (FP64)
//   k_retrieve  x += ||r|| (g - u_T zeta - u_W omega)  (update in FP64)
//   k_project_t a = U^T h (transposed preconditioner, first step)
//   k_dstage_t  l = D^{-T}(h - V^T w), then x += ||r|| l
#include "common.cuh"
#include "internal.h"
#include "tile_ops.cuh"

namespace lrs {

constexpr int RBS = 256;  // rows per CTA in the row-parallel kernels

// Block reduction of NR per-column sums into partial[blockIdx.x][c]; the last
// CTA (atomic ticket) sums all partials in CTA order and writes the norms.
template <int NR>
__device__ void reduce_columns(double (&ss)[NR], int nrhs, double *partial, unsigned *counter,
                               double *nrm_out, double *inv_out, StopRule st = StopRule()) {
    __shared__ double red[NR][RBS / 32];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        const double v = warp_sum(ss[c]);
        if (lane == 0) red[c][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < nrhs) {
        double t = 0.0;
        for (int w = 0; w < RBS / 32; ++w) t += red[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * nrhs + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (is_last) {
        // fixed assignment of partials to threads and a fixed tree: deterministic
        __threadfence();
        __shared__ double tot[RBS / 32];
        for (int c = 0; c < nrhs; ++c) {
            double t = 0.0;
            for (unsigned b = threadIdx.x; b < gridDim.x; b += RBS) t += __ldcg(&partial[(int64_t)b * nrhs + c]);
            t = warp_sum(t);
            if (lane == 0) tot[wid] = t;
            __syncthreads();
            if (threadIdx.x == 0) {
                double sum = 0.0;
                for (int w = 0; w < RBS / 32; ++w) sum += tot[w];
                const double nv = sqrt(sum);
                nrm_out[c] = nv;
                if (inv_out) inv_out[c] = (nv > 0.0) ? 1.0 / nv : 0.0;
            }
            __syncthreads();
        }
        if (st.flag && threadIdx.x == 0) {  // early-exit rule (NaN norms never meet it)
            bool met = true;
            for (int c = 0; c < nrhs; ++c) met = met && nrm_out[c] <= st.tol * st.fnrm[c];
            if (met) st.flag[0] = 1;
            else st.flag[1] += st.count;
        }
    }
    if (is_last && threadIdx.x == 0) *counter = 0u;  // ready for the next launch
}

template <int NR>
__global__ void __launch_bounds__(RBS)
    k_residual(const double *__restrict__ band, int64_t ldb, int k, int64_t n,
               const double *__restrict__ f, const double *__restrict__ x, int64_t ld, int nrhs,
               int trans, int xzero, double *__restrict__ r, double *partial, unsigned *counter,
               double *nrm_out, double *inv_out, const int *__restrict__ dlist, int ndl, StopRule st) {
    if (st.flag && *(volatile int *)st.flag) return;  // an earlier residual met tol: x is final
    const int64_t i = blockIdx.x * (int64_t)RBS + threadIdx.x;
    double acc[NR], ss[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) { acc[c] = 0.0; ss[c] = 0.0; }
    if (i < n) {
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) acc[c] = f[c * ld + i];
        if (!xzero) {
            // t = j - i + k; with a list of the band rows that hold nonzeros
            // (row d = 2k - t of A, row t of A^T) only those are visited
            const int nt = dlist ? ndl : 2 * k + 1;
            for (int u = 0; u < nt; ++u) {
                const int t = dlist ? (trans ? dlist[u] : 2 * k - dlist[u]) : u;
                const int64_t j = i - k + t;
                if (j < 0 || j >= n) continue;
                // A[i][j] = band[(k+i-j) ld + j];  A^T[i][j] = A[j][i] = band[(k+j-i) ld + i]
                const double a = trans ? band[(int64_t)t * ldb + i] : band[(int64_t)(2 * k - t) * ldb + j];
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if (c < nrhs) acc[c] = fma(-a, x[c * ld + j], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) {
                r[c * n + i] = acc[c];
                ss[c] = acc[c] * acc[c];
            }
    }
    reduce_columns<NR>(ss, nrhs, partial, counter, nrm_out, inv_out, st);
}

// One row of the retrieval, shared by k_retrieve1 and k_residual_ret so the two
// round identically: d = g - u . z (working precision, 16-byte loads of u
// where the type allows), then x + nrm d with the product and the sum each
// rounded once (no contraction).
template <typename T, int NQ>
__device__ __forceinline__ T retrieve_row(T g, const T *__restrict__ u, const T *z, int n2) {
    T d = g;
    if (sizeof(T) == 4 && n2 % 4 == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q += 4)
            if (q < n2) {
                const float4 v = *reinterpret_cast<const float4 *>(u + q);
                d -= v.x * z[q] + v.y * z[q + 1] + v.z * z[q + 2] + v.w * z[q + 3];
            }
    } else {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < n2) d -= u[q] * z[q];
    }
    return d;
}
__device__ __forceinline__ double retrieve_update(double x, double nrm, double d, bool accumulate) {
    const double upd = __dmul_rn(nrm, d);
    return accumulate ? __dadd_rn(x, upd) : upd;
}

// The retrieval of one preconditioner application fused into the next
// residual (one right-hand side, A not transposed, unpivoted k <= 64 factors):
// x_out = x_in + nrm (g - U z) on the CTA's rows and k halo rows on each side
// (the same arithmetic as k_retrieve1), the CTA's own rows written to x_out (a
// different buffer from x_in: halo rows belong to other CTAs), then
// r = f - A x_out on its rows from shared memory (the arithmetic of
// k_residual), column norms as there.  Every partition holds at least
// RBS + 2k rows, so the rows a CTA touches span at most two partitions.
template <typename T, int NQ>
__global__ void __launch_bounds__(RBS)
    k_residual_ret(const double *__restrict__ band, int64_t ldb, int k, int64_t n,
                   const double *__restrict__ f, const double *__restrict__ x_in, double *__restrict__ x_out,
                   const T *__restrict__ Gv, const T *__restrict__ Ucat, const double *__restrict__ zr, Parts P,
                   int r, const double *nrm_in, double *__restrict__ rres, double *partial,
                   unsigned *counter, double *nrm_out, double *inv_out) {
    extern __shared__ double xs[];  // rows i0-k .. i0+RBS+k-1
    __shared__ T zs[2][NQ];
    __shared__ int pa_s;
    const int64_t i0 = blockIdx.x * (int64_t)RBS;
    const int64_t lo = i0 - k > 0 ? i0 - k : 0, hi = i0 + RBS + k < n ? i0 + RBS + k : n;
    const int n2 = 2 * r;
    if (threadIdx.x == 0) {  // partition holding row lo
        int a = 0, b = P.p - 1;
        while (a < b) {
            const int mid = (a + b + 1) / 2;
            if (P.off[mid] <= lo) a = mid;
            else b = mid - 1;
        }
        pa_s = a;
    }
    __syncthreads();
    const int pa = pa_s;
    for (int e = threadIdx.x; e < 2 * NQ; e += RBS) {
        const int side = e / NQ, j = e % NQ, part = pa + side;
        double v = 0.0;
        if (part < P.p && j < n2) {
            if (j < r) { if (part <= P.p - 2) v = zr[(int64_t)part * n2 + j]; }
            else if (part >= 1) v = zr[(int64_t)(part - 1) * n2 + j];
        }
        zs[side][j] = (T)v;
    }
    __syncthreads();
    // |r| of the preconditioned residual; nrm_in is also nrm_out, which only the
    // last CTA writes, after every CTA has taken its ticket (and so read this)
    const double sc = nrm_in[0];
    const int64_t pb = (pa + 1 < P.p) ? P.off[pa + 1] : n;  // first row of partition pa+1
    for (int64_t j = lo + threadIdx.x; j < hi; j += RBS) {
        const T d = retrieve_row<T, NQ>(Gv[j], Ucat + j * n2, zs[j >= pb ? 1 : 0], n2);
        const double xv = retrieve_update(x_in[j], sc, (double)d, true);
        xs[j - (i0 - k)] = xv;
        if (j >= i0 && j < i0 + RBS) x_out[j] = xv;
    }
    __syncthreads();
    const int64_t i = i0 + threadIdx.x;
    double ss[1] = {0.0};
    if (i < n) {
        double acc = f[i];
        for (int t = 0; t < 2 * k + 1; ++t) {
            const int64_t j = i - k + t;
            if (j < 0 || j >= n) continue;
            acc = fma(-band[(int64_t)(2 * k - t) * ldb + j], xs[j - (i0 - k)], acc);
        }
        rres[i] = acc;
        ss[0] = acc * acc;
    }
    reduce_columns<1>(ss, 1, partial, counter, nrm_out, inv_out);
}

template <int NR>
__global__ void __launch_bounds__(RBS)
    k_sumsq(const double *__restrict__ v, int64_t ld, int64_t n, int nrhs, double *partial,
            unsigned *counter, double *nrm_out, double *inv_out) {
    const int64_t i = blockIdx.x * (int64_t)RBS + threadIdx.x;
    double ss[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        ss[c] = 0.0;
        if (i < n && c < nrhs) { const double t = v[c * ld + i]; ss[c] = t * t; }
    }
    reduce_columns<NR>(ss, nrhs, partial, counter, nrm_out, inv_out);
}

// Row stride of the staged factor tiles of the D-stage.  FP32 KB = 64 uses 80
// (= 16 mod 32 words): the two rows a quarter-warp reads then fall on
// disjoint bank halves, and with the rotated chunk order of ds_row64 the four
// lanes of a row on disjoint quarters, so the 16-byte tile loads are free of
// bank conflicts.  Otherwise one 16-byte pad per row.
template <typename T, int KB>
__host__ __device__ constexpr int ds_ldp() {
    return (sizeof(T) == 4 && KB == 64) ? 80 : KB + 16 / (int)sizeof(T);
}

// FP32, KB = 64, one right-hand side: lane q of row a owns the quarter row
// [16q, 16q+16), visited in four 4-entry chunks in the rotated order
// (u + q) mod 4 (chunk offsets co[u]).  mv holds the quarter of the tile row
// (loaded once per block step, used by both triangular products); masks m
// select the product's entries (INV: the complement).
template <bool INV>
__device__ __forceinline__ float ds_dot64(const float (&mv)[16], const float *v, const int (&co)[4],
                                         const unsigned (&m)[16]) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 f = *reinterpret_cast<const float4 *>(v + co[u]);
        const float vv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const unsigned mk = INV ? ~m[4 * u + w] : m[4 * u + w];
            acc[w] = fmaf(__uint_as_float(__float_as_uint(mv[4 * u + w]) & mk), vv[w], acc[w]);
        }
    }
    return quad_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
}

__device__ __forceinline__ void ds_row64(const float *row, const int (&co)[4], float (&mv)[16]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 f = *reinterpret_cast<const float4 *>(row + co[u]);
        mv[4 * u] = f.x; mv[4 * u + 1] = f.y; mv[4 * u + 2] = f.z; mv[4 * u + 3] = f.w;
    }
}

// ---------------------------------------------------------------------------
template <typename T, int KB, Split S, int NBUF>
__device__ void dstage_body(const T *__restrict__ LT, const T *__restrict__ UT, const T *__restrict__ DI,
                            const T *__restrict__ PQ, Parts P, int k, int r, int64_t n,
                            const double *__restrict__ rin, const double *__restrict__ inv,
                            int nrhs, T *__restrict__ Yv, T *__restrict__ Gv, double *__restrict__ psi,
                            unsigned char *smem_raw) {
    constexpr int NT = Geo<KB>::NT, LDP = ds_ldp<T, KB>();
    constexpr int PDS = NBUF - 1;  // steps staged ahead (the factor tile of a step is 16 KB from HBM)
    const int pm = KB * nrhs;
    double *ib = reinterpret_cast<double *>(smem_raw);  // [NBUF][KB x nrhs] staged input rows
    T *tb = reinterpret_cast<T *>(ib + NBUF * pm);       // [NBUF][KB x LDP] staged factor tiles
    T *db = tb + NBUF * KB * LDP;                         // [NBUF][KB] staged D^{-1}
    T *Tt = db + NBUF * KB;
    T *Yp = Tt + pm;
    T *Yk = Yp + pm;  // forward output of block nb-2, kept for the backward sweep
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int steps = 2 * nb;
    // step t < nb: forward block t (LT, input rows of r); step t >= nb:
    // backward block 2nb-1-t (UT, DI, input rows of y written by the forward
    // sweep).  A backward input is staged PDS steps ahead from global memory
    // only for blocks J <= nb-3, whose forward writes are at least two steps
    // (and barriers) older; blocks nb-1 and nb-2 take it from Yp and Yk.
    auto stage = [&](int t) {
        const int buf = t % NBUF;
        double *in = ib + buf * pm;
        if (t < nb) {
            stage_tile<T, KB, LDP>(LT + (b0 + t) * KB * KB, tb + buf * KB * LDP, nullptr, nullptr);
            for (int e = threadIdx.x; e < pm; e += NT) {
                const int c = e / KB, a = e % KB;
                const int64_t row = (int64_t)t * KB + a;
                if (row < ni) cp_async_small<8>(in + a * nrhs + c, rin + c * n + s + row);
            }
        } else {
            const int J = steps - 1 - t;
            const int64_t g = b0 + J;
            stage_tile<T, KB, LDP>(UT + g * KB * KB, tb + buf * KB * LDP, DI + g * KB, db + buf * KB);
            if (J < nb - 2) {
                T *inT = reinterpret_cast<T *>(in);
                for (int e = threadIdx.x; e < pm; e += NT) {
                    const int c = e / KB, a = e % KB;
                    const int64_t row = (int64_t)J * KB + a;
                    if (row < ni) cp_async_small<(int)sizeof(T)>(inT + a * nrhs + c, Yv + c * n + s + row);
                }
            }
        }
    };
    for (int t = 0; t < PDS; ++t) {
        if (t < steps) stage(t);
        cp_async_commit();
    }
    bool fused = false;
    if constexpr (sizeof(T) == 4 && KB == 64) {
        if (nrhs == 1) {
            // One right-hand side, KB = 64: two barriers per block step; the
            // tile row chunks are read from shared memory once and serve both
            // triangular products (forward j >= a and j < a, backward j <= a
            // and j > a).
            fused = true;
            const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
            int co[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) co[u] = 16 * q + 4 * ((u + q) & 3);
            unsigned m[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) m[e] = (co[e / 4] + (e % 4) >= a) ? ~0u : 0u;
            const double inv0 = inv[0];
            float mv[16];
            for (int t = 0; t < nb; ++t) {
                cp_async_wait<PDS - 1>();
                __syncthreads();
                // buffer (t + PDS) % NBUF last served step t-1, closed by the barrier above
                if (t + PDS < steps) stage(t + PDS);
                cp_async_commit();
                ds_row64(tb + (t % NBUF) * KB * LDP + a * LDP, co, mv);
                const int64_t row = (int64_t)t * KB + a;
                // the scaled input (an FP64 product, on the slow FP64 pipe) only where it is stored
                const float b = (q != 0 || row >= ni) ? 0.f : (float)(ib[(t % NBUF) * pm + a] * inv0);
                // t = b_J - L_{J,J-1} y_{J-1}  (t and y are kept by lane q = 0)
                const float tv = b - ((t > 0) ? ds_dot64<false>(mv, Yp, co, m) : 0.f);
                if (q == 0) Tt[a] = tv;
                __syncthreads();
                // y_J = t + (L^{-1} strictly lower) t
                const float y = tv + ds_dot64<true>(mv, Tt, co, m);
                if (q == 0) {
                    Yp[a] = y;
                    if (row < ni) Yv[s + row] = y;
                    if (t == nb - 2) Yk[a] = y;
                }
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) m[e] = (co[e / 4] + (e % 4) <= a) ? ~0u : 0u;
            for (int t = nb; t < steps; ++t) {
                cp_async_wait<PDS - 1>();
                __syncthreads();
                if (t + PDS < steps) stage(t + PDS);
                cp_async_commit();
                ds_row64(tb + (t % NBUF) * KB * LDP + a * LDP, co, mv);
                const int J = steps - 1 - t;
                const int64_t row = (int64_t)J * KB + a;
                const float *inT = reinterpret_cast<const float *>(ib + (t % NBUF) * pm);
                const float yin = (row >= ni) ? 0.f : (J == nb - 1) ? Yp[a] : (J == nb - 2) ? Yk[a] : inT[a];
                const float dsm = db[(t % NBUF) * KB + a];
                // t = D^{-1} y_J - (D^{-1}U_{J,J+1}) x_{J+1}
                const float tv = yin * dsm - ((J < nb - 1) ? ds_dot64<false>(mv, Yp, co, m) : 0.f);
                if (q == 0) Tt[a] = tv;
                __syncthreads();
                // x_J = t + ((D^{-1}U_JJ)^{-1} strictly upper) t
                const float x = tv + ds_dot64<true>(mv, Tt, co, m);
                if (q == 0) {
                    Yp[a] = x;
                    if (row < ni) Gv[s + row] = x;
                }
            }
            __syncthreads();
        }
    } else if constexpr (sizeof(T) == 4) {
        if (nrhs == 1) {
            // One right-hand side in FP32 (FP64 keeps the bounded triangular
            // loops below, its multiply-adds being scarce): two barriers per block step.  The loop-top
            // barrier publishes the staged step and closes the previous one; the
            // input scaling is fused into the first product, the output stores
            // into the second.  Lane q of row a keeps bit masks of its quarter row:
            // forward j >= a (L_{J,J-1}, upper with diagonal) and its complement
            // j < a (L_JJ^{-1}); backward j <= a (D^{-1}U_{J,J+1}) and j > a.
            fused = true;
            constexpr int QW = KB / 4;
            const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
            const double inv0 = inv[0];
            unsigned msk[QW];
#pragma unroll
            for (int w = 0; w < QW; ++w) msk[w] = (q * QW + w >= a) ? ~0u : 0u;
            for (int t = 0; t < nb; ++t) {
                cp_async_wait<PDS - 1>();
                __syncthreads();
                // buffer (t + PDS) % NBUF last served step t-1, closed by the barrier above
                if (t + PDS < steps) stage(t + PDS);
                cp_async_commit();
                const float *tile = tb + (t % NBUF) * KB * LDP + a * LDP;
                const double *in = ib + (t % NBUF) * pm;
                const int64_t row = (int64_t)t * KB + a;
                // t = b_J - L_{J,J-1} y_{J-1}
                const float p1 = (t > 0) ? tri_dot1m<KB, false>(tile, Yp, q, msk) : 0.f;
                if (q == 0) {
                    const float b = (row >= ni) ? 0.f : (float)(in[a] * inv0);
                    Tt[a] = b - p1;
                }
                __syncthreads();
                // y_J = t + (L^{-1} strictly lower) t
                const float y = Tt[a] + tri_dot1m<KB, true>(tile, Tt, q, msk);
                if (q == 0) {
                    Yp[a] = y;
                    if (row < ni) Yv[s + row] = y;
                    if (t == nb - 2) Yk[a] = y;
                }
            }
#pragma unroll
            for (int w = 0; w < QW; ++w) msk[w] = (q * QW + w <= a) ? ~0u : 0u;
            for (int t = nb; t < steps; ++t) {
                cp_async_wait<PDS - 1>();
                __syncthreads();
                if (t + PDS < steps) stage(t + PDS);
                cp_async_commit();
                const float *tile = tb + (t % NBUF) * KB * LDP + a * LDP;
                const double *in = ib + (t % NBUF) * pm;
                const int J = steps - 1 - t;
                const int64_t row = (int64_t)J * KB + a;
                const float *inT = reinterpret_cast<const float *>(in);
                const float yin = (row >= ni) ? 0.f : (J == nb - 1) ? Yp[a] : (J == nb - 2) ? Yk[a] : inT[a];
                const float dsm = db[(t % NBUF) * KB + a];
                // t = D^{-1} y_J - (D^{-1}U_{J,J+1}) x_{J+1}
                const float p1 = (J < nb - 1) ? tri_dot1m<KB, false>(tile, Yp, q, msk) : 0.f;
                if (q == 0) Tt[a] = yin * dsm - p1;
                __syncthreads();
                // x_J = t + ((D^{-1}U_JJ)^{-1} strictly upper) t
                const float x = Tt[a] + tri_dot1m<KB, true>(tile, Tt, q, msk);
                if (q == 0) {
                    Yp[a] = x;
                    if (row < ni) Gv[s + row] = x;
                }
            }
            __syncthreads();
        }
    }
    if (!fused)
    for (int t = 0; t < steps; ++t) {
        // buffer (t + PDS) % NBUF last served step t-1, closed by the barrier ending it
        if (t + PDS < steps) stage(t + PDS);
        cp_async_commit();
        cp_async_wait<PDS>();
        __syncthreads();
        const T *tile = tb + (t % NBUF) * KB * LDP;
        const double *in = ib + (t % NBUF) * pm;
        if (t < nb) {
            const int J = t;
            for (int e = threadIdx.x; e < pm; e += NT) {
                const int a = e / nrhs, c = e % nrhs;
                const int64_t row = (int64_t)J * KB + a;
                Tt[e] = (row < ni) ? (T)(in[e] * inv[c]) : T(0);
            }
            __syncthreads();
            fwd_step<T, KB, S>(tile, LDP, Tt, Yp, nrhs, nrhs, J == 0);
            for (int e = threadIdx.x; e < pm; e += NT) {
                const int a = e / nrhs, c = e % nrhs;
                const int64_t row = (int64_t)J * KB + a;
                if (row < ni) Yv[c * n + s + row] = Yp[e];
                if (J == nb - 2) Yk[e] = Yp[e];
            }
        } else {
            const int J = steps - 1 - t;
            const T *inT = reinterpret_cast<const T *>(in);
            for (int e = threadIdx.x; e < pm; e += NT) {
                const int a = e / nrhs;
                const int64_t row = (int64_t)J * KB + a;
                Tt[e] = (row >= ni) ? T(0) : (J == nb - 1) ? Yp[e] : (J == nb - 2) ? Yk[e] : inT[e];
            }
            __syncthreads();
            bwd_step<T, KB, S>(tile, LDP, db + (t % NBUF) * KB, Tt, Yp, nrhs, nrhs, J == nb - 1);
            for (int e = threadIdx.x; e < pm; e += NT) {
                const int a = e / nrhs, c = e % nrhs;
                const int64_t row = (int64_t)J * KB + a;
                if (row < ni) Gv[c * n + s + row] = Yp[e];
            }
        }
        __syncthreads();
    }
    if (r == 0) return;
    // psi_{part-1}[0:r] = P_{part-1} g_t ;  psi_part[r:2r] = Q_{part+1} g_b
    const int n2 = 2 * r;
    for (int o = threadIdx.x; o < 2 * r * nrhs; o += NT) {
        const int side = o / (r * nrhs), rem = o % (r * nrhs), j = rem / nrhs, c = rem % nrhs;
        if (side == 0 && part >= 1) {
            const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * KB + j * KB;
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += (double)Pm[q] * (double)Gv[c * n + s + q];
            psi[((int64_t)(part - 1) * n2 + j) * nrhs + c] = acc;
        } else if (side == 1 && part <= P.p - 2) {
            const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * KB + j * KB;
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += (double)Qm[q] * (double)Gv[c * n + s + ni - k + q];
            psi[((int64_t)part * n2 + r + j) * nrhs + c] = acc;
        }
    }
}

template <typename T, int KB, int NBUF>
__global__ void __launch_bounds__(Geo<KB>::NT, 2)
    k_dstage(const T *__restrict__ LT, const T *__restrict__ UT, const T *__restrict__ DI,
             const T *__restrict__ PQ, Parts P, int k, int r, int64_t n, const double *__restrict__ rin,
             const double *__restrict__ inv, int nrhs, T *__restrict__ Yv, T *__restrict__ Gv,
             double *__restrict__ psi, const int *skip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (skip && *skip) return;
    if (nrhs < 4)
        dstage_body<T, KB, Split::DOTS, NBUF>(LT, UT, DI, PQ, P, k, r, n, rin, inv, nrhs, Yv, Gv, psi, smem_raw);
    else
        dstage_body<T, KB, Split::COLS, NBUF>(LT, UT, DI, PQ, P, k, r, n, rin, inv, nrhs, Yv, Gv, psi, smem_raw);
}

// x (+)= nrm * (g - u_T zeta - u_W omega) for one partition's rows.  Each
// thread updates all NC (>= nrhs) columns of its row in registers; per column
// the expression is the same as in the one-column form (d -= u_j z_j +
// u_j+1 z_j+1 + ...), so the rounding is unchanged.  The CTA's rows of u
// (row-major, 2r values a row) are staged 32 columns at a time in shared
// memory with coalesced loads (rows padded to RU_LD values: conflict-free
// 16-byte reads for FP32, 2-way for FP64), and each thread reads its row there.
// zeta and omega are converted to the working precision once, when staged (a
// conversion per use would run on GB300's slow FP64 units).
constexpr int RU_CW = 32;
template <typename T> constexpr int ru_ld() { return sizeof(T) == 4 ? RU_CW + 4 : RU_CW + 1; }
template <typename T> __host__ __device__ inline size_t retrieve_zbytes(int n2, int nrhs) { return ((size_t)n2 * nrhs * sizeof(T) + 15) / 16 * 16; }
template <typename T>
size_t retrieve_smem(int n2, int nrhs) {
    return retrieve_zbytes<T>(n2, nrhs) + (size_t)RBS * ru_ld<T>() * sizeof(T);
}

template <typename T, int NC>
__global__ void __launch_bounds__(RBS)
    k_retrieve(const T *__restrict__ Gv, const T *__restrict__ Ucat, const double *__restrict__ zr,
               Parts P, int r, int64_t n, int nrhs, const double *__restrict__ nrm, double *__restrict__ x,
               int64_t ld, int accumulate, const int *skip) {
    extern __shared__ __align__(16) unsigned char rsm[];  // [2r][nrhs] zeta_part, omega_part; staged u rows
    if (skip && *skip) return;
    constexpr int LDU = ru_ld<T>();
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t first = blockIdx.x * (int64_t)RBS;
    if (first >= ni) return;  // the whole CTA lies past this partition's rows
    const int n2 = 2 * r;
    T *zs = reinterpret_cast<T *>(rsm);
    T *us = reinterpret_cast<T *>(rsm + retrieve_zbytes<T>(n2, nrhs));
    for (int e = threadIdx.x; e < n2 * nrhs; e += RBS) {
        const int j = e / nrhs, c = e % nrhs;
        double v = 0.0;
        if (j < r) { if (part <= P.p - 2) v = zr[((int64_t)part * n2 + j) * nrhs + c]; }
        else if (part >= 1) v = zr[((int64_t)(part - 1) * n2 + j) * nrhs + c];
        zs[e] = (T)v;
    }
    const int rows = (int)min((int64_t)RBS, ni - first);
    const bool live = threadIdx.x < rows;
    const int64_t gi = s + first + threadIdx.x;
    T d[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) d[c] = (live && c < nrhs) ? Gv[c * n + gi] : T(0);
    const T *ublk = Ucat + (s + first) * n2;
    for (int j0 = 0; j0 < n2; j0 += RU_CW) {
        const int cw = min(RU_CW, n2 - j0);
        __syncthreads();  // zs written; the previous chunk consumed
        for (int e = threadIdx.x; e < rows * cw; e += RBS) {
            const int a = e / cw, j = e % cw;
            us[a * LDU + j] = ublk[(int64_t)a * n2 + j0 + j];
        }
        __syncthreads();
        if (!live) continue;
        const T *u = us + threadIdx.x * LDU;
        int j = 0;
        if constexpr (sizeof(T) == 4) {
            if ((n2 & 3) == 0)
                for (; j < cw; j += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(u + j);
                    const int jz = j0 + j;
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        if (c < nrhs)
                            d[c] -= v.x * zs[jz * nrhs + c] + v.y * zs[(jz + 1) * nrhs + c] +
                                    v.z * zs[(jz + 2) * nrhs + c] + v.w * zs[(jz + 3) * nrhs + c];
                }
        }
        for (; j < cw; ++j) {
            const T uj = u[j];
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (c < nrhs) d[c] -= uj * zs[(j0 + j) * nrhs + c];
        }
    }
    if (!live) return;
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (c < nrhs) {
            const double upd = nrm[c] * (double)d[c];
            x[c * ld + gi] = accumulate ? x[c * ld + gi] + upd : upd;
        }
}

// One right-hand side: zeta and omega of the partition (2r <= NQ values) sit
// in registers and every thread streams RPT rows (the shared-memory reads of
// the general kernel made it issue-bound).  Same arithmetic order.
template <typename T, int NQ>
__global__ void __launch_bounds__(RBS)
    k_retrieve1(const T *__restrict__ Gv, const T *__restrict__ Ucat, const double *__restrict__ zr, Parts P,
                int r, int64_t n, const double *__restrict__ nrm, double *__restrict__ x, int accumulate,
                const int *skip) {
    if (skip && *skip) return;
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int n2 = 2 * r;
    T z[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        double v = 0.0;
        if (j < r) { if (part <= P.p - 2) v = zr[(int64_t)part * n2 + j]; }
        else if (j < n2 && part >= 1) v = zr[(int64_t)(part - 1) * n2 + j];
        z[j] = (T)v;
    }
    const double sc = nrm[0];
    for (int64_t row = blockIdx.x * (int64_t)RBS + threadIdx.x; row < ni; row += (int64_t)gridDim.x * RBS) {
        const int64_t gi = s + row;
        const T d = retrieve_row<T, NQ>(Gv[gi], Ucat + gi * n2, z, n2);
        x[gi] = retrieve_update(accumulate ? x[gi] : 0.0, sc, (double)d, accumulate);
    }
}

// ---------------------------------------------------------------------------
// a = U^T h per partition: alpha_i = u_{T,i}^T h_i -> interface i, rows 0..r-1;
// beta_i = u_{W,i}^T h_i -> interface i-1, rows r..2r-1.
template <typename T>
__global__ void k_project_t(const T *__restrict__ Ucat, Parts P, int r, int64_t n,
                            const double *__restrict__ hin, const double *__restrict__ inv, int nrhs,
                            double *__restrict__ psi) {
    extern __shared__ double red[];
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int n2 = 2 * r, O = n2 * nrhs;
    auto put = [&](int o, double v) {
        const int j = o / nrhs, c = o % nrhs;
        if (j < r) { if (part <= P.p - 2) psi[((int64_t)part * n2 + j) * nrhs + c] = v; }
        else if (part >= 1) psi[((int64_t)(part - 1) * n2 + j) * nrhs + c] = v;
    };
    auto dot = [&](int o, int64_t r0, int64_t step) {
        const int j = o / nrhs, c = o % nrhs;
        double acc = 0.0;
        for (int64_t row = r0; row < ni; row += step)
            acc += (double)(Ucat[(s + row) * n2 + j] * (T)(hin[c * n + s + row] * inv[c]));
        return acc;
    };
    if (O <= (int)blockDim.x) {
        const int groups = blockDim.x / O;
        const int g = threadIdx.x / O, o = threadIdx.x % O;
        if (g < groups) red[g * O + o] = dot(o, g, groups);
        __syncthreads();
        if ((int)threadIdx.x < O) {
            double acc = 0.0;
            for (int q = 0; q < groups; ++q) acc += red[q * O + threadIdx.x];
            put(threadIdx.x, acc);
        }
    } else {
        for (int o = threadIdx.x; o < O; o += blockDim.x) put(o, dot(o, 0, 1));
    }
}

template <typename T, int KB, Split S>
__device__ void dstage_t_body(const T *__restrict__ LT, const T *__restrict__ UT, const T *__restrict__ DI,
                              const T *__restrict__ PQ, Parts P, int k, int r, int64_t n,
                              const double *__restrict__ hin, const double *__restrict__ inv,
                              const double *__restrict__ zr, int nrhs, T *__restrict__ Yv,
                              const double *__restrict__ nrm, double *__restrict__ x, int64_t ldx,
                              int accumulate, unsigned char *smem_raw) {
    constexpr int NT = Geo<KB>::NT, LDS = KB + 1;
    T *Ta = reinterpret_cast<T *>(smem_raw);   // tile buffer 0
    T *Tb = Ta + KB * LDS;                     // tile buffer 1
    T *Tt = Tb + KB * LDS;
    T *Zp = Tt + KB * nrhs;
    T *corr = Zp + KB * nrhs;                  // [2][KB][nrhs]: top / bottom tip corrections
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int pm = KB * nrhs, n2 = 2 * r;
    // y = h - V^T w: top rows get P_{part-1}^T w_zeta(part-1), bottom rows Q_{part+1}^T w_omega(part)
    for (int e = threadIdx.x; e < 2 * pm; e += NT) {
        const int side = e / pm, rem = e % pm, q = rem / nrhs, c = rem % nrhs;
        double acc = 0.0;
        if (q < k && r > 0) {
            if (side == 0 && part >= 1) {
                const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * KB;
                for (int j = 0; j < r; ++j)
                    acc += (double)Pm[j * KB + q] * zr[((int64_t)(part - 1) * n2 + j) * nrhs + c];
            } else if (side == 1 && part <= P.p - 2) {
                const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * KB;
                for (int j = 0; j < r; ++j)
                    acc += (double)Qm[j * KB + q] * zr[((int64_t)part * n2 + r + j) * nrhs + c];
            }
        }
        corr[e] = (T)acc;
    }
    __syncthreads();
    // forward with U^T, carrying z^ = D z
    for (int J = 0; J < nb; ++J) {
        T *Ucur = (J & 1) ? Tb : Ta;
        T *Uprev = (J & 1) ? Ta : Tb;
        load_tile<T, KB>(UT + (b0 + J) * KB * KB, Ucur, LDS);
        for (int e = threadIdx.x; e < pm; e += NT) {
            const int a = e / nrhs, c = e % nrhs;
            const int64_t row = (int64_t)J * KB + a;
            T v = T(0);
            if (row < ni) {
                v = (T)(hin[c * n + s + row] * inv[c]);
                if (row < k) v -= corr[row * nrhs + c];
                if (row >= ni - k) v -= corr[pm + (row - (ni - k)) * nrhs + c];
            }
            Tt[e] = v;
        }
        __syncthreads();
        fwdT_step<T, KB, S>(Uprev, Ucur, LDS, Tt, Zp, nrhs, nrhs, J == 0);
        for (int e = threadIdx.x; e < pm; e += NT) {
            const int a = e / nrhs, c = e % nrhs;
            const int64_t row = (int64_t)J * KB + a;
            if (row < ni) Yv[c * n + s + row] = Zp[e] * DI[(b0 + J) * KB + a];
        }
    }
    __syncthreads();
    // backward with L^T
    for (int J = nb - 1; J >= 0; --J) {
        T *Lcur = (J & 1) ? Tb : Ta;
        T *Lnext = (J & 1) ? Ta : Tb;
        load_tile<T, KB>(LT + (b0 + J) * KB * KB, Lcur, LDS);
        for (int e = threadIdx.x; e < pm; e += NT) {
            const int a = e / nrhs, c = e % nrhs;
            const int64_t row = (int64_t)J * KB + a;
            Tt[e] = (row < ni) ? Yv[c * n + s + row] : T(0);
        }
        __syncthreads();
        bwdT_step<T, KB, S>(Lnext, Lcur, LDS, Tt, Zp, nrhs, nrhs, J == nb - 1);
        for (int e = threadIdx.x; e < pm; e += NT) {
            const int a = e / nrhs, c = e % nrhs;
            const int64_t row = (int64_t)J * KB + a;
            if (row < ni) {
                const double upd = nrm[c] * (double)Zp[e];
                const int64_t xi = c * ldx + s + row;
                x[xi] = accumulate ? x[xi] + upd : upd;
            }
        }
    }
}

template <typename T, int KB>
__global__ void __launch_bounds__(Geo<KB>::NT)
    k_dstage_t(const T *__restrict__ LT, const T *__restrict__ UT, const T *__restrict__ DI,
               const T *__restrict__ PQ, Parts P, int k, int r, int64_t n, const double *__restrict__ hin,
               const double *__restrict__ inv, const double *__restrict__ zr, int nrhs, T *__restrict__ Yv,
               const double *__restrict__ nrm, double *__restrict__ x, int64_t ldx, int accumulate,
               const int *skip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (skip && *skip) return;
    if (nrhs < 4)
        dstage_t_body<T, KB, Split::DOTS>(LT, UT, DI, PQ, P, k, r, n, hin, inv, zr, nrhs, Yv, nrm, x, ldx,
                                          accumulate, smem_raw);
    else
        dstage_t_body<T, KB, Split::COLS>(LT, UT, DI, PQ, P, k, r, n, hin, inv, zr, nrhs, Yv, nrm, x, ldx,
                                          accumulate, smem_raw);
}

// ---------------------------------------------------------------------------
static inline unsigned row_blocks(int64_t n) { return (unsigned)((n + RBS - 1) / RBS); }

template <int NR>
static bool residual_nr(Ctx *c, const double *f, const double *x, int64_t ld, int nrhs, bool trans,
                        bool xz) {
    return launch(c, KID_RESIDUAL, [&] {
        k_residual<NR><<<row_blocks(c->n), RBS, 0, c->stream>>>(
            c->band, c->ld, c->k, c->n, f, x, ld, nrhs, trans, xz, c->rv, c->partial, c->counter,
            c->nrm + c->opt.max_nrhs, c->nrm + 2 * c->opt.max_nrhs, c->diag_list, c->ndiag, c->stop);
    });
}

// Launches the residual kernel on caller-provided scratch (per-CTA partial
// sums and the ticket counter); no handle involved.
bool launch_residual_raw(const double *band, int64_t ldb, int k, int64_t n, const double *f,
                         const double *x, int64_t ld, int nrhs, double *r, double *partial,
                         unsigned *counter, double *nrm, cudaStream_t st) {
    const unsigned g = row_blocks(n);
    switch (nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16) {
        case 1: k_residual<1><<<g, RBS, 0, st>>>(band, ldb, k, n, f, x, ld, nrhs, 0, 0, r, partial, counter, nrm, nullptr, nullptr, 0, StopRule()); break;
        case 2: k_residual<2><<<g, RBS, 0, st>>>(band, ldb, k, n, f, x, ld, nrhs, 0, 0, r, partial, counter, nrm, nullptr, nullptr, 0, StopRule()); break;
        case 4: k_residual<4><<<g, RBS, 0, st>>>(band, ldb, k, n, f, x, ld, nrhs, 0, 0, r, partial, counter, nrm, nullptr, nullptr, 0, StopRule()); break;
        case 8: k_residual<8><<<g, RBS, 0, st>>>(band, ldb, k, n, f, x, ld, nrhs, 0, 0, r, partial, counter, nrm, nullptr, nullptr, 0, StopRule()); break;
        default: k_residual<16><<<g, RBS, 0, st>>>(band, ldb, k, n, f, x, ld, nrhs, 0, 0, r, partial, counter, nrm, nullptr, nullptr, 0, StopRule()); break;
    }
    return cudaGetLastError() == cudaSuccess;
}

bool run_residual(Ctx *c, const double *f, const double *x, int64_t ld, int nrhs, bool trans, bool xz) {
    if (nrhs <= 1) return residual_nr<1>(c, f, x, ld, nrhs, trans, xz);
    if (nrhs <= 2) return residual_nr<2>(c, f, x, ld, nrhs, trans, xz);
    if (nrhs <= 4) return residual_nr<4>(c, f, x, ld, nrhs, trans, xz);
    if (nrhs <= 8) return residual_nr<8>(c, f, x, ld, nrhs, trans, xz);
    return residual_nr<16>(c, f, x, ld, nrhs, trans, xz);
}

template <int NR>
static bool sumsq_nr(Ctx *c, const double *v, int64_t ld, int nrhs, double *out, double *inv) {
    return launch(c, KID_NORM, [&] {
        k_sumsq<NR><<<row_blocks(c->n), RBS, 0, c->stream>>>(v, ld, c->n, nrhs, c->partial, c->counter,
                                                            out, inv);
    });
}

bool run_norms(Ctx *c, const double *v, int64_t ld, int nrhs, double *out) {
    if (nrhs <= 1) return sumsq_nr<1>(c, v, ld, nrhs, out, nullptr);
    if (nrhs <= 2) return sumsq_nr<2>(c, v, ld, nrhs, out, nullptr);
    if (nrhs <= 4) return sumsq_nr<4>(c, v, ld, nrhs, out, nullptr);
    if (nrhs <= 8) return sumsq_nr<8>(c, v, ld, nrhs, out, nullptr);
    return sumsq_nr<16>(c, v, ld, nrhs, out, nullptr);
}

template <typename T, int KB, int NBUF>
static size_t dstage_smem(int nrhs) {
    return (size_t)NBUF * KB * nrhs * sizeof(double) +
           ((size_t)NBUF * KB * ds_ldp<T, KB>() + NBUF * KB + 3 * KB * nrhs) * sizeof(T);
}

template <typename T, int KB, int NBUF>
static bool dstage_launch(Ctx *c, const double *rin, int nrhs, const double *inv) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = dstage_smem<T, KB, NBUF>(nrhs);
    auto kern = k_dstage<T, KB, NBUF>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_DSTAGE, [&] {
        kern<<<c->p, Geo<KB>::NT, smem, c->stream>>>((const T *)c->LT, (const T *)c->UT, (const T *)c->DI,
                                                     (const T *)c->PQ, P, c->k, c->r, c->n, rin, inv, nrhs,
                                                     (T *)c->Yv, (T *)c->Gv, c->psi, c->skip);
    });
}

// Four stage buffers (three steps of factor tiles in flight) while two CTAs
// still fit on an SM; two otherwise.
template <typename T, int KB>
static bool dstage_impl(Ctx *c, const double *rin, int nrhs, const double *inv) {
    if (dstage_smem<T, KB, 4>(nrhs) <= 110 * 1024) return dstage_launch<T, KB, 4>(c, rin, nrhs, inv);
    return dstage_launch<T, KB, 2>(c, rin, nrhs, inv);
}

template <typename T, int KB>
static bool dstage_t_impl(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, int acc) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (2 * KB * (KB + 1) + 4 * KB * nrhs) * sizeof(T);
    auto kern = k_dstage_t<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_DSTAGE_T, [&] {
        kern<<<c->p, Geo<KB>::NT, smem, c->stream>>>((const T *)c->LT, (const T *)c->UT, (const T *)c->DI,
                                                     (const T *)c->PQ, P, c->k, c->r, c->n, hin,
                                                     c->nrm + 2 * c->opt.max_nrhs, c->zr, nrhs, (T *)c->Yv,
                                                     c->nrm + c->opt.max_nrhs, x, ldx, acc, c->skip);
    });
}

template <typename T, int NQ>
static bool retrieve1_nq(Ctx *c, double *x, int acc) {
    Parts P{c->off_d, c->boff_d, c->p};
    constexpr int RPT = 8;  // rows per thread
    dim3 grid((unsigned)((c->maxni + RBS * RPT - 1) / (RBS * RPT)), c->p);
    return launch(c, KID_RETRIEVE, [&] {
        k_retrieve1<T, NQ><<<grid, RBS, 0, c->stream>>>((const T *)c->Gv, (const T *)c->Ucat, c->zr, P, c->r, c->n,
                                                        c->nrm + c->opt.max_nrhs, x, acc, c->skip);
    });
}

template <typename T>
static bool retrieve_impl(Ctx *c, double *x, int64_t ld, int nrhs, int acc) {
    if (nrhs == 1) {
        const int n2 = 2 * c->r;
        if (n2 <= 8) return retrieve1_nq<T, 8>(c, x, acc);
        if (n2 <= 16) return retrieve1_nq<T, 16>(c, x, acc);
        if (n2 <= 32) return retrieve1_nq<T, 32>(c, x, acc);
        if (n2 <= 64) return retrieve1_nq<T, 64>(c, x, acc);
        return retrieve1_nq<T, 128>(c, x, acc);
    }
    Parts P{c->off_d, c->boff_d, c->p};
    dim3 grid(row_blocks(c->maxni), c->p);
    const size_t smem = retrieve_smem<T>(2 * c->r, nrhs);
    for (auto kern : {k_retrieve<T, 4>, k_retrieve<T, 8>, k_retrieve<T, 16>})
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_RETRIEVE, [&] {
        if (nrhs <= 4)
            k_retrieve<T, 4><<<grid, RBS, smem, c->stream>>>((const T *)c->Gv, (const T *)c->Ucat, c->zr, P, c->r,
                                                            c->n, nrhs, c->nrm + c->opt.max_nrhs, x, ld, acc, c->skip);
        else if (nrhs <= 8)
            k_retrieve<T, 8><<<grid, RBS, smem, c->stream>>>((const T *)c->Gv, (const T *)c->Ucat, c->zr, P, c->r,
                                                            c->n, nrhs, c->nrm + c->opt.max_nrhs, x, ld, acc, c->skip);
        else
            k_retrieve<T, 16><<<grid, RBS, smem, c->stream>>>((const T *)c->Gv, (const T *)c->Ucat, c->zr, P,
                                                             c->r, c->n, nrhs, c->nrm + c->opt.max_nrhs, x, ld, acc, c->skip);
    });
}

template <typename T>
static bool project_t_impl(Ctx *c, const double *hin, int nrhs) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (size_t)256 * sizeof(double) + (size_t)2 * c->r * nrhs * sizeof(double);
    return launch(c, KID_PROJECT_T, [&] {
        k_project_t<T><<<c->p, 256, smem, c->stream>>>((const T *)c->Ucat, P, c->r, c->n, hin,
                                                      c->nrm + 2 * c->opt.max_nrhs, nrhs, c->psi);
    });
}

bool run_dstage_inv(Ctx *c, const double *rin, int nrhs, const double *inv) {
    if (c->wide) return run_wide_dstage_inv(c, rin, nrhs, inv);
    if (c->fp64) {
        switch (c->KB) {
            case 8: return dstage_impl<double, 8>(c, rin, nrhs, inv);
            case 16: return dstage_impl<double, 16>(c, rin, nrhs, inv);
            case 32: return dstage_impl<double, 32>(c, rin, nrhs, inv);
            default: return dstage_impl<double, 64>(c, rin, nrhs, inv);
        }
    }
    switch (c->KB) {
        case 8: return dstage_impl<float, 8>(c, rin, nrhs, inv);
        case 16: return dstage_impl<float, 16>(c, rin, nrhs, inv);
        case 32: return dstage_impl<float, 32>(c, rin, nrhs, inv);
        default: return dstage_impl<float, 64>(c, rin, nrhs, inv);
    }
}

bool run_dstage(Ctx *c, const double *rin, int64_t, int nrhs) {
    if (c->wide) return run_wide_dstage(c, rin, nrhs);
    if (c->opt.pivoting) return run_dstage_piv(c, rin, nrhs);
    return run_dstage_inv(c, rin, nrhs, c->nrm + 2 * c->opt.max_nrhs);
}

bool run_dstage_t(Ctx *c, const double *hin, int64_t, double *x, int64_t ldx, int nrhs, bool accumulate) {
    if (c->wide) return run_wide_dstage_t(c, hin, x, ldx, nrhs, accumulate);
    if (c->opt.pivoting) return run_dstage_t_piv(c, hin, x, ldx, nrhs, accumulate);
    const int acc = accumulate ? 1 : 0;
    if (c->fp64) {
        switch (c->KB) {
            case 8: return dstage_t_impl<double, 8>(c, hin, x, ldx, nrhs, acc);
            case 16: return dstage_t_impl<double, 16>(c, hin, x, ldx, nrhs, acc);
            case 32: return dstage_t_impl<double, 32>(c, hin, x, ldx, nrhs, acc);
            default: return dstage_t_impl<double, 64>(c, hin, x, ldx, nrhs, acc);
        }
    }
    switch (c->KB) {
        case 8: return dstage_t_impl<float, 8>(c, hin, x, ldx, nrhs, acc);
        case 16: return dstage_t_impl<float, 16>(c, hin, x, ldx, nrhs, acc);
        case 32: return dstage_t_impl<float, 32>(c, hin, x, ldx, nrhs, acc);
        default: return dstage_t_impl<float, 64>(c, hin, x, ldx, nrhs, acc);
    }
}

bool run_retrieve(Ctx *c, double *x, int64_t ld, int nrhs, bool accumulate) {
    const int acc = accumulate ? 1 : 0;
    return c->fp64 ? retrieve_impl<double>(c, x, ld, nrhs, acc) : retrieve_impl<float>(c, x, ld, nrhs, acc);
}

bool run_project_t(Ctx *c, const double *hin, int64_t, int nrhs) {
    if (c->p < 2 || c->r == 0) return true;
    return c->fp64 ? project_t_impl<double>(c, hin, nrhs) : project_t_impl<float>(c, hin, nrhs);
}

bool fused_retrieve_ok(const Ctx *c, int nrhs, bool trans) {
    return c->xalt && nrhs == 1 && !trans && !c->otf && !c->wide && !c->opt.pivoting;
}

bool apply_precond_deferred(Ctx *c, const double *in, int nrhs) {
    return run_dstage(c, in, c->n, nrhs) && run_reduced_solve(c, nrhs, false);
}

template <typename T, int NQ>
static bool residual_ret_nq(Ctx *c, const double *f, const double *x_in, double *x_out) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (size_t)(RBS + 2 * c->k) * sizeof(double);
    return launch(c, KID_RESIDUAL, [&] {
        k_residual_ret<T, NQ><<<row_blocks(c->n), RBS, smem, c->stream>>>(
            c->band, c->ld, c->k, c->n, f, x_in, x_out, (const T *)c->Gv, (const T *)c->Ucat, c->zr, P, c->r,
            c->nrm + c->opt.max_nrhs, c->rv, c->partial, c->counter, c->nrm + c->opt.max_nrhs,
            c->nrm + 2 * c->opt.max_nrhs);
    });
}

template <typename T>
static bool residual_ret_impl(Ctx *c, const double *f, const double *x_in, double *x_out) {
    const int n2 = 2 * c->r;
    if (n2 <= 8) return residual_ret_nq<T, 8>(c, f, x_in, x_out);
    if (n2 <= 16) return residual_ret_nq<T, 16>(c, f, x_in, x_out);
    if (n2 <= 32) return residual_ret_nq<T, 32>(c, f, x_in, x_out);
    return residual_ret_nq<T, 64>(c, f, x_in, x_out);
}

bool run_residual_retrieve(Ctx *c, const double *f, const double *x_in, double *x_out) {
    return c->fp64 ? residual_ret_impl<double>(c, f, x_in, x_out) : residual_ret_impl<float>(c, f, x_in, x_out);
}

bool apply_precond(Ctx *c, const double *in, double *out, int64_t ldo, int nrhs, bool trans, bool accumulate) {
    if (c->otf && !trans) return apply_otf(c, in, out, ldo, nrhs, accumulate);
    if (!trans) {
        if (!run_dstage(c, in, c->n, nrhs)) return false;
        if (!run_reduced_solve(c, nrhs, false)) return false;
        return run_retrieve(c, out, ldo, nrhs, accumulate);
    }
    if (!run_project_t(c, in, c->n, nrhs)) return false;
    if (!run_reduced_solve(c, nrhs, true)) return false;
    return run_dstage_t(c, in, c->n, out, ldo, nrhs, accumulate);
}

}  // namespace lrs
