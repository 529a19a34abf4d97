// Partial pivoting inside each partition (the weakly dominant systems of
// section 4.2, where the paper's direct solver pivots; row exchanges never
// cross a partition, so the coupling blocks B_i, C_i and the whole SPIKE
// structure are those of the unpivoted matrix).
//
// Factorisation of A_i: LAPACK's banded order (gbtf2) in blocks of KB >= k
// columns.  For column j the pivot candidates are rows j..j+k; with KB >= k
// they lie in block rows J and J+1, so block step J eliminates the KB columns
// of block J inside the 2KB x 3KB window [block rows J, J+1] x [column blocks
// J, J+1, J+2].  Rows exchanged upwards carry their entries up to 2k columns
// right of the diagonal: the upper factor grows to block J+2.  The pivot is
// the candidate of largest magnitude; ties go to the row in the lowest
// current position, as in gbtf2.  Per block J the library keeps
//   pi_J     gather permutation of the 2KB stacked rows (new a <- old pi_J[a])
//   L_JJ^{-1}, L_{J+1,J}, U_JJ^{-1}, U_{J,J+1}, U_{J,J+2}   (KB x KB each)
// so that one forward step is  [y_J; y_{J+1}] <- pi_J [y_J; y_{J+1}],
// y_J <- L_JJ^{-1} y_J,  y_{J+1} -= L_{J+1,J} y_J,  and one backward step is
// x_J = U_JJ^{-1}(y_J - U_{J,J+1} x_{J+1} - U_{J,J+2} x_{J+2}).
//
// Kernels:
//   k_band_lu_piv   one CTA per partition; the window lives in registers,
//                   one row per group of H threads (rows never move between
//                   threads: the exchanges are kept as positions)
//   k_sweep_piv     spikes X <- A_i^{-1} X in place, W columns per CTA
//   k_dstage_piv    g = A_i^{-1}(r / |r|) and the psi epilogue
//   k_dstage_t_piv  the transposed D-stage of M^{-T}
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace lrs {

namespace {

// ---------------------------------------------------------------------------
// factorisation
// Three threads per window row: group 0 updates the row's KB panel columns,
// which stay in shared memory (the pivot search reads them there), groups 1
// and 2 hold the row's 2KB trailing columns in registers (their rank-1 updates
// never need a column mask).

template <typename T, int KB> struct PivLU {
    static constexpr int H = 3;
    static constexpr int R2 = 2 * KB;     // window rows
    static constexpr int WC = 3 * KB;     // window columns
    static constexpr int NT = R2 * H;     // threads
    static constexpr int CPT = WC / H;    // window columns per thread
    static constexpr int LDS = WC + 16 / (int)sizeof(T);  // shared row stride (16-byte rows)
    static constexpr int VW = 16 / (int)sizeof(T);  // vector width of a 16-byte load
    // FP32: the next block row of the band is prefetched (raw FP64) while the
    // current block is eliminated; FP64 has no shared memory left for it
    static constexpr bool PREFETCH = sizeof(T) == 4;
    static constexpr int RB = PREFETCH ? (2 * KB + 1) * KB : 0;  // raw band doubles
    static constexpr size_t smem_bytes = (size_t)R2 * LDS * sizeof(T) + (size_t)RB * sizeof(double) +
                                         (4 * KB + 2 * KB) * sizeof(T) + 2 * R2 * (sizeof(unsigned long long) + sizeof(unsigned)) +
                                         R2 * sizeof(int);
    static_assert(CPT % VW == 0, "columns per thread must fill vector loads");
};

__device__ __forceinline__ float abs_t(float v) { return fabsf(v); }
__device__ __forceinline__ double abs_t(double v) { return fabs(v); }

template <typename T> __device__ __forceinline__ bool pivot_ok(T v) { return isfinite(v) && abs_t(v) > T(0); }

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Block row b of A_i (local rows b*KB ..) as (band row d, column c) pairs:
// row = b*KB + c, column = row + k - d, window column = column - J*KB.
// Consecutive c are consecutive band addresses (coalesced).
struct BandRowMap {
    int64_t row, col, wcol;
    bool inside;  // row and column inside the partition
};
template <int KB>
__device__ __forceinline__ BandRowMap band_row_map(int e, int k, int64_t ni, int b, int J) {
    const int d = e / KB, c = e % KB;
    BandRowMap m;
    m.row = (int64_t)b * KB + c;
    m.col = m.row + k - d;
    m.wcol = m.col - (int64_t)J * KB;
    m.inside = m.row < ni && m.col >= 0 && m.col < ni;
    return m;
}

// Scatters block row b into window rows wr0 .. wr0+KB-1 (already zero).
// Rows past the partition are identity rows (the padding).  src(e) gives
// the band value of pair e when it is inside the partition.
template <typename T, int KB, typename Src>
__device__ void put_block_row(int k, int64_t ni, int b, int J, T *S, int wr0, Src &&src) {
    using G = PivLU<T, KB>;
    for (int e = threadIdx.x; e < (2 * k + 1) * KB; e += G::NT) {
        const BandRowMap m = band_row_map<KB>(e, k, ni, b, J);
        const int c = e % KB, d = e / KB;
        if (m.wcol < 0 || m.wcol >= G::WC) continue;
        if (m.inside) S[(wr0 + c) * G::LDS + m.wcol] = (T)src(e, m);
        else if (m.row >= ni && d == k) S[(wr0 + c) * G::LDS + m.wcol] = T(1);
    }
}

template <typename T, int KB>
__global__ void __launch_bounds__(PivLU<T, KB>::NT)
    k_band_lu_piv(const double *__restrict__ band, int64_t ld, int k, Parts P, T *__restrict__ PF,
                  unsigned char *__restrict__ PIV, int64_t *__restrict__ status) {
    using G = PivLU<T, KB>;
    constexpr int R2 = G::R2, WC = G::WC, CPT = G::CPT, LDS = G::LDS, NT = G::NT, VW = G::VW;
    constexpr int TT = KB * KB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);                       // [R2][LDS] window at final positions
    double *Rb = reinterpret_cast<double *>(S + R2 * LDS);        // [2k+1][KB] prefetched band (FP32 only)
    T *rowp = reinterpret_cast<T *>(Rb + G::RB);                  // [2][2KB] trailing part of the pivot row
    T *pinvs = rowp + 4 * KB;                                     // [KB] 1 / pivot of column j
    T *dinv = pinvs + KB;                                         // [KB] 1 / U_jj
    unsigned long long *khi = reinterpret_cast<unsigned long long *>(dinv + KB);  // [2][R2] |value| bits
    unsigned *klo = reinterpret_cast<unsigned *>(khi + 2 * R2);   // [2][R2] (0xffff - position) << 16 | row
    int *rowAt = reinterpret_cast<int *>(klo + 2 * R2);           // [R2] window row at final position q

    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int i = threadIdx.x % R2, h = threadIdx.x / R2;
    const int lane = threadIdx.x & 31;
    auto from_band = [&](int e, const BandRowMap &m) { return band[(int64_t)(e / KB) * ld + s + m.col]; };
    // pivot search key of a row: larger |value| first, then lower position;
    // finished rows get 0 (below every candidate, including a zero value)
    auto put_key = [&](int buf, T v, int mypos, bool done) {
        unsigned long long hi = 0;
        unsigned lo = 0;
        if (!done) {
            const T av = isnan(v) ? T(INFINITY) : abs_t(v);
            if constexpr (sizeof(T) == 4) hi = (unsigned long long)__float_as_uint(av);
            else hi = (unsigned long long)__double_as_longlong(av);
            lo = ((0xffffu - (unsigned)mypos) << 16) | (unsigned)i;
        }
        khi[buf * R2 + i] = hi;
        klo[buf * R2 + i] = lo;
    };

    for (int e = threadIdx.x; e < R2 * LDS; e += NT) S[e] = T(0);
    __syncthreads();
    put_block_row<T, KB>(k, ni, 0, 0, S, 0, from_band);
    put_block_row<T, KB>(k, ni, 1, 0, S, KB, from_band);
    __syncthreads();
    T a[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) a[q] = S[i * LDS + h * CPT + q];

    for (int J = 0; J < nb; ++J) {
        if constexpr (G::PREFETCH) {
            // block row J+2 of the band lands in Rb while block J is eliminated
            if (J + 1 < nb) {
                for (int e = threadIdx.x; e < (2 * k + 1) * KB; e += NT) {
                    const BandRowMap m = band_row_map<KB>(e, k, ni, J + 2, J + 1);
                    if (m.inside) cp_async8(Rb + e, band + (int64_t)(e / KB) * ld + s + m.col);
                }
            }
            cp_async_commit_all();
        }
        bool done = false;
        int mystep = KB, mypos = i;  // positions are tracked by every thread of the row
        T *prow = S + i * LDS;       // the row's panel columns
        if (h == 0) put_key(0, prow[0], mypos, false);
        for (int j = 0; j < KB; ++j) {
            const int buf = j & 1;
            __syncthreads();
            // pivot search, repeated by every warp
            unsigned long long bh = 0;
            unsigned bl = 0;
            for (int q = lane; q < R2; q += 32) {
                const unsigned long long vh = khi[buf * R2 + q];
                const unsigned vl = klo[buf * R2 + q];
                if (vh > bh || (vh == bh && vl > bl)) { bh = vh; bl = vl; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long oh = __shfl_xor_sync(0xffffffffu, bh, o);
                const unsigned ol = __shfl_xor_sync(0xffffffffu, bl, o);
                if (oh > bh || (oh == bh && ol > bl)) { bh = oh; bl = ol; }
            }
            const int p = (int)(bl & 0xffffu), pos_p = 0xffff - (int)(bl >> 16);
            const T piv = S[p * LDS + j];
            const bool ok = pivot_ok<T>(piv);
            const T pinv = ok ? T(1) / piv : T(1);
            if (i == p && h > 0) {
                T *dst = rowp + buf * 2 * KB + (h - 1) * KB;
#pragma unroll
                for (int g = 0; g < CPT / VW; ++g) {
                    if constexpr (VW == 4)
                        *reinterpret_cast<float4 *>(dst + 4 * g) = make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
                    else
                        *reinterpret_cast<double2 *>(dst + 2 * g) = make_double2(a[2 * g], a[2 * g + 1]);
                }
            }
            // gbtf2's row exchange: the row at position j moves to p's position
            if (i == p) {
                done = true;
                mystep = j;
                mypos = j;
            } else if (mypos == j) {
                mypos = pos_p;
            }
            if (threadIdx.x == 0) {
                if (!ok) atomicMin((unsigned long long *)status, (unsigned long long)(s + (int64_t)J * KB + j));
                pinvs[j] = pinv;
            }
            __syncthreads();
            // rank-1 update right of column j; the multiplier stays unscaled in
            // column j and is scaled when the window is written out
            const T m = done ? T(0) : prow[j] * pinv;
            if (h == 0) {
                if (!done) {
                    const T *pr = S + p * LDS;
                    int l = j + 1;
                    for (; l < KB && (l % VW) != 0; ++l) prow[l] -= m * pr[l];
                    for (; l < KB; l += VW) {
                        if constexpr (VW == 4) {
                            float4 x = *reinterpret_cast<const float4 *>(prow + l);
                            const float4 y = *reinterpret_cast<const float4 *>(pr + l);
                            x.x -= m * y.x; x.y -= m * y.y; x.z -= m * y.z; x.w -= m * y.w;
                            *reinterpret_cast<float4 *>(prow + l) = x;
                        } else {
                            double2 x = *reinterpret_cast<const double2 *>(prow + l);
                            const double2 y = *reinterpret_cast<const double2 *>(pr + l);
                            x.x -= m * y.x; x.y -= m * y.y;
                            *reinterpret_cast<double2 *>(prow + l) = x;
                        }
                    }
                }
                if (j + 1 < KB) put_key(buf ^ 1, prow[j + 1], mypos, done);
            } else {
                const T *up = rowp + buf * 2 * KB + (h - 1) * KB;
#pragma unroll
                for (int g = 0; g < CPT / VW; ++g) {
                    if constexpr (VW == 4) {
                        const float4 u = *reinterpret_cast<const float4 *>(up + 4 * g);
                        a[4 * g] -= m * u.x;
                        a[4 * g + 1] -= m * u.y;
                        a[4 * g + 2] -= m * u.z;
                        a[4 * g + 3] -= m * u.w;
                    } else {
                        const double2 u = *reinterpret_cast<const double2 *>(up + 2 * g);
                        a[2 * g] -= m * u.x;
                        a[2 * g + 1] -= m * u.y;
                    }
                }
            }
        }
        __syncthreads();
        // window rows to their final positions; multipliers scaled by 1/pivot
        if (h == 0) {
#pragma unroll
            for (int q = 0; q < CPT; ++q) a[q] = (q < mystep) ? prow[q] * pinvs[q] : prow[q];
            rowAt[mypos] = i;
        }
        __syncthreads();
        {
            T *dst = S + mypos * LDS + h * CPT;
#pragma unroll
            for (int g = 0; g < CPT / VW; ++g) {
                if constexpr (VW == 4)
                    *reinterpret_cast<float4 *>(dst + 4 * g) = make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
                else
                    *reinterpret_cast<double2 *>(dst + 2 * g) = make_double2(a[2 * g], a[2 * g + 1]);
            }
        }
        __syncthreads();
        const int64_t g = b0 + J;
        T *F = PF + g * 5 * TT;
        for (int e = threadIdx.x; e < TT; e += NT) {
            const int r = e / KB, c = e % KB;
            F[1 * TT + e] = S[(KB + r) * LDS + c];           // L_{J+1,J}
            F[3 * TT + e] = S[r * LDS + KB + c];             // U_{J,J+1}
            F[4 * TT + e] = S[r * LDS + 2 * KB + c];         // U_{J,J+2}
        }
        if (threadIdx.x < R2) PIV[g * R2 + threadIdx.x] = (unsigned char)rowAt[threadIdx.x];
        if (threadIdx.x < KB) {
            const T d = S[threadIdx.x * LDS + threadIdx.x];
            dinv[threadIdx.x] = pivot_ok<T>(d) ? T(1) / d : T(1);
        }
        __syncthreads();
        // triangular inverses, written over the L_{J+1,J} block (L^{-1}) and
        // the U_{J,J+1} block (U^{-1}) of S
        if constexpr (sizeof(T) == 4) {
            // one column per thread, the column held in registers (the window's
            // registers are free until the next block is loaded)
            if (threadIdx.x < 2 * KB) {
                const int c = threadIdx.x % KB;
                T x[KB];
                if (threadIdx.x < KB) {  // L^{-1}, unit lower: x_r = -sum_{b<r} L_rb x_b
#pragma unroll
                    for (int r = 0; r < KB; ++r) {
                        T s4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
                        for (int b = 0; b < r; ++b) s4[b & 3] += S[r * LDS + b] * x[b];
                        x[r] = (r == c) ? T(1) : -((s4[0] + s4[1]) + (s4[2] + s4[3]));
                    }
#pragma unroll
                    for (int r = 0; r < KB; ++r) S[(KB + r) * LDS + c] = x[r];
                } else {  // U^{-1}: x_r = -(sum_{b>r} U_rb x_b) / U_rr
#pragma unroll
                    for (int r = KB - 1; r >= 0; --r) {
                        T s4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
                        for (int b = r + 1; b < KB; ++b) s4[b & 3] += S[r * LDS + b] * x[b];
                        x[r] = (r > c) ? T(0) : (r == c) ? dinv[c] : -((s4[0] + s4[1]) + (s4[2] + s4[3])) * dinv[r];
                    }
#pragma unroll
                    for (int r = 0; r < KB; ++r) S[r * LDS + KB + c] = x[r];
                }
            }
        } else {
            // FP64 (register budget of 512 threads): four lanes per column
            const int quad = threadIdx.x >> 2, l4 = threadIdx.x & 3;
            const unsigned qmask = 0xFu << (lane & ~3);
            constexpr int NQ = NT / 4;
            for (int col = quad; col < 2 * KB; col += NQ) {
                if (col < KB) {  // column c of L^{-1}: unit lower
                    const int c = col;
                    T *X = S + KB * LDS;  // X[r][c] = S[KB + r][c]
                    for (int r = 0; r < KB; ++r) {
                        T sum = T(0);
                        if (r > c)
                            for (int b = c + l4; b < r; b += 4) sum += S[r * LDS + b] * X[b * LDS + c];
                        sum += __shfl_xor_sync(qmask, sum, 1);
                        sum += __shfl_xor_sync(qmask, sum, 2);
                        if (l4 == 0) X[r * LDS + c] = (r < c) ? T(0) : (r == c) ? T(1) : -sum;
                        __syncwarp(qmask);
                    }
                } else {  // column c of U^{-1}: upper
                    const int c = col - KB;
                    T *Y = S + KB;  // Y[r][c] = S[r][KB + c]
                    for (int r = KB - 1; r >= 0; --r) {
                        T sum = T(0);
                        if (r < c)
                            for (int b = r + 1 + l4; b <= c; b += 4) sum += S[r * LDS + b] * Y[b * LDS + c];
                        sum += __shfl_xor_sync(qmask, sum, 1);
                        sum += __shfl_xor_sync(qmask, sum, 2);
                        if (l4 == 0) Y[r * LDS + c] = (r > c) ? T(0) : (r == c) ? dinv[c] : -sum * dinv[r];
                        __syncwarp(qmask);
                    }
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TT; e += NT) {
            const int r = e / KB, c = e % KB;
            F[0 * TT + e] = S[(KB + r) * LDS + c];  // L_JJ^{-1}
            F[2 * TT + e] = S[r * LDS + KB + c];    // U_JJ^{-1}
        }
        if (J + 1 == nb) break;
        __syncthreads();
        // next window: rows 0..KB-1 <- the Schur rows (columns J+1, J+2),
        // rows KB..2KB-1 <- block row J+2 of A_i; then every thread reloads
        // its row (one unconditional load keeps the registers free above)
        for (int e = threadIdx.x; e < KB * WC; e += NT) {
            const int r = e / WC, l = e % WC;
            S[r * LDS + l] = (l < 2 * KB) ? S[(KB + r) * LDS + KB + l] : T(0);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < KB * LDS; e += NT) S[KB * LDS + e] = T(0);
        if constexpr (G::PREFETCH) {
            cp_async_wait_all();
            __syncthreads();
            put_block_row<T, KB>(k, ni, J + 2, J + 1, S, KB, [&](int e, const BandRowMap &) { return Rb[e]; });
        } else {
            __syncthreads();
            put_block_row<T, KB>(k, ni, J + 2, J + 1, S, KB, from_band);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < CPT; ++q) a[q] = S[i * LDS + h * CPT + q];
    }
    if constexpr (G::PREFETCH) cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// solves: register-tiled KB x KB by KB x W products in shared memory
template <typename T> struct SolvePad { static constexpr int v = 16 / (int)sizeof(T); };

template <typename T, int KB, int W> struct PivS {
    static constexpr int NT = 4 * KB;
    static constexpr int LDF = KB + SolvePad<T>::v;  // factor tile stride
    static constexpr int LDW = W + SolvePad<T>::v;   // panel stride
    static constexpr int RC = W / 16;                // panel columns per thread
};

// Y (KB x W) = A X  or  Y - A1 X1 - A2 X2 (NTERM terms, SUB), A optionally transposed.
template <typename T, int KB, int W, bool TRA, int NTERM, bool SUB>
__device__ __forceinline__ void tprod(const T *A1, const T *X1, const T *A2, const T *X2, T *Y) {
    using G = PivS<T, KB, W>;
    constexpr int RC = G::RC, LDF = G::LDF, LDW = G::LDW;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const int r0 = ty * 4, c0 = tx * RC;
    T acc[4][RC];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < RC; ++v) acc[u][v] = T(0);
#pragma unroll
    for (int t = 0; t < NTERM; ++t) {
        const T *A = t ? A2 : A1;
        const T *X = t ? X2 : X1;
#pragma unroll 4
        for (int q = 0; q < KB; ++q) {
            T av[4], xv[RC];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = TRA ? A[q * LDF + r0 + u] : A[(r0 + u) * LDF + q];
#pragma unroll
            for (int v = 0; v < RC; ++v) xv[v] = X[q * LDW + c0 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < RC; ++v) acc[u][v] += av[u] * xv[v];
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < RC; ++v) {
            T *y = &Y[(r0 + u) * LDW + c0 + v];
            *y = SUB ? *y - acc[u][v] : acc[u][v];
        }
}

template <typename T, int KB, int W>
__device__ __forceinline__ void load_ftile(const T *__restrict__ g, T *S) {
    using G = PivS<T, KB, W>;
    for (int e = threadIdx.x; e < KB * KB; e += G::NT) S[(e / KB) * G::LDF + e % KB] = g[e];
}

template <typename T, int KB, int W>
__device__ __forceinline__ void zero_panel(T *S) {
    using G = PivS<T, KB, W>;
    for (int e = threadIdx.x; e < KB * G::LDW; e += G::NT) S[e] = T(0);
}

// Shared layout of the solve kernels: 3 factor tiles, 5 panels of KB x W, pi.
template <typename T, int KB, int W> struct PivSmem {
    using G = PivS<T, KB, W>;
    static constexpr size_t bytes =
        (3 * (size_t)KB * G::LDF + 5 * (size_t)KB * G::LDW) * sizeof(T) + 2 * KB * sizeof(int);
};

// A_i^{-1} applied to a KB-row-blocked right-hand side panel of W columns.
// IO provides in(J, panel) (fill rows of block J, zeros past the partition),
// put_fwd / get_fwd (the forward result of block J) and out(J, panel).
template <typename T, int KB, int W, typename IO>
__device__ void piv_solve(const T *__restrict__ PF, const unsigned char *__restrict__ PIV, int64_t b0, int nb,
                          unsigned char *smem_raw, IO &io) {
    using G = PivS<T, KB, W>;
    constexpr int NT = G::NT, LDF = G::LDF, LDW = G::LDW, TT = KB * KB;
    T *F0 = reinterpret_cast<T *>(smem_raw);
    T *F1 = F0 + KB * LDF;
    T *F2 = F1 + KB * LDF;
    T *P0 = F2 + KB * LDF;  // five panels
    T *P1 = P0 + KB * LDW;
    T *P2 = P1 + KB * LDW;
    T *P3 = P2 + KB * LDW;
    T *P4 = P3 + KB * LDW;
    int *pi = reinterpret_cast<int *>(P4 + KB * LDW);
    // forward: P0 holds block J, P1 block J+1; the gather writes [P2; P3];
    // y_J goes to P4; the updated P3 is block J+1's panel for the next step
    io.in(0, P0);
    for (int J = 0; J < nb; ++J) {
        const T *Fg = PF + (b0 + J) * 5 * TT;
        load_ftile<T, KB, W>(Fg + 0 * TT, F0);
        load_ftile<T, KB, W>(Fg + 1 * TT, F1);
        if (threadIdx.x < 2 * KB) pi[threadIdx.x] = PIV[(b0 + J) * 2 * KB + threadIdx.x];
        if (J + 1 < nb) io.in(J + 1, P1); else zero_panel<T, KB, W>(P1);
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * KB * W; e += NT) {
            const int r = e / W, c = e % W, src = pi[r];
            const T v = (src < KB) ? P0[src * LDW + c] : P1[(src - KB) * LDW + c];
            (r < KB ? P2 : P3)[(r % KB) * LDW + c] = v;
        }
        __syncthreads();
        tprod<T, KB, W, false, 1, false>(F0, P2, nullptr, nullptr, P4);  // y_J = L_JJ^{-1} top
        __syncthreads();
        io.put_fwd(J, P4);
        tprod<T, KB, W, false, 1, true>(F1, P4, nullptr, nullptr, P3);   // bottom -= L_{J+1,J} y_J
        __syncthreads();
        for (int e = threadIdx.x; e < KB * W; e += NT) P0[(e / W) * LDW + e % W] = P3[(e / W) * LDW + e % W];
        __syncthreads();
    }
    // backward: x_{J+1} in X1, x_{J+2} in X2
    T *X1 = P0, *X2 = P1, *Tt = P2, *X0 = P3;
    zero_panel<T, KB, W>(X1);
    zero_panel<T, KB, W>(X2);
    for (int J = nb - 1; J >= 0; --J) {
        const T *Fg = PF + (b0 + J) * 5 * TT;
        load_ftile<T, KB, W>(Fg + 2 * TT, F0);
        load_ftile<T, KB, W>(Fg + 3 * TT, F1);
        load_ftile<T, KB, W>(Fg + 4 * TT, F2);
        io.get_fwd(J, Tt);
        __syncthreads();
        tprod<T, KB, W, false, 2, true>(F1, X1, F2, X2, Tt);
        __syncthreads();
        tprod<T, KB, W, false, 1, false>(F0, Tt, nullptr, nullptr, X0);
        __syncthreads();
        io.out(J, X0);
        T *t = X2;
        X2 = X1;
        X1 = X0;
        X0 = t;
        __syncthreads();
    }
}

// transposed solve: A_i^{-T} = pi^T L^{-T} ... U^{-T} in the order of the
// factorisation: forward with U^T, backward with L^T, each backward step
// followed by the scatter [w_J; w_{J+1}] <- pi_J^T [w_J; w_{J+1}]
template <typename T, int KB, int W, typename IO>
__device__ void piv_solve_t(const T *__restrict__ PF, const unsigned char *__restrict__ PIV, int64_t b0, int nb,
                            unsigned char *smem_raw, IO &io) {
    using G = PivS<T, KB, W>;
    constexpr int NT = G::NT, LDF = G::LDF, LDW = G::LDW, TT = KB * KB;
    T *F0 = reinterpret_cast<T *>(smem_raw);
    T *F1 = F0 + KB * LDF;
    T *F2 = F1 + KB * LDF;
    T *P0 = F2 + KB * LDF;
    T *P1 = P0 + KB * LDW;
    T *P2 = P1 + KB * LDW;
    T *P3 = P2 + KB * LDW;
    T *P4 = P3 + KB * LDW;
    int *pi = reinterpret_cast<int *>(P4 + KB * LDW);
    // forward: z_J = U_JJ^{-T}(h_J - U_{J-1,J}^T z_{J-1} - U_{J-2,J}^T z_{J-2})
    T *Z1 = P0, *Z2 = P1, *Tt = P2, *Z0 = P3;
    for (int J = 0; J < nb; ++J) {
        load_ftile<T, KB, W>(PF + (b0 + J) * 5 * TT + 2 * TT, F0);
        if (J >= 1) load_ftile<T, KB, W>(PF + (b0 + J - 1) * 5 * TT + 3 * TT, F1);
        if (J >= 2) load_ftile<T, KB, W>(PF + (b0 + J - 2) * 5 * TT + 4 * TT, F2);
        io.in(J, Tt);
        __syncthreads();
        if (J >= 2) tprod<T, KB, W, true, 2, true>(F1, Z1, F2, Z2, Tt);
        else if (J == 1) tprod<T, KB, W, true, 1, true>(F1, Z1, nullptr, nullptr, Tt);
        __syncthreads();
        tprod<T, KB, W, true, 1, false>(F0, Tt, nullptr, nullptr, Z0);
        __syncthreads();
        io.put_fwd(J, Z0);
        T *t = Z2;
        Z2 = Z1;
        Z1 = Z0;
        Z0 = t;
        __syncthreads();
    }
    // backward: Wn holds w_{J+1} (not yet final: step J's scatter may change it)
    T *Wn = P0, *Tb = P1, *Wc = P2, *G0 = P3, *G1 = P4;
    zero_panel<T, KB, W>(Wn);
    for (int J = nb - 1; J >= 0; --J) {
        const T *Fg = PF + (b0 + J) * 5 * TT;
        load_ftile<T, KB, W>(Fg + 0 * TT, F0);
        load_ftile<T, KB, W>(Fg + 1 * TT, F1);
        if (threadIdx.x < 2 * KB) pi[threadIdx.x] = PIV[(b0 + J) * 2 * KB + threadIdx.x];
        io.get_fwd(J, Tb);
        __syncthreads();
        if (J + 1 < nb) tprod<T, KB, W, true, 1, true>(F1, Wn, nullptr, nullptr, Tb);
        __syncthreads();
        tprod<T, KB, W, true, 1, false>(F0, Tb, nullptr, nullptr, Wc);
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * KB * W; e += NT) {
            const int r = e / W, c = e % W, dst = pi[r];
            const T v = (r < KB) ? Wc[r * LDW + c] : Wn[(r - KB) * LDW + c];
            (dst < KB ? G0 : G1)[(dst % KB) * LDW + c] = v;
        }
        __syncthreads();
        if (J + 1 < nb) io.out(J + 1, G1);
        for (int e = threadIdx.x; e < KB * W; e += NT) Wn[(e / W) * LDW + e % W] = G0[(e / W) * LDW + e % W];
        __syncthreads();
    }
    io.out(0, Wn);
}

// Spike panels: X blocked [block][KB][m]; this CTA owns columns c0 .. c0+W-1.
template <typename T, int KB, int W> struct SpikeIO {
    T *X;
    int64_t b0;
    int m, c0;
    __device__ T *blk(int J) const { return X + (b0 + J) * (int64_t)KB * m + c0; }
    __device__ void in(int J, T *Pn) const {
        const T *g = blk(J);
        for (int e = threadIdx.x; e < KB * W; e += 4 * KB) Pn[(e / W) * PivS<T, KB, W>::LDW + e % W] = g[(e / W) * m + e % W];
    }
    __device__ void get_fwd(int J, T *Pn) const { in(J, Pn); }
    __device__ void put_fwd(int J, const T *Pn) const {
        T *g = blk(J);
        for (int e = threadIdx.x; e < KB * W; e += 4 * KB) g[(e / W) * m + e % W] = Pn[(e / W) * PivS<T, KB, W>::LDW + e % W];
    }
    __device__ void out(int J, const T *Pn) const { put_fwd(J, Pn); }
};

template <typename T, int KB, int W>
__global__ void __launch_bounds__(4 * KB)
    k_sweep_piv(const T *__restrict__ PF, const unsigned char *__restrict__ PIV, Parts P, T *__restrict__ X, int m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int part = blockIdx.x;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    SpikeIO<T, KB, W> io{X, b0, m, (int)blockIdx.y * W};
    piv_solve<T, KB, W>(PF, PIV, b0, nb, smem_raw, io);
}

// Vector panels of the D-stages: column c of the panel is right-hand side c
// (c < nrhs), rows a of block J are local rows J*KB + a; consecutive threads
// take consecutive rows (coalesced).
constexpr int VW16 = 16;

template <typename T, int KB> struct VecPanel {
    static constexpr int LDW = PivS<T, KB, VW16>::LDW;
    int64_t n, s, ni;
    int nrhs;
    template <typename F> __device__ void each(int J, F &&f) const {
        for (int e = threadIdx.x; e < KB * VW16; e += 4 * KB) {
            const int a = e % KB, c = e / KB;
            const int64_t row = (int64_t)J * KB + a;
            f(a, c, row, row < ni && c < nrhs);
        }
    }
};

template <typename T, int KB> struct DstageIO {
    VecPanel<T, KB> vp;
    const double *rin, *inv;
    T *Yv, *Gv;
    __device__ void in(int J, T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            Pn[a * vp.LDW + c] = ok ? (T)(rin[c * vp.n + vp.s + row] * inv[c]) : T(0);
        });
    }
    __device__ void put_fwd(int J, const T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            if (ok) Yv[c * vp.n + vp.s + row] = Pn[a * vp.LDW + c];
        });
    }
    __device__ void get_fwd(int J, T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            Pn[a * vp.LDW + c] = ok ? Yv[c * vp.n + vp.s + row] : T(0);
        });
    }
    __device__ void out(int J, const T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            if (ok) Gv[c * vp.n + vp.s + row] = Pn[a * vp.LDW + c];
        });
    }
};

template <typename T, int KB>
__global__ void __launch_bounds__(4 * KB)
    k_dstage_piv(const T *__restrict__ PF, const unsigned char *__restrict__ PIV, const T *__restrict__ PQ, Parts P,
                 int k, int r, int64_t n, const double *__restrict__ rin, const double *__restrict__ inv, int nrhs,
                 T *__restrict__ Yv, T *__restrict__ Gv, double *__restrict__ psi, const int *skip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (skip && *skip) return;  // graph-safe refinement already met tol
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    DstageIO<T, KB> io{{n, s, ni, nrhs}, rin, inv, Yv, Gv};
    piv_solve<T, KB, VW16>(PF, PIV, b0, nb, smem_raw, io);
    if (r == 0) return;
    __syncthreads();  // g of this partition is complete (written by this CTA)
    // psi_{part-1}[0:r] = P_{part-1} g_t ;  psi_part[r:2r] = Q_{part+1} g_b
    const int n2 = 2 * r;
    for (int o = threadIdx.x; o < 2 * r * nrhs; o += 4 * KB) {
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

template <typename T, int KB> struct DstageTIO {
    VecPanel<T, KB> vp;
    const double *hin, *inv, *nrm;
    const T *corr;  // [2][KB][16]: top and bottom tip corrections V^T w
    int k;
    T *Yv;
    double *x;
    int64_t ldx;
    int accumulate;
    __device__ void in(int J, T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            T v = T(0);
            if (ok) {
                v = (T)(hin[c * vp.n + vp.s + row] * inv[c]);
                if (row < k) v -= corr[row * VW16 + c];
                if (row >= vp.ni - k) v -= corr[KB * VW16 + (row - (vp.ni - k)) * VW16 + c];
            }
            Pn[a * vp.LDW + c] = v;
        });
    }
    __device__ void put_fwd(int J, const T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            if (ok) Yv[c * vp.n + vp.s + row] = Pn[a * vp.LDW + c];
        });
    }
    __device__ void get_fwd(int J, T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            Pn[a * vp.LDW + c] = ok ? Yv[c * vp.n + vp.s + row] : T(0);
        });
    }
    __device__ void out(int J, const T *Pn) const {
        vp.each(J, [&](int a, int c, int64_t row, bool ok) {
            if (!ok) return;
            const double upd = nrm[c] * (double)Pn[a * vp.LDW + c];
            const int64_t xi = c * ldx + vp.s + row;
            x[xi] = accumulate ? x[xi] + upd : upd;
        });
    }
};

template <typename T, int KB>
__global__ void __launch_bounds__(4 * KB)
    k_dstage_t_piv(const T *__restrict__ PF, const unsigned char *__restrict__ PIV, const T *__restrict__ PQ,
                   Parts P, int k, int r, int64_t n, const double *__restrict__ hin, const double *__restrict__ inv,
                   const double *__restrict__ zr, int nrhs, T *__restrict__ Yv, const double *__restrict__ nrm,
                   double *__restrict__ x, int64_t ldx, int accumulate, const int *skip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (skip && *skip) return;
    T *corr = reinterpret_cast<T *>(smem_raw + PivSmem<T, KB, VW16>::bytes);
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int n2 = 2 * r;
    // y = h - V^T w at the tips: top rows P_{part-1}^T w_zeta, bottom rows Q_{part+1}^T w_omega
    for (int e = threadIdx.x; e < 2 * KB * VW16; e += 4 * KB) {
        const int side = e / (KB * VW16), rem = e % (KB * VW16), q = rem / VW16, c = rem % VW16;
        double acc = 0.0;
        if (q < k && r > 0 && c < nrhs) {
            if (side == 0 && part >= 1) {
                const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * KB;
                for (int j = 0; j < r; ++j) acc += (double)Pm[j * KB + q] * zr[((int64_t)(part - 1) * n2 + j) * nrhs + c];
            } else if (side == 1 && part <= P.p - 2) {
                const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * KB;
                for (int j = 0; j < r; ++j) acc += (double)Qm[j * KB + q] * zr[((int64_t)part * n2 + r + j) * nrhs + c];
            }
        }
        corr[e] = (T)acc;
    }
    __syncthreads();
    DstageTIO<T, KB> io{{n, s, ni, nrhs}, hin, inv, nrm, corr, k, Yv, x, ldx, accumulate};
    piv_solve_t<T, KB, VW16>(PF, PIV, b0, nb, smem_raw, io);
}

// ---- launchers --------------------------------------------------------------
template <typename T, int KB>
bool lu_piv_impl(Ctx *c) {
    using G = PivLU<T, KB>;
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = G::smem_bytes;
    auto kern = k_band_lu_piv<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_LU, [&] {
        kern<<<c->p, G::NT, smem, c->stream>>>(c->band, c->ld, c->k, P, (T *)c->PF, c->PIVP, c->status);
    });
}

template <typename T, int KB, int W>
bool sweep_piv_w(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = PivSmem<T, KB, W>::bytes;
    auto kern = k_sweep_piv<T, KB, W>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(c->p, c->m / W);
    return launch(c, KID_SWEEP, [&] {
        kern<<<grid, 4 * KB, smem, c->stream>>>((const T *)c->PF, c->PIVP, P, (T *)c->X, c->m);
    });
}

template <typename T, int KB>
bool sweep_piv_impl(Ctx *c) {
    constexpr int WMAX = sizeof(T) == 4 ? 64 : 32;
    const int w = c->m < WMAX ? c->m : WMAX;  // m is a multiple of 16
    if (w == 16) return sweep_piv_w<T, KB, 16>(c);
    if (w == 32) return sweep_piv_w<T, KB, 32>(c);
    return sweep_piv_w<T, KB, WMAX>(c);
}

template <typename T, int KB>
bool dstage_piv_impl(Ctx *c, const double *rin, int nrhs) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = PivSmem<T, KB, VW16>::bytes;
    auto kern = k_dstage_piv<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_DSTAGE, [&] {
        kern<<<c->p, 4 * KB, smem, c->stream>>>((const T *)c->PF, c->PIVP, (const T *)c->PQ, P, c->k, c->r, c->n,
                                               rin, c->nrm + 2 * c->opt.max_nrhs, nrhs, (T *)c->Yv, (T *)c->Gv,
                                               c->psi, c->skip);
    });
}

template <typename T, int KB>
bool dstage_t_piv_impl(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, int acc) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = PivSmem<T, KB, VW16>::bytes + 2 * KB * VW16 * sizeof(T);
    auto kern = k_dstage_t_piv<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_DSTAGE_T, [&] {
        kern<<<c->p, 4 * KB, smem, c->stream>>>((const T *)c->PF, c->PIVP, (const T *)c->PQ, P, c->k, c->r, c->n,
                                               hin, c->nrm + 2 * c->opt.max_nrhs, c->zr, nrhs, (T *)c->Yv,
                                               c->nrm + c->opt.max_nrhs, x, ldx, acc, c->skip);
    });
}

template <typename T>
bool lu_piv_t(Ctx *c) {
    switch (c->KB) {
        case 8: return lu_piv_impl<T, 8>(c);
        case 16: return lu_piv_impl<T, 16>(c);
        case 32: return lu_piv_impl<T, 32>(c);
        default: return lu_piv_impl<T, 64>(c);
    }
}
template <typename T>
bool sweep_piv_t(Ctx *c) {
    switch (c->KB) {
        case 8: return sweep_piv_impl<T, 8>(c);
        case 16: return sweep_piv_impl<T, 16>(c);
        case 32: return sweep_piv_impl<T, 32>(c);
        default: return sweep_piv_impl<T, 64>(c);
    }
}
template <typename T>
bool dstage_piv_t(Ctx *c, const double *rin, int nrhs) {
    switch (c->KB) {
        case 8: return dstage_piv_impl<T, 8>(c, rin, nrhs);
        case 16: return dstage_piv_impl<T, 16>(c, rin, nrhs);
        case 32: return dstage_piv_impl<T, 32>(c, rin, nrhs);
        default: return dstage_piv_impl<T, 64>(c, rin, nrhs);
    }
}
template <typename T>
bool dstage_t_piv_t(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, int acc) {
    switch (c->KB) {
        case 8: return dstage_t_piv_impl<T, 8>(c, hin, x, ldx, nrhs, acc);
        case 16: return dstage_t_piv_impl<T, 16>(c, hin, x, ldx, nrhs, acc);
        case 32: return dstage_t_piv_impl<T, 32>(c, hin, x, ldx, nrhs, acc);
        default: return dstage_t_piv_impl<T, 64>(c, hin, x, ldx, nrhs, acc);
    }
}

}  // namespace

bool run_band_lu_piv(Ctx *c) { return c->fp64 ? lu_piv_t<double>(c) : lu_piv_t<float>(c); }
bool run_sweep_piv(Ctx *c) { return c->fp64 ? sweep_piv_t<double>(c) : sweep_piv_t<float>(c); }
bool run_dstage_piv(Ctx *c, const double *rin, int nrhs) {
    return c->fp64 ? dstage_piv_t<double>(c, rin, nrhs) : dstage_piv_t<float>(c, rin, nrhs);
}
bool run_dstage_t_piv(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, bool accumulate) {
    const int acc = accumulate ? 1 : 0;
    return c->fp64 ? dstage_t_piv_t<double>(c, hin, x, ldx, nrhs, acc) : dstage_t_piv_t<float>(c, hin, x, ldx, nrhs, acc);
}

}  // namespace lrs
