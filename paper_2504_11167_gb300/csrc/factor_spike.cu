// Spikes and their rank-r compression (paper section 2.1, eq. 'Veqn';
// section 3.1).
//
//   k_spike_rhs   right-hand sides [0; B_i] and [C_i; 0] (SPIKE mode) or
//                 [0; B_i V_B] and [C_i V_C; 0] (COUPLING mode) in the spike
//                 buffer X, one KB x m panel per block
//   k_sweep       X <- A_i^{-1} X per partition: forward then backward chain
//                 over the packed factor tiles (m = 2KB or 2r columns)
//   k_gram        partial Gram matrices T_i^T T_i and W_i^T W_i per chunk
//   k_gram_reduce fixed-order sum of the chunk partials (deterministic)
//   k_coupling_gram  B_i^T B_i and C_i^T C_i straight from the band
//   k_jacobi      cyclic two-sided Jacobi eigensolver (round-robin ordering,
//                 KB/2 disjoint rotations at a time) of each Gram matrix; the
//                 r leading eigenvectors V_r give the truncated SVD subspace
//   k_make_u      u-factors of the low-rank spikes
//
// Compression identity used here: for a spike X with SVD U S V^T, the best
// rank-r approximation is X V_r V_r^T, so the low-rank spike is stored as
// u = X V_r (n_i x r, columns orthogonal with norms sigma_j) and P = V_r^T
// (r x k).  V_r comes from the eigenvectors of X^T X.  COUPLING mode
// (section 3.1's alternative) truncates B_i = U_B S_B V_B^T instead:
// T~_i = A_i^{-1}[0; B_i V_B,r] V_B,r^T, so u is the solve of r columns.
// The rank guard drops sigma_j <= rank_tol * sigma_1 (the paper lowers n_svd
// when singular values approach zero, section 4.2).
#include "common.cuh"
#include "internal.h"
#include "tile_ops.cuh"

namespace lrs {

// ---------------------------------------------------------------------------
template <typename T, int KB>
__global__ void k_spike_rhs(const double *__restrict__ band, int64_t ld, int k, Parts P, int r,
                            int coupling, const T *__restrict__ PQ, T *__restrict__ X, int m) {
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    // local row rho -> X[(b0 + rho / KB) * KB * m + (rho % KB) * m + col]
    auto xat = [&](int64_t rho, int col) -> T & {
        return X[(b0 + rho / KB) * (int64_t)KB * m + (rho % KB) * m + col];
    };
    if (part < P.p - 1) {  // right spike: rows ni-k..ni-1 hold B_i
        const int64_t sn = s + ni;
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int a = e / k, b = e % k;
            if (!coupling) {
                // B_i[a][b] = A[sn-k+a][sn+b], nonzero for b <= a
                xat(ni - k + a, b) = (b <= a) ? (T)band[(int64_t)(a - b) * ld + sn + b] : T(0);
            }
        }
        if (coupling) {
            for (int e = threadIdx.x; e < k * r; e += blockDim.x) {
                const int a = e / r, c = e % r;
                double acc = 0.0;
                for (int b = 0; b <= a; ++b)
                    acc += band[(int64_t)(a - b) * ld + sn + b] *
                           (double)PQ[(((int64_t)part * 2 + 0) * r + c) * KB + b];
                xat(ni - k + a, c) = (T)acc;
            }
        }
    }
    if (part > 0) {  // left spike: rows 0..k-1 hold C_i
        const int wc = m / 2;  // first column of the W panel
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int a = e / k, b = e % k;
            if (!coupling) {
                // C_i[a][b] = A[s+a][s-k+b], nonzero for a <= b
                xat(a, wc + b) =
                    (a <= b) ? (T)band[(int64_t)(2 * k + a - b) * ld + s - k + b] : T(0);
            }
        }
        if (coupling) {
            for (int e = threadIdx.x; e < k * r; e += blockDim.x) {
                const int a = e / r, c = e % r;
                double acc = 0.0;
                for (int b = a; b < k; ++b)
                    acc += band[(int64_t)(2 * k + a - b) * ld + s - k + b] *
                           (double)PQ[(((int64_t)part * 2 + 1) * r + c) * KB + b];
                xat(a, wc + c) = (T)acc;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// X <- A_i^{-1} X for the spike panel of every partition (one CTA each).
// Panel columns [0, M/2) hold the right spike T_i, [M/2, M) the left spike W_i.
// The right spike's right-hand side is zero above block Jv0 = (n_i - k)/KB, so
// its forward chain starts there; partition 0 has no W_i and partition p-1 no
// T_i, so those halves are skipped entirely.  The packed factor tile of each
// step is unpacked into two triangular tiles with explicit zeros and the unit
// diagonal, so the register-tiled products need no masks.
template <typename T, int KB, int MT, int CG>
__global__ void __launch_bounds__((KB / 4) * CG, (KB >= 64 && sizeof(T) == 4) ? 2 : 1)
    k_sweep(const T *__restrict__ LT, const T *__restrict__ UT, const T *__restrict__ DI, Parts P, int k,
            T *__restrict__ X) {
    // MT columns per thread, CG column groups: panel width M = MT * CG
    constexpr int NT = (KB / 4) * CG, M = MT * CG, LDA = KB + 1, HALFM = M / 2;
    constexpr int LDM = M + 16 / (int)sizeof(T);  // padded panel rows in shared memory
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *A1 = reinterpret_cast<T *>(smem_raw);  // off-diagonal factor block
    T *A2 = A1 + KB * LDA;                    // inverse of the diagonal factor
    T *Tt = A2 + KB * LDA;                    // KB x LDM
    T *Yp = Tt + KB * LDM;                    // KB x LDM
    T *dsm = Yp + KB * LDM;                   // KB
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const bool hasV = part < P.p - 1, hasW = part > 0;
    const int Jv0 = (int)((ni - k) / KB);
    int ty, tx;
    PanelMap<KB, CG>::get(threadIdx.x, ty, tx);
    const int a0 = 4 * ty, c0 = MT * tx;
    const bool isV = c0 < HALFM;
    T acc[4][MT];

    // L2 prefetch of the next block step's factor tile and panel
    auto prefetch = [&](const T *tile, const T *panel) {
        constexpr int TL = KB * KB * (int)sizeof(T) / 128, PL = KB * M * (int)sizeof(T) / 128;
        for (int e = threadIdx.x; e < TL + PL; e += NT) {
            const char *pa = (e < TL) ? (const char *)tile + e * 128 : (const char *)panel + (e - TL) * 128;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
        }
    };
    for (int J = 0; J < nb; ++J) {
        const int64_t g = b0 + J;
        const T *tile = LT + g * KB * KB;
        if (J + 1 < nb) prefetch(LT + (g + 1) * KB * KB, X + (g + 1) * KB * M);
        for (int e = threadIdx.x; e < KB * KB; e += NT) {
            const int a = e / KB, b = e % KB;
            const T v = tile[e];
            A1[a * LDA + b] = (a <= b) ? v : T(0);                        // L_{J,J-1}
            A2[a * LDA + b] = (a > b) ? v : ((a == b) ? T(1) : T(0));     // L_JJ^{-1}
        }
        const bool active = isV ? (hasV && J >= Jv0) : hasW;
        const bool first = (J == 0) || (isV && J == Jv0);
        T *xg = X + g * KB * M;
        if (active)
#pragma unroll
            for (int i = 0; i < 4; ++i) ld_row<T, MT>(xg + (a0 + i) * M + c0, acc[i]);
        __syncthreads();
        if (active) {
            if (!first) panel_mac<T, MT, true>(acc, A1, LDA, Yp, LDM, a0, c0, a0, KB);
#pragma unroll
            for (int i = 0; i < 4; ++i) st_row<T, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] = T(0);
            panel_mac<T, MT, false>(acc, A2, LDA, Tt, LDM, a0, c0, 0, a0 + 4);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                st_row<T, MT>(Yp + (a0 + i) * LDM + c0, acc[i]);
                st_row<T, MT>(xg + (a0 + i) * M + c0, acc[i]);
            }
        }
        __syncthreads();
    }
    for (int J = nb - 1; J >= 0; --J) {
        const int64_t g = b0 + J;
        const T *tile = UT + g * KB * KB;
        if (J > 0) prefetch(UT + (g - 1) * KB * KB, X + (g - 1) * KB * M);
        for (int e = threadIdx.x; e < KB * KB; e += NT) {
            const int a = e / KB, b = e % KB;
            const T v = tile[e];
            A1[a * LDA + b] = (a >= b) ? v : T(0);                        // D^{-1} U_{J,J+1}
            A2[a * LDA + b] = (a < b) ? v : ((a == b) ? T(1) : T(0));     // (D^{-1} U_JJ)^{-1}
        }
        if (threadIdx.x < KB) dsm[threadIdx.x] = DI[g * KB + threadIdx.x];
        const bool active = isV ? hasV : hasW;
        T *xg = X + g * KB * M;
        if (active)
#pragma unroll
            for (int i = 0; i < 4; ++i) ld_row<T, MT>(xg + (a0 + i) * M + c0, acc[i]);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] *= dsm[a0 + i];
            if (J < nb - 1) panel_mac<T, MT, true>(acc, A1, LDA, Yp, LDM, a0, c0, 0, a0 + 4);
#pragma unroll
            for (int i = 0; i < 4; ++i) st_row<T, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] = T(0);
            panel_mac<T, MT, false>(acc, A2, LDA, Tt, LDM, a0, c0, a0, KB);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                st_row<T, MT>(Yp + (a0 + i) * LDM + c0, acc[i]);
                st_row<T, MT>(xg + (a0 + i) * M + c0, acc[i]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The same sweep, pipelined, for FP32 panels whose staging ring fits two CTAs
// per SM (the COUPLING mode's 2r columns).  Per block step the raw factor tile,
// the panel block and D^{-1} are staged with cp.async two steps ahead into a
// ring of three buffers.  The triangular products read the raw tile and mask
// only the thread's 4-row diagonal chunk (compile-time masks: row a0+i,
// column a0+u).  Two barriers per step: the loop-top barrier publishes the
// staged step and closes the previous one.  The backward sweep's first block
// (J = nb-1) takes its input from Yp, the forward output that is still in
// shared memory; every other backward input was written to X at least one
// step (and a barrier) before its staging.
template <typename T, int KB, int MT, int CG> struct SweepPipe {
    static constexpr int NT = (KB / 4) * CG, M = MT * CG, NBUF = 3, PDS = 2;
    static constexpr int LDT = KB + 16 / (int)sizeof(T), LDM = M + 16 / (int)sizeof(T);
    static constexpr size_t bytes =
        ((size_t)NBUF * (KB * LDT + KB * LDM + KB) + (size_t)2 * KB * LDM) * sizeof(T);
};

template <typename T, int KB, int MT, int CG>
__global__ void __launch_bounds__((KB / 4) * CG)
    k_sweep_pipe(const T *__restrict__ LT, const T *__restrict__ UT, const T *__restrict__ DI, Parts P, int k,
                 T *__restrict__ X) {
    using SP = SweepPipe<T, KB, MT, CG>;
    constexpr int NT = SP::NT, M = SP::M, HALFM = M / 2, NBUF = SP::NBUF, PDS = SP::PDS;
    constexpr int LDT = SP::LDT, LDM = SP::LDM, CH = 16 / (int)sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tiles = reinterpret_cast<T *>(smem_raw);  // [NBUF][KB x LDT] raw factor tiles
    T *pans = tiles + NBUF * KB * LDT;           // [NBUF][KB x LDM] panel blocks
    T *dis = pans + NBUF * KB * LDM;             // [NBUF][KB] D^{-1}
    T *Tt = dis + NBUF * KB;                     // KB x LDM
    T *Yp = Tt + KB * LDM;                       // KB x LDM
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0), steps = 2 * nb;
    const bool hasV = part < P.p - 1, hasW = part > 0;
    const int Jv0 = (int)((ni - k) / KB);
    int ty, tx;
    PanelMap<KB, CG>::get(threadIdx.x, ty, tx);
    const int a0 = 4 * ty, c0 = MT * tx;
    const bool isV = c0 < HALFM;

    auto stage = [&](int t) {
        const int buf = t % NBUF;
        const bool fwd = t < nb;
        const int J = fwd ? t : steps - 1 - t;
        const int64_t g = b0 + J;
        const T *tsrc = (fwd ? LT : UT) + g * KB * KB;
        T *tdst = tiles + buf * KB * LDT;
        for (int e = threadIdx.x; e < KB * (KB / CH); e += NT) {
            const int row = e / (KB / CH), ch = e % (KB / CH);
            cp_async16(tdst + row * LDT + ch * CH, tsrc + row * KB + ch * CH);
        }
        if (fwd || J < nb - 1) {
            const T *psrc = X + g * KB * M;
            T *pdst = pans + buf * KB * LDM;
            for (int e = threadIdx.x; e < KB * (M / CH); e += NT) {
                const int row = e / (M / CH), ch = e % (M / CH);
                cp_async16(pdst + row * LDM + ch * CH, psrc + row * M + ch * CH);
            }
        }
        if (!fwd && threadIdx.x < KB / CH) cp_async16(dis + buf * KB + threadIdx.x * CH, DI + g * KB + threadIdx.x * CH);
    };
    // acc (+/-)= tile rows a0..a0+3 x B over q in [a0, a0+4), masked per (row, column)
    auto chunk = [&](T (&acc)[4][MT], const T *tile, const T *B, int mode, bool sub) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            T bv[MT];
            ld_row<T, MT>(B + (a0 + u) * LDM + c0, bv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                // column a0+u against row a0+i: 0: q >= a, 1: q < a, 2: q <= a, 3: q > a
                const bool in = mode == 0 ? u >= i : mode == 1 ? u < i : mode == 2 ? u <= i : u > i;
                if (!in) continue;
                const T av = tile[(a0 + i) * LDT + a0 + u];
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] = sub ? acc[i][j] - av * bv[j] : acc[i][j] + av * bv[j];
            }
        }
    };

    // acc (+/-)= tile rows a0..a0+3 x B over q in [q0, q1) (multiples of 4):
    // four inner indices per 16-byte load of each tile row
    auto mac4 = [&](T (&acc)[4][MT], const T *tile, const T *B, int q0, int q1, bool sub) {
        for (int q = q0; q < q1; q += 4) {
            T av[4][4], bv[4][MT];
#pragma unroll
            for (int i = 0; i < 4; ++i) ld_row<T, 4>(tile + (a0 + i) * LDT + q, av[i]);
#pragma unroll
            for (int u = 0; u < 4; ++u) ld_row<T, MT>(B + (q + u) * LDM + c0, bv[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < MT; ++j)
                        acc[i][j] = sub ? acc[i][j] - av[i][u] * bv[u][j] : acc[i][j] + av[i][u] * bv[u][j];
        }
    };
    for (int t = 0; t < PDS; ++t) {
        if (t < steps) stage(t);
        cp_async_commit();
    }
    T acc[4][MT];
    for (int t = 0; t < steps; ++t) {
        cp_async_wait<PDS - 1>();
        __syncthreads();
        // buffer (t + PDS) % NBUF last served step t-1, closed by the barrier above
        if (t + PDS < steps) stage(t + PDS);
        cp_async_commit();
        const int buf = t % NBUF;
        const T *tile = tiles + buf * KB * LDT, *pan = pans + buf * KB * LDM;
        if (t < nb) {
            const int J = t;
            const bool active = isV ? (hasV && J >= Jv0) : hasW;
            const bool first = (J == 0) || (isV && J == Jv0);
            if (active) {
                // t = b_J - L_{J,J-1} y_{J-1}   (L_{J,J-1} upper incl. diagonal: q >= a)
#pragma unroll
                for (int i = 0; i < 4; ++i) ld_row<T, MT>(pan + (a0 + i) * LDM + c0, acc[i]);
                if (!first) {
                    chunk(acc, tile, Yp, 0, true);
                    mac4(acc, tile, Yp, a0 + 4, KB, true);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) st_row<T, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
            }
            __syncthreads();
            if (active) {
                // y_J = t + (L_JJ^{-1} strictly lower) t
#pragma unroll
                for (int i = 0; i < 4; ++i) ld_row<T, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
                mac4(acc, tile, Tt, 0, a0, false);
                chunk(acc, tile, Tt, 1, false);
                T *xg = X + (b0 + J) * KB * M;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    st_row<T, MT>(Yp + (a0 + i) * LDM + c0, acc[i]);
                    st_row<T, MT>(xg + (a0 + i) * M + c0, acc[i]);
                }
            }
        } else {
            const int J = steps - 1 - t;
            const bool active = isV ? hasV : hasW;
            const T *dsm = dis + buf * KB;
            if (active) {
                // t = D^{-1} y_J - (D^{-1}U_{J,J+1}) x_{J+1}   (lower incl. diagonal: q <= a)
                const T *src = (J == nb - 1) ? Yp : pan;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ld_row<T, MT>(src + (a0 + i) * LDM + c0, acc[i]);
#pragma unroll
                    for (int j = 0; j < MT; ++j) acc[i][j] *= dsm[a0 + i];
                }
                if (J < nb - 1) {
                    mac4(acc, tile, Yp, 0, a0, true);
                    chunk(acc, tile, Yp, 2, true);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) st_row<T, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
            }
            __syncthreads();
            if (active) {
                // x_J = t + ((D^{-1}U_JJ)^{-1} strictly upper) t
#pragma unroll
                for (int i = 0; i < 4; ++i) ld_row<T, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
                chunk(acc, tile, Tt, 3, false);
                mac4(acc, tile, Tt, a0 + 4, KB, false);
                T *xg = X + (b0 + J) * KB * M;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    st_row<T, MT>(Yp + (a0 + i) * LDM + c0, acc[i]);
                    st_row<T, MT>(xg + (a0 + i) * M + c0, acc[i]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The pipelined sweep for FP32, KB = 64 and 32 MT panel columns with a balanced
// thread map.  In k_sweep_pipe a thread owns one group of four rows, and the two
// triangular products of a block step cost row group g about 15 - g and g
// four-column chunks: the barrier between them makes every step pay the
// longest of each.  Here thread (pair, column) owns the row groups pair and
// 15 - pair (pair = 0..7) and MT columns, so both products cost every thread
// about 15 chunks.  A warp covers two pairs and the 16 column groups of one
// half of the panel (T_i or W_i columns: a whole warp skips an inactive half);
// the two tile rows a quarter-warp reads are 4 apart (68 floats: 16 mod 32
// words), so the 16-byte tile loads are conflict-free.  Staging, ring and
// barriers as in k_sweep_pipe.  The backward sweep's results are the
// COUPLING-mode u-factors themselves: they go straight to Ucat (row
// [u_T | u_W], panel column c -> c for c < r, r + c - M/2 for the W half;
// zeros where a partition has no such spike), not back to the panel.
template <int MT> struct SweepBal {
    static constexpr int KB = 64, NT = 256, M = 32 * MT, NBUF = 3, PDS = 2;
    static constexpr int LDT = KB + 4, LDM = M + 4;
    static constexpr size_t bytes =
        ((size_t)NBUF * (KB * LDT + KB * LDM + KB) + (size_t)2 * KB * LDM) * sizeof(float);
};

template <int MT>
__global__ void __launch_bounds__(256)
    k_sweep_bal(const float *__restrict__ LT, const float *__restrict__ UT, const float *__restrict__ DI, Parts P,
                int k, float *__restrict__ X, int r, float *__restrict__ Ucat) {
    using SB = SweepBal<MT>;
    constexpr int KB = SB::KB, NT = SB::NT, M = SB::M, NBUF = SB::NBUF, PDS = SB::PDS;
    constexpr int LDT = SB::LDT, LDM = SB::LDM, CH = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);  // [NBUF][KB x LDT] raw factor tiles
    float *pans = tiles + NBUF * KB * LDT;               // [NBUF][KB x LDM] panel blocks
    float *dis = pans + NBUF * KB * LDM;                 // [NBUF][KB] D^{-1}
    float *Tt = dis + NBUF * KB;                         // KB x LDM
    float *Yp = Tt + KB * LDM;                           // KB x LDM
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0), steps = 2 * nb;
    const bool hasV = part < P.p - 1, hasW = part > 0;
    const int Jv0 = (int)((ni - k) / KB);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const bool isV = (w >> 2) == 0;
    const int pair = (w & 3) * 2 + (l & 1);
    const int c0 = MT * ((w >> 2) * 16 + (l >> 1));
    const int ga[2] = {4 * pair, 4 * (15 - pair)};  // first rows of the two row groups
    const int n2 = 2 * r;
    // Ucat column of panel column c0 + j (-1: padding column)
    int ucol[MT];
#pragma unroll
    for (int j = 0; j < MT; ++j) {
        const int c = c0 + j, half = M / 2;
        ucol[j] = (c < half) ? (c < r ? c : -1) : (c - half < r ? r + c - half : -1);
    }

    auto stage = [&](int t) {
        const int buf = t % NBUF;
        const bool fwd = t < nb;
        const int J = fwd ? t : steps - 1 - t;
        const int64_t g = b0 + J;
        const float *tsrc = (fwd ? LT : UT) + g * KB * KB;
        float *tdst = tiles + buf * KB * LDT;
#pragma unroll
        for (int i = 0; i < KB * (KB / CH) / NT; ++i) {
            const int e = threadIdx.x + i * NT, row = e / (KB / CH), ch = e % (KB / CH);
            cp_async16(tdst + row * LDT + ch * CH, tsrc + row * KB + ch * CH);
        }
        if (fwd || J < nb - 1) {
            const float *psrc = X + g * KB * M;
            float *pdst = pans + buf * KB * LDM;
#pragma unroll
            for (int i = 0; i < KB * (M / CH) / NT; ++i) {
                const int e = threadIdx.x + i * NT, row = e / (M / CH), ch = e % (M / CH);
                cp_async16(pdst + row * LDM + ch * CH, psrc + row * M + ch * CH);
            }
        }
        if (!fwd && threadIdx.x < KB / CH) cp_async16(dis + buf * KB + threadIdx.x * CH, DI + g * KB + threadIdx.x * CH);
    };
    // acc (+/-)= tile rows a0..a0+3 x B over q in [a0, a0+4), masked per (row, column)
    auto chunk = [&](float (&acc)[4][MT], const float *tile, const float *B, int a0, int mode, bool sub) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float bv[MT];
            ld_row<float, MT>(B + (a0 + u) * LDM + c0, bv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                // column a0+u against row a0+i: 0: q >= a, 1: q < a, 2: q <= a, 3: q > a
                const bool in = mode == 0 ? u >= i : mode == 1 ? u < i : mode == 2 ? u <= i : u > i;
                if (!in) continue;
                const float av = tile[(a0 + i) * LDT + a0 + u];
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] = sub ? acc[i][j] - av * bv[j] : acc[i][j] + av * bv[j];
            }
        }
    };
    // acc (+/-)= tile rows a0..a0+3 x B over q in [q0, q1) (multiples of 4).
    // One column per thread: the products of even and odd q go to the two
    // halves of a packed FP32 FMA (__ffma2_rn), whose sum then updates acc.
    auto mac4 = [&](float (&acc)[4][MT], const float *tile, const float *B, int a0, int q0, int q1, bool sub) {
        if constexpr (MT == 1) {
            float2 s2[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) s2[i] = make_float2(0.f, 0.f);
            for (int q = q0; q < q1; q += 4) {
                float av[4][4], bq[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) ld_row<float, 4>(tile + (a0 + i) * LDT + q, av[i]);
#pragma unroll
                for (int u = 0; u < 4; ++u) bq[u] = B[(q + u) * LDM + c0];
                const float2 b01 = make_float2(bq[0], bq[1]), b23 = make_float2(bq[2], bq[3]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    s2[i] = __ffma2_rn(make_float2(av[i][0], av[i][1]), b01, s2[i]);
                    s2[i] = __ffma2_rn(make_float2(av[i][2], av[i][3]), b23, s2[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float t = s2[i].x + s2[i].y;
                acc[i][0] = sub ? acc[i][0] - t : acc[i][0] + t;
            }
            return;
        }
        for (int q = q0; q < q1; q += 4) {
            float av[4][4], bv[4][MT];
#pragma unroll
            for (int i = 0; i < 4; ++i) ld_row<float, 4>(tile + (a0 + i) * LDT + q, av[i]);
#pragma unroll
            for (int u = 0; u < 4; ++u) ld_row<float, MT>(B + (q + u) * LDM + c0, bv[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < MT; ++j)
                        acc[i][j] = sub ? acc[i][j] - av[i][u] * bv[u][j] : acc[i][j] + av[i][u] * bv[u][j];
        }
    };
    for (int t = 0; t < PDS; ++t) {
        if (t < steps) stage(t);
        cp_async_commit();
    }
    float acc[4][MT];
    for (int t = 0; t < steps; ++t) {
        cp_async_wait<PDS - 1>();
        __syncthreads();
        // buffer (t + PDS) % NBUF last served step t-1, closed by the barrier above
        if (t + PDS < steps) stage(t + PDS);
        cp_async_commit();
        const int buf = t % NBUF;
        const float *tile = tiles + buf * KB * LDT, *pan = pans + buf * KB * LDM;
        if (t < nb) {
            const int J = t;
            const bool active = isV ? (hasV && J >= Jv0) : hasW;
            const bool first = (J == 0) || (isV && J == Jv0);
            if (active) {
                // t = b_J - L_{J,J-1} y_{J-1}   (L_{J,J-1} upper incl. diagonal: q >= a)
#pragma unroll
                for (int G = 0; G < 2; ++G) {
                    const int a0 = ga[G];
#pragma unroll
                    for (int i = 0; i < 4; ++i) ld_row<float, MT>(pan + (a0 + i) * LDM + c0, acc[i]);
                    if (!first) {
                        chunk(acc, tile, Yp, a0, 0, true);
                        mac4(acc, tile, Yp, a0, a0 + 4, KB, true);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) st_row<float, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
                }
            }
            __syncthreads();
            if (active) {
                // y_J = t + (L_JJ^{-1} strictly lower) t
                float *xg = X + (b0 + J) * KB * M;
#pragma unroll
                for (int G = 0; G < 2; ++G) {
                    const int a0 = ga[G];
#pragma unroll
                    for (int i = 0; i < 4; ++i) ld_row<float, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
                    mac4(acc, tile, Tt, a0, 0, a0, false);
                    chunk(acc, tile, Tt, a0, 1, false);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        st_row<float, MT>(Yp + (a0 + i) * LDM + c0, acc[i]);
                        st_row<float, MT>(xg + (a0 + i) * M + c0, acc[i]);
                    }
                }
            }
        } else {
            const int J = steps - 1 - t;
            const bool active = isV ? hasV : hasW;
            const float *dsm = dis + buf * KB;
            if (active) {
                // t = D^{-1} y_J - (D^{-1}U_{J,J+1}) x_{J+1}   (lower incl. diagonal: q <= a)
                const float *src = (J == nb - 1) ? Yp : pan;
#pragma unroll
                for (int G = 0; G < 2; ++G) {
                    const int a0 = ga[G];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        ld_row<float, MT>(src + (a0 + i) * LDM + c0, acc[i]);
#pragma unroll
                        for (int j = 0; j < MT; ++j) acc[i][j] *= dsm[a0 + i];
                    }
                    if (J < nb - 1) {
                        mac4(acc, tile, Yp, a0, 0, a0, true);
                        chunk(acc, tile, Yp, a0, 2, true);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) st_row<float, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
                }
            }
            __syncthreads();
            // x_J = t + ((D^{-1}U_JJ)^{-1} strictly upper) t   (zeros for an absent spike)
#pragma unroll
            for (int G = 0; G < 2; ++G) {
                const int a0 = ga[G];
                if (active) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) ld_row<float, MT>(Tt + (a0 + i) * LDM + c0, acc[i]);
                    chunk(acc, tile, Tt, a0, 3, false);
                    mac4(acc, tile, Tt, a0, a0 + 4, KB, false);
#pragma unroll
                    for (int i = 0; i < 4; ++i) st_row<float, MT>(Yp + (a0 + i) * LDM + c0, acc[i]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t row = (int64_t)J * KB + a0 + i;
                    if (row < ni)
#pragma unroll
                        for (int j = 0; j < MT; ++j)
                            if (ucol[j] >= 0) Ucat[(s + row) * n2 + ucol[j]] = active ? acc[i][j] : 0.f;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Gram matrices of the two spike panels, partial sums over a chunk of blocks.
// Thread tile: 4 rows x GC columns of one Gram matrix (GC = KB/8).
template <typename T, int KB>
__global__ void __launch_bounds__(4 * KB)
    k_gram(const T *__restrict__ X, Parts P, int chunks, double *__restrict__ Gpart) {
    constexpr int NT = 4 * KB, M = 2 * KB, GC = (KB >= 8) ? KB / 8 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);  // [2][KB x M]
    const int part = blockIdx.y, ch = blockIdx.x;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int J0 = (int)((int64_t)ch * nb / chunks), J1 = (int)((int64_t)(ch + 1) * nb / chunks);
    const int gsel = threadIdx.x / (2 * KB), rem = threadIdx.x % (2 * KB);
    const int a0 = 4 * (rem / 8), b0c = GC * (rem % 8);
    const int off = gsel * KB;
    T acc[4][GC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < GC; ++j) acc[i][j] = T(0);
    // double buffer: block J+1 is copied (cp.async) while block J is multiplied
    constexpr int CH = 16 / (int)sizeof(T);
    auto stage = [&](int J, T *dst) {
        const T *src = X + (b0 + J) * (int64_t)KB * M;
        for (int e = threadIdx.x; e < KB * M / CH; e += NT) cp_async16(dst + e * CH, src + e * CH);
    };
    if (J0 < J1) stage(J0, Xs);
    cp_async_commit();
    for (int J = J0; J < J1; ++J) {
        T *cur = Xs + ((J - J0) & 1) * KB * M;
        if (J + 1 < J1) stage(J + 1, Xs + ((J + 1 - J0) & 1) * KB * M);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        for (int q = 0; q < KB; ++q) {
            T av[4], bv[GC];
            ld_row<T, 4>(cur + q * M + off + a0, av);
            ld_row<T, GC>(cur + q * M + off + b0c, bv);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < GC; ++jj) acc[i][jj] += av[i] * bv[jj];
        }
        __syncthreads();
    }
    double *dst = Gpart + (((int64_t)part * chunks + ch) * 2 + gsel) * KB * KB;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < GC; ++jj) dst[(a0 + i) * KB + b0c + jj] = (double)acc[i][jj];
}

__global__ void k_gram_reduce(const double *__restrict__ Gpart, int chunks, int64_t per_part,
                              int64_t total, double *__restrict__ G) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t part = e / per_part, rem = e % per_part;
    double s = 0.0;
    for (int ch = 0; ch < chunks; ++ch) s += Gpart[(part * chunks + ch) * per_part + rem];
    G[e] = s;
}

// B_i^T B_i and C_i^T C_i (KB x KB, zero-padded beyond k), FP64.
template <int KB>
__global__ void k_coupling_gram(const double *__restrict__ band, int64_t ld, int k, Parts P,
                                double *__restrict__ G) {
    const int part = blockIdx.x;
    const int64_t s = P.off[part], sn = P.off[part + 1];
    for (int e = threadIdx.x; e < 2 * KB * KB; e += blockDim.x) {
        const int gsel = e / (KB * KB), b = (e / KB) % KB, c = e % KB;
        double acc = 0.0;
        if (b < k && c < k) {
            if (gsel == 0 && part < P.p - 1) {
                for (int a = 0; a < k; ++a) {  // B[a][b] = band[(a-b)*ld + sn+b], b <= a
                    const double vb = (b <= a) ? band[(int64_t)(a - b) * ld + sn + b] : 0.0;
                    const double vc = (c <= a) ? band[(int64_t)(a - c) * ld + sn + c] : 0.0;
                    acc += vb * vc;
                }
            } else if (gsel == 1 && part > 0) {
                for (int a = 0; a < k; ++a) {  // C[a][b] = band[(2k+a-b)*ld + s-k+b], a <= b
                    const double vb = (a <= b) ? band[(int64_t)(2 * k + a - b) * ld + s - k + b] : 0.0;
                    const double vc = (a <= c) ? band[(int64_t)(2 * k + a - c) * ld + s - k + c] : 0.0;
                    acc += vb * vc;
                }
            }
        }
        G[(int64_t)part * 2 * KB * KB + e] = acc;
    }
}

// ---------------------------------------------------------------------------
// Jacobi eigen-decomposition of one KB x KB symmetric PSD Gram matrix.
template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr float v = 1.1920929e-07f; };

template <typename T, int KB>
__global__ void __launch_bounds__(Geo<KB>::NT)
    k_jacobi(const double *__restrict__ Gram, int r, double rank_tol, int max_sweeps,
             T *__restrict__ PQ, double *__restrict__ sigma) {
    constexpr int NT = Geo<KB>::NT, LD = KB + 1, NP = KB / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *A = reinterpret_cast<T *>(smem_raw), *V = A + KB * LD;
    __shared__ T cs[NP], sn[NP];
    __shared__ int pp[NP], qq[NP];
    __shared__ int rotated;
    __shared__ int order[KB];
    __shared__ T lam[KB];
    const int id = blockIdx.x;  // part * 2 + g
    const double *G = Gram + (int64_t)id * KB * KB;
    __shared__ T amax;
    for (int e = threadIdx.x; e < KB * KB; e += NT) {
        const int a = e / KB, b = e % KB;
        A[a * LD + b] = (T)G[e];
        V[a * LD + b] = (a == b) ? T(1) : T(0);
    }
    if (threadIdx.x == 0) {
        T m = T(0);
        for (int a = 0; a < KB; ++a) m = fmax(m, fabs((T)G[a * KB + a]));
        amax = m;
    }
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < KB - 1; ++round) {
            if (threadIdx.x < NP) {
                const int i = threadIdx.x;
                // circle method: position 0 fixed, positions 1..KB-1 rotate
                auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (KB - 1); };
                int p = player(i), q = player(KB - 1 - i);
                if (p > q) { const int t = p; p = q; q = t; }
                const T app = A[p * LD + p], aqq = A[q * LD + q], apq = A[p * LD + q];
                T c = T(1), s = T(0);
                // rotate while the pair is not yet diagonal to working precision:
                // relative to the pair, with an absolute floor of eps * (largest
                // initial diagonal entry) below which off-diagonals are rounding noise
                // (in the working precision: GB300's FP64 units are scarce, and
                // sqrt|a_pp| sqrt|a_qq| cannot overflow)
                const T thr = fmax(Eps<T>::v * (sqrt(fabs(app)) * sqrt(fabs(aqq))), T(2) * Eps<T>::v * amax);
                if (apq != T(0) && fabs(apq) > thr) {
                    const T tau = (aqq - app) / (T(2) * apq);
                    const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                    c = T(1) / sqrt(T(1) + t * t);
                    s = t * c;
                    rotated = 1;
                }
                pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
            }
            __syncthreads();
            // warp w applies the rotations of pairs w*PPW.. in turn, its lanes over
            // consecutive entries (conflict-free); a pair's indices and
            // coefficients are read once per pass, and a pair left as it is
            // (c = 1, s = 0: already diagonal) is skipped by the whole warp
            constexpr int NWJ = NT / 32, PPW = (NP + NWJ - 1) / NWJ;  // warps, pairs per warp
            const int wj = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
            for (int ii = 0; ii < PPW; ++ii) {  // rows p, q
                const int i = wj * PPW + ii;
                if (i >= NP) break;
                const T c = cs[i], s = sn[i];
                if (s == T(0)) continue;
                const int p = pp[i], q = qq[i];
                for (int j = lane; j < KB; j += 32) {
                    const T ap = A[p * LD + j], aq = A[q * LD + j];
                    A[p * LD + j] = c * ap - s * aq;
                    A[q * LD + j] = s * ap + c * aq;
                }
            }
            __syncthreads();
#pragma unroll
            for (int ii = 0; ii < PPW; ++ii) {  // columns p, q and V
                const int i = wj * PPW + ii;
                if (i >= NP) break;
                const T c = cs[i], s = sn[i];
                if (s == T(0)) continue;
                const int p = pp[i], q = qq[i];
                for (int j = lane; j < KB; j += 32) {
                    const T ap = A[j * LD + p], aq = A[j * LD + q];
                    A[j * LD + p] = c * ap - s * aq;
                    A[j * LD + q] = s * ap + c * aq;
                    const T vp = V[j * LD + p], vq = V[j * LD + q];
                    V[j * LD + p] = c * vp - s * vq;
                    V[j * LD + q] = s * vp + c * vq;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // eigenvalues, ranked by decreasing value (ties: lower index first)
    // a NaN (from a singular factorisation) ranks last so that order[] stays a permutation
    if (threadIdx.x < KB) {
        const T v = A[threadIdx.x * LD + threadIdx.x];
        lam[threadIdx.x] = (v == v) ? v : T(-INFINITY);
    }
    __syncthreads();
    if (threadIdx.x < KB) {
        const int j = threadIdx.x;
        int rk = 0;
        for (int i = 0; i < KB; ++i) rk += (lam[i] > lam[j]) || (lam[i] == lam[j] && i < j);
        order[rk] = j;
    }
    __syncthreads();
    const double s1 = sqrt(fmax((double)lam[order[0]], 0.0));
    T *out = PQ + (int64_t)id * r * KB;
    for (int c = threadIdx.x / 4; c < r; c += NT / 4) {
        // all four lanes of the group write part of row c; sign fixed so that
        // the largest-magnitude entry of each kept vector is positive
        const int j = order[c];
        const double sg = sqrt(fmax((double)lam[j], 0.0));
        const bool keep = (s1 > 0.0) && (sg > rank_tol * s1);
        int imax = 0;
        for (int q = 1; q < KB; ++q)
            if (fabs(V[q * LD + j]) > fabs(V[imax * LD + j])) imax = q;
        const T sgn = (V[imax * LD + j] < T(0)) ? T(-1) : T(1);
        for (int q = threadIdx.x % 4; q < KB; q += 4) out[c * KB + q] = keep ? sgn * V[q * LD + j] : T(0);
        if (threadIdx.x % 4 == 0) sigma[(int64_t)id * r + c] = keep ? sg : 0.0;
    }
}

// ---------------------------------------------------------------------------
// u-factors: SPIKE mode u = X V_r (panel columns times P^T); COUPLING mode the
// solved columns are u already.  Ucat row = [u_T (r) | u_W (r)].  One CTA per
// (chunk of blocks, partition); the projections are staged once.  Thread
// tile: 4 rows x UC columns of the KB x 2r output block.
template <typename T, int KB, int UC>
__global__ void __launch_bounds__(4 * KB)
    k_make_u(const T *__restrict__ X, int m, const T *__restrict__ PQ, Parts P, int r, int coupling,
             int chunks, T *__restrict__ Ucat) {
    constexpr int NT = 4 * KB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);  // KB x m
    T *Ps = Xs + KB * m;                      // KB x 2r (transposed projections)
    const int part = blockIdx.y, ch = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int J0 = (int)((int64_t)ch * nb / chunks), J1 = (int)((int64_t)(ch + 1) * nb / chunks);
    const int n2 = 2 * r, half = m / 2;
    if (!coupling)
        for (int e = threadIdx.x; e < n2 * KB; e += NT)
            Ps[(e % KB) * n2 + e / KB] = PQ[(int64_t)part * n2 * KB + e];
    const int a0 = 4 * (threadIdx.x / 16), cb = UC * (threadIdx.x % 16);
    // the halves of the panel this thread's columns read (T for col < r, W after)
    const bool needT = cb < r, needW = cb + UC > r && cb < n2;
    constexpr int CH = 16 / (int)sizeof(T);
    T *Xs1 = Ps + KB * n2;  // second staged block (after the projections)
    auto stage = [&](int J, T *dst) {
        const T *src = X + (b0 + J) * (int64_t)KB * m;
        for (int e = threadIdx.x; e < KB * m / CH; e += NT) cp_async16(dst + e * CH, src + e * CH);
    };
    if (J0 < J1) stage(J0, Xs);
    cp_async_commit();
    for (int J = J0; J < J1; ++J) {
        T *cur = ((J - J0) & 1) ? Xs1 : Xs;
        if (J + 1 < J1) stage(J + 1, ((J + 1 - J0) & 1) ? Xs1 : Xs);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        T acc[4][UC];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int u = 0; u < UC; ++u) {
                const int col = cb + u;
                const int xcol = (col < r) ? col : half + (col - r);   // coupling: panel column
                acc[i][u] = (coupling && col < n2) ? cur[(a0 + i) * m + xcol] : T(0);
            }
        if (!coupling) {
            for (int j = 0; j < KB; j += 4) {
                T xv[4][4], xw[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (needT) ld_row<T, 4>(cur + (a0 + i) * m + j, xv[i]);
                    if (needW) ld_row<T, 4>(cur + (a0 + i) * m + KB + j, xw[i]);
                }
#pragma unroll
                for (int u = 0; u < UC; ++u) {
                    const int col = cb + u;
                    if (col < n2) {
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const T pv = Ps[(j + jj) * n2 + col];
#pragma unroll
                            for (int i = 0; i < 4; ++i) acc[i][u] += ((col < r) ? xv[i][jj] : xw[i][jj]) * pv;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = (int64_t)J * KB + a0 + i;
            if (row < ni)
#pragma unroll
                for (int u = 0; u < UC; ++u)
                    if (cb + u < n2) Ucat[(s + row) * n2 + cb + u] = acc[i][u];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <typename T, int KB>
static bool spike_rhs_impl(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    if (cudaMemsetAsync(c->X, 0, (size_t)c->NB * KB * c->m * sizeof(T), c->stream) != cudaSuccess) {
        c->err = "cudaMemsetAsync failed";
        return false;
    }
    return launch(c, KID_SPIKE_RHS, [&] {
        k_spike_rhs<T, KB><<<c->p, 256, 0, c->stream>>>(c->band, c->ld, c->k, P, c->r,
                                                        c->opt.compress == LRSPIKE_COMPRESS_COUPLING,
                                                        (const T *)c->PQ, (T *)c->X, c->m);
    });
}

template <typename T, int KB, int MT, int CG>
static bool sweep_mt(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    constexpr int M = MT * CG, LDM = M + 16 / (int)sizeof(T), NT = (KB / 4) * CG;
    // (32 panel columns with KB = 64 occur in COUPLING mode only: SPIKE panels are 2 KB wide)
    if constexpr (sizeof(T) == 4 && KB == 64 && M == 32) {
        using SB = SweepBal<1>;
        static_assert(SB::bytes <= 110 * 1024, "two CTAs per SM");
        auto kb = k_sweep_bal<1>;
        cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SB::bytes);
        c->u_by_sweep = true;
        return launch(c, KID_SWEEP, [&] {
            kb<<<c->p, SB::NT, SB::bytes, c->stream>>>((const float *)c->LT, (const float *)c->UT,
                                                       (const float *)c->DI, P, c->k, (float *)c->X, c->r,
                                                       (float *)c->Ucat);
        });
    }
    if constexpr (sizeof(T) == 4) {
        using SP = SweepPipe<T, KB, MT, CG>;
        if (SP::bytes <= 110 * 1024) {
            auto kp = k_sweep_pipe<T, KB, MT, CG>;
            cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SP::bytes);
            return launch(c, KID_SWEEP, [&] {
                kp<<<c->p, NT, SP::bytes, c->stream>>>((const T *)c->LT, (const T *)c->UT, (const T *)c->DI, P,
                                                       c->k, (T *)c->X);
            });
        }
    }
    const size_t smem = (2 * KB * (KB + 1) + 2 * KB * LDM + KB) * sizeof(T);
    auto kern = k_sweep<T, KB, MT, CG>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_SWEEP, [&] {
        kern<<<c->p, NT, smem, c->stream>>>((const T *)c->LT, (const T *)c->UT, (const T *)c->DI, P, c->k,
                                            (T *)c->X);
    });
}

template <typename T, int KB>
static bool sweep_impl(Ctx *c) {
    // wide panels of the widest block use 32 column groups (8 * KB threads)
    switch (c->m / 16) {
        case 1: return sweep_mt<T, KB, 1, 16>(c);
        case 2: return sweep_mt<T, KB, 2, 16>(c);
        case 4: return sweep_mt<T, KB, 4, 16>(c);
        default:
            if constexpr (KB == 64) return sweep_mt<T, KB, 4, 32>(c);
            else return sweep_mt<T, KB, 8, 16>(c);
    }
}

template <typename T, int KB>
static bool gram_impl(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    dim3 grid(c->gram_chunks, c->p);
    const size_t smem = (size_t)2 * KB * 2 * KB * sizeof(T);  // two staged blocks
    auto kern = k_gram<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!launch(c, KID_GRAM, [&] {
            kern<<<grid, Geo<KB>::NT, smem, c->stream>>>((const T *)c->X, P, c->gram_chunks, c->Gpart);
        }))
        return false;
    const int64_t per = 2LL * KB * KB, total = per * c->p;
    return launch(c, KID_GRAM_REDUCE, [&] {
        k_gram_reduce<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(c->Gpart, c->gram_chunks,
                                                                           per, total, c->Gram);
    });
}

template <typename T, int KB>
static bool coupling_gram_impl(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    return launch(c, KID_COUPLING_GRAM, [&] {
        k_coupling_gram<KB><<<c->p, 256, 0, c->stream>>>(c->band, c->ld, c->k, P, c->Gram);
    });
}

template <typename T, int KB>
static bool jacobi_impl(Ctx *c) {
    const size_t smem = 2 * KB * (KB + 1) * sizeof(T);
    auto kern = k_jacobi<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_JACOBI, [&] {
        kern<<<2 * c->p, Geo<KB>::NT, smem, c->stream>>>(c->Gram, c->r, c->opt.rank_tol, c->fp64 ? 30 : 20, (T *)c->PQ,
                                                         c->sigma);
    });
}

// Eigendecompositions of nmat symmetric n x n FP64 matrices (n in {16, 32,
// 64}; G row-major, one per CTA): the rout leading eigenvectors as rows of
// `out` (stride n), sqrt(eigenvalue) in sigma, the rank guard of k_jacobi.
template <typename T, int KB>
static bool jacobi_batch_kb(Ctx *c, const double *G, int nmat, int rout, double rank_tol, void *out, double *sigma) {
    const size_t smem = 2 * KB * (KB + 1) * sizeof(T);
    auto kern = k_jacobi<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_JACOBI, [&] {
        kern<<<nmat, Geo<KB>::NT, smem, c->stream>>>(G, rout, rank_tol, c->fp64 ? 30 : 20, (T *)out, sigma);
    });
}

bool run_jacobi_batch(Ctx *c, int n, const double *G, int nmat, int rout, double rank_tol, void *out,
                      double *sigma) {
    if (c->fp64) {
        if (n == 16) return jacobi_batch_kb<double, 16>(c, G, nmat, rout, rank_tol, out, sigma);
        if (n == 32) return jacobi_batch_kb<double, 32>(c, G, nmat, rout, rank_tol, out, sigma);
        return jacobi_batch_kb<double, 64>(c, G, nmat, rout, rank_tol, out, sigma);
    }
    if (n == 16) return jacobi_batch_kb<float, 16>(c, G, nmat, rout, rank_tol, out, sigma);
    if (n == 32) return jacobi_batch_kb<float, 32>(c, G, nmat, rout, rank_tol, out, sigma);
    if (n == 128) return jacobi_batch_kb<float, 128>(c, G, nmat, rout, rank_tol, out, sigma);
    return jacobi_batch_kb<float, 64>(c, G, nmat, rout, rank_tol, out, sigma);
}

template <typename T, int KB, int UC>
static bool make_u_uc(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (2 * KB * c->m + 2 * c->r * KB) * sizeof(T);  // two staged blocks + projections
    auto kern = k_make_u<T, KB, UC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(c->gram_chunks, c->p);
    return launch(c, KID_MAKE_U, [&] {
        kern<<<grid, 4 * KB, smem, c->stream>>>((const T *)c->X, c->m, (const T *)c->PQ, P, c->r,
                                                c->opt.compress == LRSPIKE_COMPRESS_COUPLING, c->gram_chunks,
                                                (T *)c->Ucat);
    });
}

template <typename T, int KB>
static bool make_u_impl(Ctx *c) {
    const int uc = (2 * c->r + 15) / 16;
    if (uc <= 1) return make_u_uc<T, KB, 1>(c);
    if (uc <= 2) return make_u_uc<T, KB, 2>(c);
    return make_u_uc<T, KB, 4>(c);
}

#define LRS_KB_DISPATCH(FN)                                \
    template <typename T>                                  \
    static bool FN##_kb(Ctx *c) {                          \
        switch (c->KB) {                                   \
            case 8: return FN<T, 8>(c);                    \
            case 16: return FN<T, 16>(c);                  \
            case 32: return FN<T, 32>(c);                  \
            default: return FN<T, 64>(c);                  \
        }                                                  \
    }

LRS_KB_DISPATCH(spike_rhs_impl)
LRS_KB_DISPATCH(sweep_impl)
LRS_KB_DISPATCH(gram_impl)
LRS_KB_DISPATCH(coupling_gram_impl)
LRS_KB_DISPATCH(jacobi_impl)
LRS_KB_DISPATCH(make_u_impl)

bool run_spike_rhs(Ctx *c) { return c->fp64 ? spike_rhs_impl_kb<double>(c) : spike_rhs_impl_kb<float>(c); }
bool run_sweep(Ctx *c) {
    c->u_by_sweep = false;
    if (c->opt.pivoting) return run_sweep_piv(c);
    return c->fp64 ? sweep_impl_kb<double>(c) : sweep_impl_kb<float>(c);
}
bool run_gram(Ctx *c) { return c->fp64 ? gram_impl_kb<double>(c) : gram_impl_kb<float>(c); }
bool run_coupling_gram(Ctx *c) { return coupling_gram_impl_kb<double>(c); }
bool run_jacobi(Ctx *c) { return c->fp64 ? jacobi_impl_kb<double>(c) : jacobi_impl_kb<float>(c); }
bool run_make_u(Ctx *c) {
    if (c->u_by_sweep) return true;  // the sweep wrote Ucat itself
    return c->fp64 ? make_u_impl_kb<double>(c) : make_u_impl_kb<float>(c);
}

}  // namespace lrs
