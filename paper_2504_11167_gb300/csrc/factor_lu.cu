// Banded LU of every partition A_i (the D-stage factorisation of paper
// section 2.1, "A = D S": D holds the diagonal blocks A_i, factorised
// independently; section 3.3 states each A_i is factorised by a direct
// solver).  No pivoting here; the matrices of this mode are diagonally
// dominant.
//
// One CTA per partition walks the chain of nb_i block steps.  With blocks of
// KB >= k rows the partition is block tridiagonal, and block step J is
//   1. S_J = L U, together with L^{-1} and U^{-1}: a recursive blocked
//      factorisation (halves, then 16 x 16 base cases that eliminate against
//      appended identity blocks, so that the row operations build L^{-1} and
//      the column multipliers build U^{-1}); the off-diagonal blocks of the
//      halves are register-tiled products on shared-memory tiles;
//   2. U_{J,J+1} = L^{-1} A_{J,J+1},  L_{J+1,J} = A_{J+1,J} U^{-1}  (products);
//   3. S_{J+1} = A_{J+1,J+1} - L_{J+1,J} U_{J,J+1}                   (product).
// This is exactly the scalar band LU grouped in blocks (no pivoting, the band
// does not grow): U_{J,J+1} is lower and L_{J+1,J} upper triangular, and the
// products skip the structurally zero triangles.  Every step writes the
// packed solve tiles of its block directly:
//   LT[J] = [ L_JJ^{-1} strictly lower | L_{J,J-1} upper incl. diagonal ]
//   UT[J] = [ (D^{-1}U_JJ)^{-1} strictly upper | D^{-1}U_{J,J+1} lower incl. diagonal ]
//   DI[J] = D^{-1},  D = diag(U_JJ)
// so the solve kernels need only matrix-vector products per block step.
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "tile_ops.cuh"

namespace lrs {

template <typename T> struct Pad { static constexpr int v = 16 / (int)sizeof(T); };

// Stages band column block jc of a partition into three KB x KB tiles of row
// stride LDt: up = A_{jc-1,jc}, dg = A_{jc,jc}, lo = A_{jc+1,jc} (partition-
// local, with the identity on padding rows).  Reads are coalesced (one band
// diagonal is KB consecutive doubles) and issued eight per thread before any
// is consumed; the column block after jc is prefetched into L2 for the next
// block step.
template <typename T, int KB>
__device__ void load_colblock(const double *__restrict__ band, int64_t ld, int k, int64_t s,
                              int64_t ni, int64_t jc, T *up, T *dg, T *lo, int LDt) {
    constexpr int NT = 4 * KB, BATCH = 8;
    for (int e = threadIdx.x; e < KB * LDt; e += NT) {
        up[e] = T(0);
        dg[e] = T(0);
        lo[e] = T(0);
    }
    const int64_t col0 = jc * KB;
    const int nd = 2 * k + 1;
    // L2 prefetch of column block jc+1 (128-byte lines of each diagonal)
    if ((jc + 1) * KB < ni) {
        constexpr int LINES = (KB * 8 + 127) / 128 + 1;
        for (int e = threadIdx.x; e < nd * LINES; e += NT) {
            const int d = e / LINES, l = e % LINES;
            const int64_t c0 = (jc + 1) * KB + (int64_t)l * 16;
            if (c0 < ni) {
                const double *pa = band + (int64_t)d * ld + s + c0;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
            }
        }
    }
    __syncthreads();
    // scatter one band value (diagonal d, column b of the block) into its tile
    auto put = [&](int d, int b, double v) {
        const int64_t col = col0 + b;
        const int arel = b + d - k;
        const int64_t row = col0 + arel;
        if (col >= ni) {
            if (d != k) return;
            v = 1.0;
        } else if (row < 0 || row >= ni) {
            return;
        }
        if (arel < 0) up[(KB + arel) * LDt + b] = (T)v;
        else if (arel < KB) dg[arel * LDt + b] = (T)v;
        else lo[(arel - KB) * LDt + b] = (T)v;
    };
    const double *src0 = band + s + col0;
    if (((ld | (s + col0)) & 1) == 0) {
        // 16-byte loads: a warp reads 64 / KB diagonals per instruction and
        // all of its loads are issued before any value is stored
        constexpr int CH = KB / 2;                 // double2 per diagonal segment
        constexpr int RPI = 32 / CH;               // diagonals per warp instruction
        constexpr int NW = NT / 32;
        constexpr int MAXR = (2 * KB + 1 + NW * RPI - 1) / (NW * RPI);
        constexpr int RB = (MAXR < 9) ? MAXR : 9;  // loads in flight per lane
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        const int dl = l / CH, ch = l % CH;
        for (int it0 = 0; it0 < MAXR; it0 += RB) {
            double2 v[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int d = ((it0 + u) * NW + w) * RPI + dl;
                const int b = 2 * ch;
                v[u] = make_double2(0.0, 0.0);
                if (it0 + u < MAXR && d < nd) {
                    if (col0 + b + 1 < ni)
                        v[u] = __ldg(reinterpret_cast<const double2 *>(src0 + (int64_t)d * ld + b));
                    else if (col0 + b < ni)
                        v[u].x = __ldg(src0 + (int64_t)d * ld + b);
                }
            }
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int d = ((it0 + u) * NW + w) * RPI + dl;
                if (it0 + u < MAXR && d < nd) {
                    put(d, 2 * ch, v[u].x);
                    put(d, 2 * ch + 1, v[u].y);
                }
            }
        }
    } else {
        for (int base = threadIdx.x; base < nd * KB; base += NT * BATCH) {
            double v[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
                const int e = base + u * NT;
                v[u] = 0.0;
                if (e < nd * KB && col0 + e % KB < ni) v[u] = __ldg(src0 + (int64_t)(e / KB) * ld + e % KB);
            }
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
                const int e = base + u * NT;
                if (e < nd * KB) put(e / KB, e % KB, v[u]);
            }
        }
    }
    __syncthreads();
}

// ---- register-tiled products of S x S shared-memory tiles -----------------
enum Shape { FULL = 0, LOWER = 1, UPPER = 2 };  // lower/upper incl. the diagonal

template <int S, int NT> struct GemmGeo {
    static constexpr int EPT = (S * S >= NT) ? S * S / NT : 1;  // outputs per thread
    static constexpr int TN = (EPT >= 4) ? 4 : EPT;
    static constexpr int TM = EPT / TN;
    static constexpr int GX = S / TN, GY = S / TM;
    static constexpr int ACTIVE = GX * GY;
};

// One thread's TM x TN tile of A * B (rows a0.., columns b0..), through
// registers so that the result may overwrite an operand after a barrier.
// Triangular operands bound the inner index: exact zeros elsewhere.
template <typename T, int S, int NT, int SA, int SB>
struct TileGemm {
    using G = GemmGeo<S, NT>;
    T acc[G::TM][G::TN];
    int a0 = 0, b0 = 0;
    bool act = false;
    __device__ __forceinline__ void compute(const T *A, const T *B, int ld) {
        act = threadIdx.x < G::ACTIVE;
        a0 = (threadIdx.x / G::GX) * G::TM;
        b0 = (threadIdx.x % G::GX) * G::TN;
#pragma unroll
        for (int i = 0; i < G::TM; ++i)
#pragma unroll
            for (int j = 0; j < G::TN; ++j) acc[i][j] = T(0);
        if (!act) return;
        int qlo = 0, qhi = S;
        if (SA == UPPER) qlo = a0;
        if (SB == LOWER) qlo = (b0 > qlo) ? b0 : qlo;
        if (SA == LOWER) qhi = a0 + G::TM;
        if (SB == UPPER) qhi = (b0 + G::TN < qhi) ? b0 + G::TN : qhi;
#pragma unroll 4
        for (int q = qlo; q < qhi; ++q) {
            T av[G::TM], bv[G::TN];
#pragma unroll
            for (int i = 0; i < G::TM; ++i) av[i] = A[(a0 + i) * ld + q];
            ld_row<T, G::TN>(B + q * ld + b0, bv);
#pragma unroll
            for (int i = 0; i < G::TM; ++i)
#pragma unroll
                for (int j = 0; j < G::TN; ++j) acc[i][j] += av[i] * bv[j];
        }
    }
    // mode 0: C = A B; 1: C = -A B; 2: C = C - A B
    __device__ __forceinline__ void store(T *C, int ld, int mode) const {
        if (!act) return;
#pragma unroll
        for (int i = 0; i < G::TM; ++i)
#pragma unroll
            for (int j = 0; j < G::TN; ++j) {
                T *c = C + (a0 + i) * ld + b0 + j;
                *c = (mode == 0) ? acc[i][j] : (mode == 1) ? -acc[i][j] : *c - acc[i][j];
            }
    }
};

// The same product on the tensor cores (TF32 operands rounded to nearest,
// FP32 accumulation): the S x S output in m16n8 tiles spread over the warps,
// mma.sync m16n8k8 over k-blocks of 8.  k-blocks outside the operands'
// triangles are skipped; inside a straddling k-block the masked elements are
// zeroed in the fragments (the unused triangles may hold temporaries).
// Fragments (m16n8k8, .tf32): lane = 4g + t; A: (g, t) (g+8, t) (g, t+4)
// (g+8, t+4); B: (t, g) (t+4, g); C: (g, 2t) (g, 2t+1) (g+8, 2t) (g+8, 2t+1).
__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}

template <int S, int NT, int SA, int SB>
struct TileGemmTC {
    static constexpr int NTL = S / 8, TILES = (S / 16) * NTL, WARPS = NT / 32;
    static constexpr int PER = (TILES + WARPS - 1) / WARPS;
    float c[PER][4];
    static __device__ __forceinline__ bool inA(int i, int q) {
        return SA == LOWER ? q <= i : SA == UPPER ? q >= i : true;
    }
    static __device__ __forceinline__ bool inB(int q, int j) {
        return SB == LOWER ? q >= j : SB == UPPER ? q <= j : true;
    }
    __device__ __forceinline__ void compute(const float *A, const float *B, int ld) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int w = 0; w < PER; ++w) {
            c[w][0] = c[w][1] = c[w][2] = c[w][3] = 0.f;
            const int tile = warp + w * WARPS;
            if (tile >= TILES) continue;
            const int m0 = (tile / NTL) * 16, n0 = (tile % NTL) * 8;
#pragma unroll
            for (int q0 = 0; q0 < S; q0 += 8) {
                if (SA == LOWER && q0 > m0 + 15) continue;
                if (SA == UPPER && q0 + 7 < m0) continue;
                if (SB == LOWER && q0 + 7 < n0) continue;
                if (SB == UPPER && q0 > n0 + 7) continue;
                const int r0 = m0 + g, r1 = m0 + g + 8, k0 = q0 + t, k1 = q0 + t + 4, cn = n0 + g;
                const unsigned a0 = to_tf32(inA(r0, k0) ? A[r0 * ld + k0] : 0.f);
                const unsigned a1 = to_tf32(inA(r1, k0) ? A[r1 * ld + k0] : 0.f);
                const unsigned a2 = to_tf32(inA(r0, k1) ? A[r0 * ld + k1] : 0.f);
                const unsigned a3 = to_tf32(inA(r1, k1) ? A[r1 * ld + k1] : 0.f);
                const unsigned b0 = to_tf32(inB(k0, cn) ? B[k0 * ld + cn] : 0.f);
                const unsigned b1 = to_tf32(inB(k1, cn) ? B[k1 * ld + cn] : 0.f);
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};\n"
                    : "+f"(c[w][0]), "+f"(c[w][1]), "+f"(c[w][2]), "+f"(c[w][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
    }
    // mode 0: C = A B; 1: C = -A B; 2: C = C - A B
    __device__ __forceinline__ void store(float *C, int ld, int mode) const {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int w = 0; w < PER; ++w) {
            const int tile = warp + w * WARPS;
            if (tile >= TILES) continue;
            const int m0 = (tile / NTL) * 16, n0 = (tile % NTL) * 8;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + g + (e >> 1) * 8, col = n0 + 2 * t + (e & 1);
                float *p = C + row * ld + col;
                *p = (mode == 0) ? c[w][e] : (mode == 1) ? -c[w][e] : *p - c[w][e];
            }
        }
    }
};

// SIMT tiles, or tensor-core tiles for FP32 with TC (blocks of 16 and more)
template <typename T, bool TC, int S, int NT, int SA, int SB>
using Gemm = typename std::conditional<TC && std::is_same<T, float>::value && (S >= 16),
                                       TileGemmTC<S, NT, SA, SB>, TileGemm<T, S, NT, SA, SB>>::type;

// Base case: N x N block S (row stride ld) factorised in place into L\U while
// the row operations turn an identity into L^{-1} and the column multipliers
// of an identity block appended below S turn into U^{-1}.  One warp does it
// with the three blocks in registers: lane l owns row l % N and the CPL
// columns (l / N) * CPL .. + CPL - 1 of S, L^{-1} and U^{-1}; the pivot row
// and column move by shuffles, so no barrier is needed between pivots.
template <typename T, int N, int NT>
__device__ void base_lu_inv(T *S, T *Li, T *Ui, int ld, int64_t grow0, int64_t *status) {
    constexpr int CPL = N * N / 32;  // columns per lane
    if (threadIdx.x < 32) {
        const int l = threadIdx.x, a = l % N, h = l / N;
        T sv[CPL], li[CPL], ui[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int b = h * CPL + j;
            sv[j] = S[a * ld + b];
            li[j] = (a == b) ? T(1) : T(0);
            ui[j] = (a == b) ? T(1) : T(0);
        }
        // pivot loop fully unrolled: every register index is a compile-time constant
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const int jc = c % CPL, hc = c / CPL;
            const T piv = __shfl_sync(0xffffffffu, sv[jc], c + N * hc);
            const T colS = __shfl_sync(0xffffffffu, sv[jc], a + N * hc);   // S[a][c]
            const T colU = __shfl_sync(0xffffffffu, ui[jc], a + N * hc);   // Ui[a][c]
            T rowS[CPL], rowL[CPL];
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                rowS[j] = __shfl_sync(0xffffffffu, sv[j], c + N * h);      // S[c][b]
                rowL[j] = __shfl_sync(0xffffffffu, li[j], c + N * h);      // Li[c][b]
            }
            const bool ok = usable_pivot<T>(piv);
            if (!ok && l == 0) atomicMin((unsigned long long *)status, (unsigned long long)(grow0 + c));
            const T pinv = ok ? fast_rcp<T>(piv) : T(1);
            const T ml = colS * pinv, mu = colU * pinv;
            const bool below = a > c;
            const T lrow = below ? ml : T(0), urow = below ? T(0) : mu;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                const int b = h * CPL + j;
                const bool right = b > c;
                const T ns = sv[j] - (right ? lrow : T(0)) * rowS[j];
                const T nl = li[j] - (right ? T(0) : lrow) * rowL[j];
                const T nu = ui[j] - (right ? urow : T(0)) * rowS[j];
                const bool isc = (b == c);
                sv[j] = (isc && below) ? ml : ns;
                li[j] = nl;
                ui[j] = (isc && !below) ? mu : nu;
            }
        }
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int b = h * CPL + j;
            S[a * ld + b] = sv[j];
            Li[a * ld + b] = li[j];
            Ui[a * ld + b] = ui[j];
        }
    }
    __syncthreads();
}

// S = L U with L^{-1} in Li and U^{-1} in Ui (N x N blocks, row stride ld).
// Halves: S11 = L11 U11 (recursively); U12 = L11^{-1} S12; L21 = S21 U11^{-1};
// S22 -= L21 U12; S22 = L22 U22 (recursively);
// (L^{-1})_21 = -L22^{-1} L21 L11^{-1},  (U^{-1})_12 = -U11^{-1} U12 U22^{-1}.
// The two temporaries live in the unused triangles Li_12 and Ui_21.
template <typename T, int N, int NT, bool TC = false>
__device__ void lu_inv(T *S, T *Li, T *Ui, int ld, int64_t grow0, int64_t *status) {
    if constexpr (N <= 16) {
        base_lu_inv<T, N, NT>(S, Li, Ui, ld, grow0, status);
    } else {
        constexpr int h = N / 2;
        T *S12 = S + h, *S21 = S + h * ld, *S22 = S + h * ld + h;
        T *Li12 = Li + h, *Li21 = Li + h * ld, *Li22 = Li + h * ld + h;
        T *Ui12 = Ui + h, *Ui21 = Ui + h * ld, *Ui22 = Ui + h * ld + h;
        lu_inv<T, h, NT, TC>(S, Li, Ui, ld, grow0, status);
        {
            Gemm<T, TC, h, NT, LOWER, FULL> g1;
            Gemm<T, TC, h, NT, FULL, UPPER> g2;
            g1.compute(Li, S12, ld);   // U12 = L11^{-1} S12
            g2.compute(S21, Ui, ld);   // L21 = S21 U11^{-1}
            __syncthreads();
            g1.store(S12, ld, 0);
            g2.store(S21, ld, 0);
            __syncthreads();
        }
        {
            Gemm<T, TC, h, NT, FULL, FULL> g;
            g.compute(S21, S12, ld);
            g.store(S22, ld, 2);       // S22 -= L21 U12
            __syncthreads();
        }
        lu_inv<T, h, NT, TC>(S22, Li22, Ui22, ld, grow0 + h, status);
        {
            Gemm<T, TC, h, NT, FULL, LOWER> g1;
            Gemm<T, TC, h, NT, FULL, UPPER> g2;
            g1.compute(S21, Li, ld);   // L21 L11^{-1}
            g2.compute(S12, Ui22, ld); // U12 U22^{-1}
            g1.store(Li12, ld, 0);
            g2.store(Ui21, ld, 0);
            __syncthreads();
        }
        {
            Gemm<T, TC, h, NT, LOWER, FULL> g1;
            Gemm<T, TC, h, NT, UPPER, FULL> g2;
            g1.compute(Li22, Li12, ld);
            g2.compute(Ui, Ui21, ld);
            g1.store(Li21, ld, 1);     // (L^{-1})_21
            g2.store(Ui12, ld, 1);     // (U^{-1})_12
            __syncthreads();
        }
        for (int e = threadIdx.x; e < h * h; e += NT) {
            Li12[(e / h) * ld + e % h] = T(0);
            Ui21[(e / h) * ld + e % h] = T(0);
        }
        __syncthreads();
    }
}

template <typename T, int KB, bool TC>
__global__ void __launch_bounds__(4 * KB)
    k_band_lu(const double *__restrict__ band, int64_t ld, int k, Parts P, T *__restrict__ LT,
              T *__restrict__ UT, T *__restrict__ DI, int64_t *__restrict__ status) {
    constexpr int NT = 4 * KB, LD = KB + Pad<T>::v, TS = KB * LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Sb = reinterpret_cast<T *>(smem_raw);  // S_J, then A_{J+1,J+1} and S_{J+1}
    T *Li = Sb + TS;                          // L_JJ^{-1}
    T *Ui = Li + TS;                          // U_JJ^{-1}
    T *Bu = Ui + TS;                          // A_{J,J+1}, then U_{J,J+1}
    T *Bl0 = Bu + TS;                         // A_{J+1,J}, then L_{J+1,J} (two by parity)
    T *Bl1 = Bl0 + TS;
    T *dU = Bl1 + TS;                         // diag(U_JJ)

    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int t = threadIdx.x;

    load_colblock<T, KB>(band, ld, k, s, ni, 0, Bu, Sb, Bl0, LD);
    for (int J = 0; J < nb; ++J) {
        const bool last = (J == nb - 1);
        T *Blc = (J & 1) ? Bl1 : Bl0;
        T *Bln = (J & 1) ? Bl0 : Bl1;
        const int64_t gJ = b0 + J;
        T *lt = LT + gJ * KB * KB;
        T *ut = UT + gJ * KB * KB;

        lu_inv<T, KB, NT, TC>(Sb, Li, Ui, LD, s + (int64_t)J * KB, status);
        if (t < KB) dU[t] = Sb[t * LD + t];
        __syncthreads();
        for (int e = t; e < KB * KB; e += NT) {
            const int a = e / KB, b = e % KB;
            if (a > b) lt[e] = Li[a * LD + b];
            else if (J == 0) lt[e] = T(0);               // L_{0,-1} does not exist
            if (a < b) ut[e] = Ui[a * LD + b] * dU[b];   // (D^{-1}U)^{-1} = U^{-1} D
            else if (last) ut[e] = T(0);                 // no U_{J,J+1} for the last block
        }
        if (t < KB) DI[gJ * KB + t] = Ui[t * LD + t];
        if (last) break;

        load_colblock<T, KB>(band, ld, k, s, ni, J + 1, Bu, Sb, Bln, LD);
        {
            Gemm<T, TC, KB, NT, LOWER, LOWER> gz;
            Gemm<T, TC, KB, NT, UPPER, UPPER> gy;
            gz.compute(Li, Bu, LD);    // U_{J,J+1} = L^{-1} A_{J,J+1}
            gy.compute(Blc, Ui, LD);   // L_{J+1,J} = A_{J+1,J} U^{-1}
            __syncthreads();
            gz.store(Bu, LD, 0);
            gy.store(Blc, LD, 0);
            __syncthreads();
        }
        {
            Gemm<T, TC, KB, NT, UPPER, LOWER> gs;
            gs.compute(Blc, Bu, LD);
            gs.store(Sb, LD, 2);       // S_{J+1} = A_{J+1,J+1} - L_{J+1,J} U_{J,J+1}
        }
        T *ltn = LT + (gJ + 1) * KB * KB;
        for (int e = t; e < KB * KB; e += NT) {
            const int a = e / KB, b = e % KB;
            if (a >= b) ut[e] = Bu[a * LD + b] / dU[a];  // D^{-1} U_{J,J+1}
            if (a <= b) ltn[e] = Blc[a * LD + b];        // L_{J+1,J}
        }
        __syncthreads();
    }
}

template <typename T, int KB>
static bool lu_impl(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    constexpr int LD = KB + Pad<T>::v;
    const size_t smem = (6 * KB * LD + KB) * sizeof(T);
    // TF32: the block products on the tensor cores (FP32 factors otherwise)
    auto kern = (c->opt.precision == LRSPIKE_MIXED_TF32) ? k_band_lu<T, KB, true> : k_band_lu<T, KB, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_LU, [&] {
        kern<<<c->p, 4 * KB, smem, c->stream>>>(c->band, c->ld, c->k, P, (T *)c->LT, (T *)c->UT, (T *)c->DI,
                                                c->status);
    });
}

template <typename T>
static bool lu_kb(Ctx *c) {
    switch (c->KB) {
        case 8: return lu_impl<T, 8>(c);
        case 16: return lu_impl<T, 16>(c);
        case 32: return lu_impl<T, 32>(c);
        default: return lu_impl<T, 64>(c);
    }
}

// Wide bands: batched LU with both triangular inverses of one 64 x 64
// diagonal sub-block per partition (the base case of the recursive block
// factorisation).  A, Li, Ui are column-major views (leading dimension lda /
// ldo, one matrix per partition at stride sA / sO); A is overwritten.
// grow0 of partition i = P.off[i] + row0 (the global row of the sub-block).
template <typename T>
__global__ void __launch_bounds__(256)
    k_lu_inv64(T *A, int lda, int64_t sA, T *Li, T *Ui, int ldo, int64_t sO, Parts P, int64_t row0,
               int64_t *status) {
    constexpr int N = 64, NT = 256, LD = N + Pad<T>::v;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Sb = reinterpret_cast<T *>(smem_raw), *Ls = Sb + N * LD, *Us = Ls + N * LD;
    const int part = blockIdx.x;
    T *a = A + part * sA;
    for (int e = threadIdx.x; e < N * N; e += NT) {
        const int r = e % N, c = e / N;  // column-major source: consecutive threads, consecutive rows
        Sb[r * LD + c] = a[(int64_t)c * lda + r];
    }
    __syncthreads();
    lu_inv<T, N, NT>(Sb, Ls, Us, LD, P.off[part] + row0, status);
    T *li = Li + part * sO, *ui = Ui + part * sO;
    for (int e = threadIdx.x; e < N * N; e += NT) {
        const int r = e % N, c = e / N;
        li[(int64_t)c * ldo + r] = Ls[r * LD + c];
        ui[(int64_t)c * ldo + r] = Us[r * LD + c];
    }
}

bool run_lu_inv64(Ctx *c, void *A, int lda, int64_t sA, void *Li, void *Ui, int ldo, int64_t sO, int64_t row0) {
    Parts P{c->off_d, c->boff_d, c->p};
    if (c->fp64) {
        constexpr int LD = 64 + Pad<double>::v;
        const size_t smem = 3 * 64 * LD * sizeof(double);
        cudaFuncSetAttribute(k_lu_inv64<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch(c, KID_WIDE_LU64, [&] {
            k_lu_inv64<double><<<c->p, 256, smem, c->stream>>>((double *)A, lda, sA, (double *)Li, (double *)Ui,
                                                              ldo, sO, P, row0, c->status);
        });
    }
    constexpr int LD = 64 + Pad<float>::v;
    const size_t smem = 3 * 64 * LD * sizeof(float);
    cudaFuncSetAttribute(k_lu_inv64<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_WIDE_LU64, [&] {
        k_lu_inv64<float><<<c->p, 256, smem, c->stream>>>((float *)A, lda, sA, (float *)Li, (float *)Ui, ldo, sO,
                                                         P, row0, c->status);
    });
}

bool run_band_lu(Ctx *c) {
    if (c->opt.pivoting) return run_band_lu_piv(c);
    // TF32 keeps the block-recursive kernel (its block products are what runs on the tensor cores)
    if (c->opt.precision != LRSPIKE_MIXED_TF32) return run_band_lu_col(c);
    return c->fp64 ? lu_kb<double>(c) : lu_kb<float>(c);
}

}  // namespace lrs
