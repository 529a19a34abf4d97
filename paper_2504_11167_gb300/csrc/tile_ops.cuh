// Block-step products shared by the multi-right-hand-side sweeps (spike
// solves and D-stage).  A sweep over a partition is a chain of block steps;
// with the tiles prepared by k_prep_inverse every step is two small
// matrix products on a KB x m panel held in shared memory:
//   forward  (L y = b):  t = b_J - L_{J,J-1} y_{J-1};   y_J = L_JJ^{-1} t
//   backward (U x = y):  t = D^{-1} y_J - (D^{-1}U_{J,J+1}) x_{J+1};
//                        x_J = (D^{-1} U_JJ)^{-1} t
// Packed tiles: LT = [L^{-1} strictly lower | L_{J,J-1} upper incl. diagonal],
// UT = [unit-upper inverse strictly upper | D^{-1}U_{J,J+1} lower incl. diag].
// Thread layout: tile row a = tid / 4; the four lanes of a row either split
// the columns (COLS, wide panels) or split the dot product and combine it
// with two shuffles (DOTS, narrow panels such as one right-hand side).
#pragma once
#include "common.cuh"

namespace lrs {

enum class Split { COLS, DOTS };

// All dot products run over the full tile row with the triangle selected by a
// mask, so the loops have compile-time trip counts and their shared-memory
// loads are issued back to back.
//   MODE 0: j >= a (upper incl. diagonal)   MODE 1: j < a (strictly lower)
//   MODE 2: j <= a (lower incl. diagonal)   MODE 3: j > a (strictly upper)
// TR = false reads the tile as stored (row a), TR = true reads its transpose
// (column a), for the transposed sweeps.
template <int MODE>
__device__ __forceinline__ bool tri_in(int j, int a) {
    return MODE == 0 ? j >= a : MODE == 1 ? j < a : MODE == 2 ? j <= a : j > a;
}

// out[a][c] = base[a][c] (op) sum_j M[a][j] V[j][c] over the masked triangle.
// SUBTRACT: out = base - sum; else out = base + sum.  base may alias out
// (each entry is read and written by the same thread).
template <typename T, int KB, Split S, int MODE, bool TR, bool SUBTRACT>
__device__ __forceinline__ void tri_product(const T *__restrict__ M, int LDS, const T *V, const T *base,
                                            T *out, int LDM, int m, const T *rowscale) {
    const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
    // FP64 multiply-adds are scarce on this GPU: there the loops stop at the
    // triangle's edge instead of masking a full row
    constexpr bool BOUNDED = sizeof(T) == 8;
    const int jlo = BOUNDED ? ((MODE == 0) ? a : (MODE == 3) ? a + 1 : 0) : 0;
    const int jhi = BOUNDED ? ((MODE == 1) ? a : (MODE == 2) ? a + 1 : KB) : KB;
    if (S == Split::COLS) {
        for (int c = q; c < m; c += 4) {
            T acc = T(0);
#pragma unroll 8
            for (int j = jlo; j < jhi; ++j) {
                const T mv = TR ? M[j * LDS + a] : M[a * LDS + j];
                acc += tri_in<MODE>(j, a) ? mv * V[j * LDM + c] : T(0);
            }
            T b0 = base[a * LDM + c];
            if (rowscale) b0 *= rowscale[a];
            out[a * LDM + c] = SUBTRACT ? b0 - acc : b0 + acc;
        }
    } else {
        for (int c = 0; c < m; ++c) {
            T acc = T(0);
            if (BOUNDED) {
                for (int j = jlo + ((q - jlo) & 3); j < jhi; j += 4) {
                    const T mv = TR ? M[j * LDS + a] : M[a * LDS + j];
                    acc += mv * V[j * LDM + c];
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < KB / 4; ++jj) {
                    const int j = q + 4 * jj;
                    const T mv = TR ? M[j * LDS + a] : M[a * LDS + j];
                    acc += tri_in<MODE>(j, a) ? mv * V[j * LDM + c] : T(0);
                }
            }
            acc = quad_sum(acc);
            if (q == 0) {
                T b0 = base[a * LDM + c];
                if (rowscale) b0 *= rowscale[a];
                out[a * LDM + c] = SUBTRACT ? b0 - acc : b0 + acc;
            }
        }
    }
}

// Forward (L y = b): Tt holds b_J on entry; Yp holds y_{J-1} on entry, y_J on exit.
template <typename T, int KB, Split S>
__device__ __forceinline__ void fwd_step(const T *__restrict__ Ls, int LDS, T *Tt, T *Yp, int LDM,
                                         int m, bool first) {
    if (!first) tri_product<T, KB, S, 0, false, true>(Ls, LDS, Yp, Tt, Tt, LDM, m, nullptr);
    __syncthreads();
    tri_product<T, KB, S, 1, false, false>(Ls, LDS, Tt, Tt, Yp, LDM, m, nullptr);
    __syncthreads();
}

// Backward (U x = y): Tt holds y_J on entry; Xn holds x_{J+1} on entry, x_J on exit.
template <typename T, int KB, Split S>
__device__ __forceinline__ void bwd_step(const T *__restrict__ Us, int LDS, const T *__restrict__ dsm,
                                         T *Tt, T *Xn, int LDM, int m, bool first) {
    if (first) {
        const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
        for (int c = q; c < m; c += 4) Tt[a * LDM + c] *= dsm[a];
    } else {
        tri_product<T, KB, S, 2, false, true>(Us, LDS, Xn, Tt, Tt, LDM, m, dsm);
    }
    __syncthreads();
    tri_product<T, KB, S, 3, false, false>(Us, LDS, Tt, Tt, Xn, LDM, m, nullptr);
    __syncthreads();
}

// Transposed steps, for A^T = U^T L^T, with the same packed tiles.
//   forward  (U^T z = h): with z^_J = D_J z_J,
//            t = h_J - (D^{-1}U_{J-1,J})^T z^_{J-1};  z^_J = ((D^{-1}U_JJ)^{-1})^T t
//            (the caller applies z_J = D_J^{-1} z^_J after the sweep)
//   backward (L^T l = z): t = z_J - L_{J+1,J}^T l_{J+1};  l_J = (L_JJ^{-1})^T t
// Uprev = UT[J-1], Ucur = UT[J]; Lnext = LT[J+1], Lcur = LT[J].  In the
// transposed product row a of the result takes column a of the tile, so the
// triangle conditions flip: (U_{J-1,J}' lower)^T -> j >= a; unit-upper^T -> j < a;
// (L_{J+1,J} upper)^T -> j <= a; (unit-lower)^T -> j > a.
template <typename T, int KB, Split S>
__device__ __forceinline__ void fwdT_step(const T *__restrict__ Uprev, const T *__restrict__ Ucur,
                                          int LDS, T *Tt, T *Zp, int LDM, int m, bool first) {
    if (!first) tri_product<T, KB, S, 0, true, true>(Uprev, LDS, Zp, Tt, Tt, LDM, m, nullptr);
    __syncthreads();
    tri_product<T, KB, S, 1, true, false>(Ucur, LDS, Tt, Tt, Zp, LDM, m, nullptr);
    __syncthreads();
}

template <typename T, int KB, Split S>
__device__ __forceinline__ void bwdT_step(const T *__restrict__ Lnext, const T *__restrict__ Lcur,
                                          int LDS, T *Tt, T *Lp, int LDM, int m, bool first) {
    if (!first) tri_product<T, KB, S, 2, true, true>(Lnext, LDS, Lp, Tt, Tt, LDM, m, nullptr);
    __syncthreads();
    tri_product<T, KB, S, 3, true, false>(Lcur, LDS, Tt, Tt, Lp, LDM, m, nullptr);
    __syncthreads();
}

// Thread map for register-tiled panel products on KB x (CG*MT) panels with
// (KB/4)*CG threads: thread (ty, tx) owns rows 4ty..4ty+3 and columns
// MT*tx..MT*tx+MT-1.  A warp covers a band of (at most) 16 rows and one half
// of the columns, so a triangular loop bound is uniform per warp band and a
// whole half of the panel (e.g. zero spike columns) can be skipped per warp.
template <int KB, int CG = 16> struct PanelMap {
    static constexpr int LRG = (KB >= 16) ? 4 : 2;  // row groups per warp
    static constexpr int CPW = 32 / LRG;            // column groups per warp
    static constexpr int WR = KB / (4 * LRG);       // warps along the rows
    __device__ static __forceinline__ void get(int t, int &ty, int &tx) {
        const int w = t >> 5, l = t & 31;
        ty = (w % WR) * LRG + (l % LRG);
        tx = (w / WR) * CPW + (l / LRG);
    }
};

// Loads MT consecutive values (16-byte vector loads where the type allows).
template <typename T, int MT>
__device__ __forceinline__ void ld_row(const T *p, T (&v)[MT]) {
    if constexpr (sizeof(T) == 4 && MT % 4 == 0) {
#pragma unroll
        for (int j = 0; j < MT; j += 4) {
            const float4 f = *reinterpret_cast<const float4 *>(p + j);
            v[j] = f.x; v[j + 1] = f.y; v[j + 2] = f.z; v[j + 3] = f.w;
        }
    } else if constexpr (sizeof(T) == 8 && MT % 2 == 0) {
#pragma unroll
        for (int j = 0; j < MT; j += 2) {
            const double2 d = *reinterpret_cast<const double2 *>(p + j);
            v[j] = d.x; v[j + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < MT; ++j) v[j] = p[j];
    }
}

template <typename T, int MT>
__device__ __forceinline__ void st_row(T *p, const T (&v)[MT]) {
    if constexpr (sizeof(T) == 4 && MT % 4 == 0) {
#pragma unroll
        for (int j = 0; j < MT; j += 4) *reinterpret_cast<float4 *>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else if constexpr (sizeof(T) == 8 && MT % 2 == 0) {
#pragma unroll
        for (int j = 0; j < MT; j += 2) *reinterpret_cast<double2 *>(p + j) = make_double2(v[j], v[j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < MT; ++j) p[j] = v[j];
    }
}

// One right-hand side, FP32: lane q of row a takes the contiguous quarter
// [q KB/4, (q+1) KB/4) of the masked dot product sum_j M[a][j] v[j] (16-byte
// vector loads of the tile row and of v, four independent partial sums; the
// quad of lanes combines them with two shuffles, every lane gets the sum).
// The triangle is given as per-lane bit masks: msk[w] is all ones where entry
// q KB/4 + w of the row belongs to the product (INV: where it does not), so
// each entry costs one AND and one fused multiply-add (masked-out entries
// contribute fma(+0, v, acc) = acc).
template <int KB, bool INV>
__device__ __forceinline__ float tri_dot1m(const float *__restrict__ Mrow, const float *v, int q,
                                          const unsigned (&msk)[KB / 4]) {
    constexpr int QW = KB / 4, VW = QW < 4 ? QW : 4;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < QW; u += VW) {
        float mv[VW], vv[VW];
        ld_row<float, VW>(Mrow + q * QW + u, mv);
        ld_row<float, VW>(v + q * QW + u, vv);
#pragma unroll
        for (int w = 0; w < VW; ++w) {
            const unsigned m = INV ? ~msk[u + w] : msk[u + w];
            acc[w] = fmaf(__uint_as_float(__float_as_uint(mv[w]) & m), vv[w], acc[w]);
        }
    }
    return quad_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
}

// acc[i][j] (+/-)= sum_{q0 <= q < q1} A[(a0+i)*LDA + q] * B[q*LDB + c0 + j]
template <typename T, int MT, bool SUB>
__device__ __forceinline__ void panel_mac(T (&acc)[4][MT], const T *__restrict__ A, int LDA,
                                          const T *__restrict__ B, int LDB, int a0, int c0, int q0,
                                          int q1) {
#pragma unroll 4
    for (int q = q0; q < q1; ++q) {
        T av[4], bv[MT];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = A[(a0 + i) * LDA + q];
        ld_row<T, MT>(B + q * LDB + c0, bv);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                if (SUB) acc[i][j] -= av[i] * bv[j];
                else acc[i][j] += av[i] * bv[j];
            }
    }
}

// Asynchronous global->shared copies (16-byte cp.async), used to prefetch the
// next factor tile of a chain while the current block step computes.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stages a KB x KB tile into shared memory rows of stride LDP (by default
// KB + 16/sizeof(T): one 16-byte pad per row), plus optionally KB diagonal values.
template <typename T, int KB, int LDP = KB + 16 / (int)sizeof(T)>
__device__ __forceinline__ void stage_tile(const T *__restrict__ src, T *dst, const T *__restrict__ dsrc,
                                           T *ddst) {
    constexpr int CH = 16 / sizeof(T), CPR = KB / CH, NT = Geo<KB>::NT;
    static_assert(LDP % CH == 0, "staged rows must stay 16-byte aligned");
    if constexpr ((KB * CPR) % NT == 0 && NT % CPR == 0) {
        // every thread copies the same chunk column of KB CPR / NT rows
        const int row0 = threadIdx.x / CPR, ch = threadIdx.x % CPR;
#pragma unroll
        for (int i = 0; i < KB * CPR / NT; ++i) {
            const int row = row0 + i * (NT / CPR);
            cp_async16(dst + row * LDP + ch * CH, src + row * KB + ch * CH);
        }
    } else {
        for (int e = threadIdx.x; e < KB * CPR; e += NT) {
            const int row = e / CPR, ch = e % CPR;
            cp_async16(dst + row * LDP + ch * CH, src + row * KB + ch * CH);
        }
    }
    if (dsrc)
        for (int e = threadIdx.x; e < CPR; e += Geo<KB>::NT) cp_async16(ddst + e * CH, dsrc + e * CH);
}

// Copies a KB x KB row-major tile from global memory into shared memory with
// row stride LDS (KB + 1 avoids bank conflicts on column reads).
template <typename T, int KB>
__device__ __forceinline__ void load_tile(const T *__restrict__ g, T *s, int LDS) {
    for (int e = threadIdx.x; e < KB * KB; e += Geo<KB>::NT) s[(e / KB) * LDS + (e % KB)] = g[e];
}

}  // namespace lrs
