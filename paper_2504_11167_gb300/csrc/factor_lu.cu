// Banded LU of every partition A_i (the D-stage factorisation of paper
// section 2.1, "A = D S": D holds the diagonal blocks A_i, factorised
// independently; section 3.3 states each A_i is factorised by a direct
// solver).  No pivoting here; the matrices of this mode are diagonally
// dominant.
//
// Kernel k_band_lu: one CTA per partition walks the chain of nb_i block steps.
// Step J eliminates the KB columns of block J inside the 2KB x 2KB window
//     [ S_J         A_{J,J+1}   ]      S_J: diagonal block after the updates
//     [ A_{J+1,J}   A_{J+1,J+1} ]           of the previous steps
// (KB right-looking rank-1 steps).  Afterwards the window holds
//     [ L_JJ \ U_JJ     U_{J,J+1}   ]   L_JJ unit lower, U_JJ upper,
//     [ L_{J+1,J}       S_{J+1}     ]   U_{J,J+1} lower- and L_{J+1,J}
// upper-triangular (the band does not grow without pivoting), i.e. exactly
// the scalar band LU grouped in blocks.  The window lives in registers: the
// thread that owns entry (a, b) also owns (a + KB, b + KB), so S_{J+1} moves
// to the top-left quadrant by a register copy.  Pivot rows and columns are
// broadcast through ping-pong shared buffers, one barrier per column.
//
// Outputs per global block J (row-major KB x KB tiles):
//   LT[J]: strictly lower = L_JJ, upper incl. diagonal = L_{J,J-1}
//   UT[J]: upper incl. diagonal = U_JJ, strictly lower = U_{J,J+1} (its
//          diagonal goes to DS[J])
// k_prep_inverse then replaces L_JJ by L_JJ^{-1}, U_JJ by the unit upper
// inverse of diag(U_JJ)^{-1} U_JJ, scales U_{J,J+1} by diag(U_JJ)^{-1} and
// stores DI[J] = 1 / diag(U_JJ): the solve kernels then need only
// matrix-vector products per block step (no sequential substitution inside
// a block).
#include "common.cuh"
#include "internal.h"

namespace lrs {

// Stages band column block jc of a partition into three KB x KB tiles:
// up = A_{jc-1,jc}, dg = A_{jc,jc}, lo = A_{jc+1,jc} (partition-local, with
// the identity on padding rows).  Reads are coalesced: one diagonal of the
// band is KB consecutive doubles.
template <typename T, int KB>
__device__ void load_colblock(const double *__restrict__ band, int64_t ld, int k, int64_t s,
                              int64_t ni, int64_t jc, T *up, T *dg, T *lo) {
    constexpr int NT = Geo<KB>::NT;
    for (int e = threadIdx.x; e < KB * KB; e += NT) {
        up[e] = T(0);
        dg[e] = T(0);
        lo[e] = T(0);
    }
    __syncthreads();
    const int64_t col0 = jc * KB;
    const int nd = 2 * k + 1;
    for (int e = threadIdx.x; e < nd * KB; e += NT) {
        const int d = e / KB, b = e - (e / KB) * KB;
        const int64_t col = col0 + b;
        const int arel = b + d - k;  // row - col0
        const int64_t row = col0 + arel;
        T v;
        if (col >= ni) {
            if (d != k) continue;
            v = T(1);
        } else {
            if (row < 0 || row >= ni) continue;
            v = (T)band[(int64_t)d * ld + s + col];
        }
        if (arel < 0) up[(KB + arel) * KB + b] = v;
        else if (arel < KB) dg[arel * KB + b] = v;
        else lo[(arel - KB) * KB + b] = v;
    }
    __syncthreads();
}

// Register layout of the LU window: a TY x TX thread grid; in each of the three
// live quadrants (TL = S_J, TR = A_{J,J+1}, BL = A_{J+1,J}) a thread owns the
// entries (ty + TY*i, tx + TX*j), i < RY, j < RX.  The fourth quadrant (the
// next diagonal block) is not touched by the column steps: it is updated once
// per block step by the Schur product S_{J+1} = A_{J+1,J+1} - L_{J+1,J} U_{J,J+1}.
template <int KB> struct LuGeo {
    static constexpr int NT = 4 * KB;
    static constexpr int TX = (KB >= 16) ? 16 : 8;
    static constexpr int TY = NT / TX;
    static constexpr int RY = KB / TY;
    static constexpr int RX = KB / TX;
};

template <typename T, int KB>
__global__ void __launch_bounds__(4 * KB)
    k_band_lu(const double *__restrict__ band, int64_t ld, int k, Parts P, T *__restrict__ LT,
              T *__restrict__ UT, T *__restrict__ DS, int64_t *__restrict__ status) {
    using G = LuGeo<KB>;
    constexpr int TX = G::TX, TY = G::TY, RY = G::RY, RX = G::RX, LDT = KB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *up = reinterpret_cast<T *>(smem_raw);  // A_{J,J+1}
    T *dg = up + KB * KB;                     // A_{J+1,J+1}
    T *lo2 = dg + KB * KB;                    // A_{J+1,J}, two buffers by block parity
    T *Ys = lo2 + 2 * KB * KB;                // L_{J+1,J}  (KB x LDT)
    T *Zs = Ys + KB * LDT;                    // U_{J,J+1}  (KB x LDT)
    T *rowb = Zs + KB * LDT;                  // [2][2KB]: pivot row of [TL | TR]
    T *colb = rowb + 4 * KB;                  // [2][2KB]: pivot column of [TL ; BL]

    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;

    T tl[RY][RX], tr[RY][RX], bl[RY][RX];
    load_colblock<T, KB>(band, ld, k, s, ni, 0, up, dg, lo2);
#pragma unroll
    for (int i = 0; i < RY; ++i)
#pragma unroll
        for (int j = 0; j < RX; ++j) tl[i][j] = dg[(ty + TY * i) * KB + tx + TX * j];
    __syncthreads();

    for (int J = 0; J < nb; ++J) {
        const bool last = (J == nb - 1);
        const T *lo_cur = lo2 + (J & 1) * KB * KB;
        T *lo_next = lo2 + ((J + 1) & 1) * KB * KB;
        if (!last) load_colblock<T, KB>(band, ld, k, s, ni, J + 1, up, dg, lo_next);
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                const int a = ty + TY * i, b = tx + TX * j;
                tr[i][j] = last ? T(0) : up[a * KB + b];
                bl[i][j] = last ? T(0) : lo_cur[a * KB + b];
            }
        if (ty == 0)
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                rowb[tx + TX * j] = tl[0][j];
                rowb[KB + tx + TX * j] = tr[0][j];
            }
        if (tx == 0)
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                colb[ty + TY * i] = tl[i][0];
                colb[KB + ty + TY * i] = bl[i][0];
            }
        __syncthreads();

        for (int c = 0; c < KB; ++c) {
            const T *rb = rowb + (c & 1) * 2 * KB;
            const T *cb = colb + (c & 1) * 2 * KB;
            const T piv = rb[c];
            const bool bad = (piv == T(0)) || !finite_val(piv);
            if (bad && threadIdx.x == 0)
                atomicMin((unsigned long long *)status, (unsigned long long)(s + (int64_t)J * KB + c));
            const T pinv = bad ? T(1) : T(1) / piv;
            T lt[RY], lb[RY], ut[RX], ur[RX];
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int a = ty + TY * i;
                lt[i] = (a > c) ? cb[a] * pinv : T(0);
                lb[i] = cb[KB + a] * pinv;
            }
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                const int b = tx + TX * j;
                ut[j] = (b > c) ? rb[b] : T(0);
                ur[j] = rb[KB + b];
            }
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int j = 0; j < RX; ++j) {
                    tl[i][j] -= lt[i] * ut[j];
                    tr[i][j] -= lt[i] * ur[j];
                    bl[i][j] -= lb[i] * ut[j];
                }
            if (tx == c % TX) {  // this thread holds column c: store the multipliers
                const int jc = c / TX;
#pragma unroll
                for (int j = 0; j < RX; ++j)
                    if (j == jc)
#pragma unroll
                        for (int i = 0; i < RY; ++i) {
                            if (ty + TY * i > c) tl[i][j] = lt[i];
                            bl[i][j] = lb[i];
                        }
            }
            if (c + 1 < KB) {
                const int r1 = c + 1;
                T *rn = rowb + (r1 & 1) * 2 * KB;
                T *cn = colb + (r1 & 1) * 2 * KB;
                if (ty == r1 % TY) {
                    const int ir = r1 / TY;
#pragma unroll
                    for (int i = 0; i < RY; ++i)
                        if (i == ir)
#pragma unroll
                            for (int j = 0; j < RX; ++j) {
                                rn[tx + TX * j] = tl[i][j];
                                rn[KB + tx + TX * j] = tr[i][j];
                            }
                }
                if (tx == r1 % TX) {
                    const int jr = r1 / TX;
#pragma unroll
                    for (int j = 0; j < RX; ++j)
                        if (j == jr)
#pragma unroll
                            for (int i = 0; i < RY; ++i) {
                                cn[ty + TY * i] = tl[i][j];
                                cn[KB + ty + TY * i] = bl[i][j];
                            }
                }
            }
            __syncthreads();
        }

        // factors of block J, and L_{J+1,J} into block J+1's tile
        const int64_t gJ = b0 + J;
        T *lt_g = LT + gJ * KB * KB;
        T *ut_g = UT + gJ * KB * KB;
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                const int a = ty + TY * i, b = tx + TX * j;
                if (a > b) lt_g[a * KB + b] = tl[i][j];
                else {
                    ut_g[a * KB + b] = tl[i][j];
                    if (J == 0) lt_g[a * KB + b] = T(0);  // L_{0,-1} does not exist
                }
                if (b < a) ut_g[a * KB + b] = tr[i][j];
                else if (b == a) DS[gJ * KB + a] = tr[i][j];
                if (!last && b >= a) LT[(gJ + 1) * KB * KB + a * KB + b] = bl[i][j];
                if (!last) {
                    Ys[a * LDT + b] = bl[i][j];
                    Zs[a * LDT + b] = tr[i][j];
                }
            }
        if (last) break;
        __syncthreads();
        // S_{J+1} = A_{J+1,J+1} - L_{J+1,J} U_{J,J+1}; L_{J+1,J} is upper and
        // U_{J,J+1} lower triangular, so only q >= max(a, b) contributes
        T acc[RY][RX];
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) acc[i][j] = dg[(ty + TY * i) * KB + tx + TX * j];
        const int q0 = (ty > tx) ? ty : tx;
        for (int q = q0; q < KB; ++q) {
            T yv[RY], zv[RX];
#pragma unroll
            for (int i = 0; i < RY; ++i) yv[i] = Ys[(ty + TY * i) * LDT + q];
#pragma unroll
            for (int j = 0; j < RX; ++j) zv[j] = Zs[q * LDT + tx + TX * j];
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int j = 0; j < RX; ++j) acc[i][j] -= yv[i] * zv[j];
        }
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) tl[i][j] = acc[i][j];
        __syncthreads();
    }
}

// Per block: L^{-1} (unit lower), the unit upper inverse of D^{-1}U, D^{-1}
// and D^{-1} U_{J,J+1}.  Each inverse is built column by column by plain
// substitution; a thread owns columns c and KB-1-c (equal total work), so no
// barrier is needed: every value a thread reads is its own earlier result or
// input.  Results are kept transposed in the unused triangle of the same
// shared tile.  A CTA of 128 threads serves 128/KB blocks (one warp, or part
// of one, per triangular factor).
template <typename T, int KB>
__global__ void __launch_bounds__(128)
    k_prep_inverse(T *__restrict__ LT, T *__restrict__ UT, const T *__restrict__ DS,
                   T *__restrict__ DI, int64_t NB) {
    constexpr int LD = KB + 1, TPM = KB / 2, BPC = 128 / KB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tiles = reinterpret_cast<T *>(smem_raw);  // [BPC][2][KB x LD]
    T *dinv = tiles + BPC * 2 * KB * LD;          // [BPC][KB]
    const int64_t blk0 = (int64_t)blockIdx.x * BPC;
    for (int e = threadIdx.x; e < BPC * KB * KB; e += 128) {
        const int bb = e / (KB * KB), rem = e % (KB * KB), a = rem / KB, b = rem % KB;
        const int64_t blk = blk0 + bb;
        if (blk >= NB) continue;
        T *Ls = tiles + (bb * 2 + 0) * KB * LD, *Us = tiles + (bb * 2 + 1) * KB * LD;
        Ls[a * LD + b] = (a > b) ? LT[blk * KB * KB + rem] : T(0);
        const T u = UT[blk * KB * KB + rem];
        Us[a * LD + b] = (a <= b) ? u : T(0);
        if (a == b) dinv[bb * KB + a] = T(1) / u;
    }
    __syncthreads();
    const int bb = threadIdx.x / (2 * TPM), role = (threadIdx.x / TPM) & 1, t = threadIdx.x % TPM;
    if (blk0 + bb < NB) {
        T *S = tiles + (bb * 2 + role) * KB * LD;
        const T *dv = dinv + bb * KB;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int col = h ? KB - 1 - t : t;
            if (role == 0) {
                // X = L^{-1}: X[a][col] = -(L[a][col] + sum_{col<j<a} L[a][j] X[j][col]),
                // stored at S[col][a] (upper triangle)
                for (int a = col + 1; a < KB; ++a) {
                    T s0 = S[a * LD + col], s1 = T(0);
                    int j = col + 1;
                    for (; j + 1 < a; j += 2) {
                        s0 += S[a * LD + j] * S[col * LD + j];
                        s1 += S[a * LD + j + 1] * S[col * LD + j + 1];
                    }
                    if (j < a) s0 += S[a * LD + j] * S[col * LD + j];
                    S[col * LD + a] = -(s0 + s1);
                }
            } else {
                // X = U^{-1}: X[col][col] = 1/u, X[a][col] = -(sum_{a<j<=col} U[a][j] X[j][col]) / U[a][a],
                // stored at S[col][a] (lower triangle); the diagonal entry lives in dinv
                for (int a = col - 1; a >= 0; --a) {
                    T s0 = S[a * LD + col] * dv[col], s1 = T(0);
                    int j = a + 1;
                    for (; j + 1 < col; j += 2) {
                        s0 += S[a * LD + j] * S[col * LD + j];
                        s1 += S[a * LD + j + 1] * S[col * LD + j + 1];
                    }
                    if (j < col) s0 += S[a * LD + j] * S[col * LD + j];
                    S[col * LD + a] = -(s0 + s1) * dv[a];
                }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BPC * KB * KB; e += 128) {
        const int bb2 = e / (KB * KB), rem = e % (KB * KB), a = rem / KB, b = rem % KB;
        const int64_t blk = blk0 + bb2;
        if (blk >= NB) continue;
        const T *Ls = tiles + (bb2 * 2 + 0) * KB * LD, *Us = tiles + (bb2 * 2 + 1) * KB * LD;
        const T *dv = dinv + bb2 * KB;
        if (a > b) {
            LT[blk * KB * KB + rem] = Ls[b * LD + a];                        // L^{-1}
            UT[blk * KB * KB + rem] = UT[blk * KB * KB + rem] * dv[a];       // D^{-1} U_{J,J+1}
        } else if (a < b) {
            UT[blk * KB * KB + rem] = Us[b * LD + a] / dv[b];                // (D^{-1}U)^{-1} = U^{-1} D
        } else {
            UT[blk * KB * KB + rem] = DS[blk * KB + a] * dv[a];              // diagonal of D^{-1}U_{J,J+1}
            DI[blk * KB + a] = dv[a];
        }
    }
}

template <typename T, int KB>
static bool lu_impl(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (4 * KB * KB + 2 * KB * (KB + 1) + 8 * KB) * sizeof(T);
    auto kern = k_band_lu<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_LU, [&] {
        kern<<<c->p, Geo<KB>::NT, smem, c->stream>>>(c->band, c->ld, c->k, P, (T *)c->LT,
                                                   (T *)c->UT, (T *)c->DS, c->status);
    });
}

template <typename T, int KB>
static bool prep_impl(Ctx *c) {
    constexpr int BPC = 128 / KB;
    const size_t smem = (BPC * 2 * KB * (KB + 1) + BPC * KB) * sizeof(T);
    auto kern = k_prep_inverse<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)((c->NB + BPC - 1) / BPC);
    return launch(c, KID_PREP, [&] {
        kern<<<grid, 128, smem, c->stream>>>((T *)c->LT, (T *)c->UT, (const T *)c->DS, (T *)c->DI, c->NB);
    });
}

#define LRS_DISPATCH(FN)                                             \
    template <typename T>                                            \
    static bool FN##_kb(Ctx *c) {                                    \
        switch (c->KB) {                                             \
            case 8: return FN<T, 8>(c);                              \
            case 16: return FN<T, 16>(c);                            \
            case 32: return FN<T, 32>(c);                            \
            default: return FN<T, 64>(c);                            \
        }                                                            \
    }

LRS_DISPATCH(lu_impl)
LRS_DISPATCH(prep_impl)

bool run_band_lu(Ctx *c) { return c->fp64 ? lu_impl_kb<double>(c) : lu_impl_kb<float>(c); }
bool run_prep(Ctx *c) { return c->fp64 ? prep_impl_kb<double>(c) : prep_impl_kb<float>(c); }

}  // namespace lrs
