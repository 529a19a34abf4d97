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

template <typename T, int KB>
__global__ void __launch_bounds__(Geo<KB>::NT)
    k_band_lu(const double *__restrict__ band, int64_t ld, int k, Parts P, T *__restrict__ LT,
              T *__restrict__ UT, T *__restrict__ DS, int64_t *__restrict__ status) {
    using G = Geo<KB>;
    constexpr int W = G::W, TX = G::TX, TY = G::TY, RY = G::RY, RX = G::RX;
    constexpr int HY = RY / 2, HX = RX / 2;  // register index of the quadrant split
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *up = reinterpret_cast<T *>(smem_raw);
    T *dg = up + KB * KB;
    T *lo2 = dg + KB * KB;        // two lower tiles (ping-pong by block parity)
    T *rowb = lo2 + 2 * KB * KB;  // [2][W]
    T *colb = rowb + 2 * W;       // [2][W]

    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t b0 = P.boff[part];
    const int nb = (int)(P.boff[part + 1] - b0);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;

    T w[RY][RX];
    // column block 0: A_00 into the window, A_10 into lo2[0]
    load_colblock<T, KB>(band, ld, k, s, ni, 0, up, dg, lo2);
#pragma unroll
    for (int i = 0; i < HY; ++i)
#pragma unroll
        for (int j = 0; j < HX; ++j) w[i][j] = dg[(ty + TY * i) * KB + tx + TX * j];
    __syncthreads();

    for (int J = 0; J < nb; ++J) {
        const bool last = (J == nb - 1);
        T *lo_cur = lo2 + (J & 1) * KB * KB;        // A_{J+1,J}
        T *lo_next = lo2 + ((J + 1) & 1) * KB * KB;  // receives A_{J+2,J+1}
        if (!last) load_colblock<T, KB>(band, ld, k, s, ni, J + 1, up, dg, lo_next);
        // remaining quadrants of the window
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                if (i < HY && j < HX) continue;
                const int a = ty + TY * i, b = tx + TX * j;
                T v;
                if (last) v = (a == b) ? T(1) : T(0);
                else if (i < HY) v = up[a * KB + (b - KB)];
                else if (j < HX) v = lo_cur[(a - KB) * KB + b];
                else v = dg[(a - KB) * KB + (b - KB)];
                w[i][j] = v;
            }
        // publish pivot row / column 0
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                const int a = ty + TY * i, b = tx + TX * j;
                if (a == 0) rowb[b] = w[i][j];
                if (b == 0) colb[a] = w[i][j];
            }
        __syncthreads();

        for (int c = 0; c < KB; ++c) {
            const T *rb = rowb + (c & 1) * W;
            const T *cb = colb + (c & 1) * W;
            T *rn = rowb + ((c + 1) & 1) * W;
            T *cn = colb + ((c + 1) & 1) * W;
            const T piv = rb[c];
            const bool bad = (piv == T(0)) || !finite_val(piv);
            if (bad && threadIdx.x == 0)
                atomicMin((unsigned long long *)status, (unsigned long long)(s + (int64_t)J * KB + c));
            const T pinv = bad ? T(1) : T(1) / piv;
            T urow[RX];
#pragma unroll
            for (int j = 0; j < RX; ++j) urow[j] = rb[tx + TX * j];
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int a = ty + TY * i;
                if (a <= c) continue;
                const T l = cb[a] * pinv;
#pragma unroll
                for (int j = 0; j < RX; ++j) {
                    const int b = tx + TX * j;
                    if (b > c) w[i][j] -= l * urow[j];
                    else if (b == c) w[i][j] = l;
                }
            }
            if (c + 1 < KB) {
#pragma unroll
                for (int i = 0; i < RY; ++i)
#pragma unroll
                    for (int j = 0; j < RX; ++j) {
                        const int a = ty + TY * i, b = tx + TX * j;
                        if (a == c + 1 && b >= c + 1) rn[b] = w[i][j];
                        if (b == c + 1 && a > c + 1) cn[a] = w[i][j];
                    }
            }
            __syncthreads();
        }

        // write the factors of block J (and L_{J+1,J} of block J+1)
        const int64_t gJ = b0 + J;
        T *lt = LT + gJ * KB * KB;
        T *ut = UT + gJ * KB * KB;
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                const int a = ty + TY * i, b = tx + TX * j;
                const T v = w[i][j];
                if (i < HY && j < HX) {
                    if (a > b) lt[a * KB + b] = v;
                    else {
                        ut[a * KB + b] = v;
                        if (J == 0) lt[a * KB + b] = T(0);  // L_{0,-1} does not exist
                    }
                } else if (i < HY) {  // U_{J,J+1}, lower triangular
                    const int bb = b - KB;
                    if (bb < a) ut[a * KB + bb] = v;
                    else if (bb == a) DS[gJ * KB + a] = v;
                } else if (j < HX) {  // L_{J+1,J}, upper triangular
                    const int aa = a - KB;
                    if (!last && b >= aa) LT[(gJ + 1) * KB * KB + aa * KB + b] = v;
                }
            }
        // S_{J+1} becomes the next top-left quadrant
#pragma unroll
        for (int i = 0; i < HY; ++i)
#pragma unroll
            for (int j = 0; j < HX; ++j) w[i][j] = w[i + HY][j + HX];
        __syncthreads();
    }
}

// Per block: L^{-1} (unit lower), the unit upper inverse of D^{-1}U, D^{-1}
// and D^{-1} U_{J,J+1}.  Both inverses are built right-looking: for pivot j
// every entry below (L) or above (U) it is updated at once, one barrier per
// j; half of the CTA works on L, the other half on U.
template <typename T, int KB>
__global__ void __launch_bounds__(Geo<KB>::NT)
    k_prep_inverse(T *__restrict__ LT, T *__restrict__ UT, const T *__restrict__ DS,
                   T *__restrict__ DI) {
    constexpr int NT = Geo<KB>::NT, LD = KB + 1, HALF = NT / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *L = reinterpret_cast<T *>(smem_raw), *U = L + KB * LD, *XL = U + KB * LD, *XU = XL + KB * LD;
    const int64_t blk = blockIdx.x;
    T *lt = LT + blk * KB * KB;
    T *ut = UT + blk * KB * KB;
    for (int e = threadIdx.x; e < KB * KB; e += NT) {
        const int a = e / KB, b = e % KB;
        const T lv = lt[e], uv = ut[e];
        L[a * LD + b] = lv;
        U[a * LD + b] = uv;
        XL[a * LD + b] = (a == b) ? T(1) : T(0);
        XU[a * LD + b] = T(0);
    }
    __syncthreads();
    if (threadIdx.x < KB) XU[threadIdx.x * LD + threadIdx.x] = T(1) / U[threadIdx.x * LD + threadIdx.x];
    __syncthreads();
    // step j: XL[a][c] -= L[a][j] XL[j][c] for a > j, c <= j  (X = L^{-1}, unit lower)
    //         XU[a][c] -= U[a][j] XU[j][c] / U[a][a] for a < j', processed with j' = KB-1-j
    //         (X = U^{-1}, back substitution by columns from the right)
    const bool lower = threadIdx.x < HALF;
    const int t = lower ? threadIdx.x : threadIdx.x - HALF;
    for (int j = 0; j < KB; ++j) {
        if (lower) {
            const int rows = KB - 1 - j, cols = j + 1;
            for (int e = t; e < rows * cols; e += HALF) {
                const int a = j + 1 + e / cols, c = e % cols;
                XL[a * LD + c] -= L[a * LD + j] * XL[j * LD + c];
            }
        } else {
            const int jj = KB - 1 - j;           // finished row of U^{-1}
            const int rows = jj, cols = KB - jj;
            for (int e = t; e < rows * cols; e += HALF) {
                const int a = e / cols, c = jj + e % cols;
                XU[a * LD + c] -= U[a * LD + jj] * XU[jj * LD + c];
            }
        }
        __syncthreads();
        if (!lower) {
            // row KB-2-j of U^{-1} is complete once all pivots to its right are
            // applied; scale it by 1 / u_aa (the diagonal entry was set above)
            const int a = KB - 2 - j;
            if (a >= 0)
                for (int c = a + 1 + t; c < KB; c += HALF) XU[a * LD + c] /= U[a * LD + a];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < KB * KB; e += NT) {
        const int a = e / KB, b = e % KB;
        if (a > b) {
            lt[e] = XL[a * LD + b];                                  // L^{-1}
            ut[e] = U[a * LD + b] / U[a * LD + a];                   // D^{-1} U_{J,J+1}
        } else if (a < b) {
            ut[e] = XU[a * LD + b] * U[b * LD + b];                  // (D^{-1}U)^{-1}
        } else {
            ut[e] = DS[blk * KB + a] / U[a * LD + a];                // diagonal of D^{-1}U_{J,J+1}
        }
    }
    if (threadIdx.x < KB) DI[blk * KB + threadIdx.x] = T(1) / U[threadIdx.x * LD + threadIdx.x];
}

template <typename T, int KB>
static bool lu_impl(Ctx *c) {
    Parts P{c->off_d, c->boff_d, c->p};
    const size_t smem = (4 * KB * KB + 4 * Geo<KB>::W) * sizeof(T);
    auto kern = k_band_lu<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_LU, [&] {
        kern<<<c->p, Geo<KB>::NT, smem, c->stream>>>(c->band, c->ld, c->k, P, (T *)c->LT,
                                                   (T *)c->UT, (T *)c->DS, c->status);
    });
}

template <typename T, int KB>
static bool prep_impl(Ctx *c) {
    const size_t smem = 4 * KB * (KB + 1) * sizeof(T);
    auto kern = k_prep_inverse<T, KB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch(c, KID_PREP, [&] {
        kern<<<(unsigned)c->NB, Geo<KB>::NT, smem, c->stream>>>(
            (T *)c->LT, (T *)c->UT, (const T *)c->DS, (T *)c->DI);
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
