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

// Tt (KB x m, ld LDM) holds b_J on entry; Yp holds y_{J-1} on entry and y_J on exit.
template <typename T, int KB, Split S>
__device__ __forceinline__ void fwd_step(const T *__restrict__ Ls, int LDS, T *Tt, T *Yp, int LDM,
                                         int m, bool first) {
    const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
    if (!first) {
        if (S == Split::COLS) {
            for (int c = q; c < m; c += 4) {
                T acc = Tt[a * LDM + c];
                for (int j = a; j < KB; ++j) acc -= Ls[a * LDS + j] * Yp[j * LDM + c];
                Tt[a * LDM + c] = acc;
            }
        } else {
            for (int c = 0; c < m; ++c) {
                T acc = T(0);
                for (int j = a + q; j < KB; j += 4) acc += Ls[a * LDS + j] * Yp[j * LDM + c];
                acc = quad_sum(acc);
                if (q == 0) Tt[a * LDM + c] -= acc;
            }
        }
    }
    __syncthreads();
    if (S == Split::COLS) {
        for (int c = q; c < m; c += 4) {
            T acc = Tt[a * LDM + c];
            for (int j = 0; j < a; ++j) acc += Ls[a * LDS + j] * Tt[j * LDM + c];
            Yp[a * LDM + c] = acc;
        }
    } else {
        for (int c = 0; c < m; ++c) {
            T acc = T(0);
            for (int j = q; j < a; j += 4) acc += Ls[a * LDS + j] * Tt[j * LDM + c];
            acc = quad_sum(acc);
            if (q == 0) Yp[a * LDM + c] = Tt[a * LDM + c] + acc;
        }
    }
    __syncthreads();
}

// Tt holds y_J on entry; Xn holds x_{J+1} on entry and x_J on exit.
template <typename T, int KB, Split S>
__device__ __forceinline__ void bwd_step(const T *__restrict__ Us, int LDS, const T *__restrict__ dsm,
                                         T *Tt, T *Xn, int LDM, int m, bool first) {
    const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
    if (S == Split::COLS) {
        for (int c = q; c < m; c += 4) {
            T acc = dsm[a] * Tt[a * LDM + c];
            if (!first)
                for (int j = 0; j <= a; ++j) acc -= Us[a * LDS + j] * Xn[j * LDM + c];
            Tt[a * LDM + c] = acc;
        }
    } else {
        for (int c = 0; c < m; ++c) {
            T acc = T(0);
            if (!first)
                for (int j = q; j <= a; j += 4) acc += Us[a * LDS + j] * Xn[j * LDM + c];
            acc = quad_sum(acc);
            if (q == 0) Tt[a * LDM + c] = dsm[a] * Tt[a * LDM + c] - acc;
        }
    }
    __syncthreads();
    if (S == Split::COLS) {
        for (int c = q; c < m; c += 4) {
            T acc = Tt[a * LDM + c];
            for (int j = a + 1; j < KB; ++j) acc += Us[a * LDS + j] * Tt[j * LDM + c];
            Xn[a * LDM + c] = acc;
        }
    } else {
        for (int c = 0; c < m; ++c) {
            T acc = T(0);
            for (int j = a + 1 + q; j < KB; j += 4) acc += Us[a * LDS + j] * Tt[j * LDM + c];
            acc = quad_sum(acc);
            if (q == 0) Xn[a * LDM + c] = Tt[a * LDM + c] + acc;
        }
    }
    __syncthreads();
}

// Transposed steps, for A^T = U^T L^T, with the same packed tiles.
//   forward  (U^T z = h): with z^_J = D_J z_J,
//            t = h_J - (D^{-1}U_{J-1,J})^T z^_{J-1};  z^_J = ((D^{-1}U_JJ)^{-1})^T t
//            (the caller applies z_J = D_J^{-1} z^_J after the sweep)
//   backward (L^T l = z): t = z_J - L_{J+1,J}^T l_{J+1};  l_J = (L_JJ^{-1})^T t
// Uprev = UT[J-1], Ucur = UT[J]; Lnext = LT[J+1], Lcur = LT[J].
template <typename T, int KB, Split S>
__device__ __forceinline__ void fwdT_step(const T *__restrict__ Uprev, const T *__restrict__ Ucur,
                                          int LDS, T *Tt, T *Zp, int LDM, int m, bool first) {
    const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
    if (!first) {
        if (S == Split::COLS) {
            for (int c = q; c < m; c += 4) {
                T acc = Tt[a * LDM + c];
                for (int j = a; j < KB; ++j) acc -= Uprev[j * LDS + a] * Zp[j * LDM + c];
                Tt[a * LDM + c] = acc;
            }
        } else {
            for (int c = 0; c < m; ++c) {
                T acc = T(0);
                for (int j = a + q; j < KB; j += 4) acc += Uprev[j * LDS + a] * Zp[j * LDM + c];
                acc = quad_sum(acc);
                if (q == 0) Tt[a * LDM + c] -= acc;
            }
        }
    }
    __syncthreads();
    if (S == Split::COLS) {
        for (int c = q; c < m; c += 4) {
            T acc = Tt[a * LDM + c];
            for (int j = 0; j < a; ++j) acc += Ucur[j * LDS + a] * Tt[j * LDM + c];
            Zp[a * LDM + c] = acc;
        }
    } else {
        for (int c = 0; c < m; ++c) {
            T acc = T(0);
            for (int j = q; j < a; j += 4) acc += Ucur[j * LDS + a] * Tt[j * LDM + c];
            acc = quad_sum(acc);
            if (q == 0) Zp[a * LDM + c] = Tt[a * LDM + c] + acc;
        }
    }
    __syncthreads();
}

template <typename T, int KB, Split S>
__device__ __forceinline__ void bwdT_step(const T *__restrict__ Lnext, const T *__restrict__ Lcur,
                                          int LDS, T *Tt, T *Lp, int LDM, int m, bool first) {
    const int a = threadIdx.x >> 2, q = threadIdx.x & 3;
    if (!first) {
        if (S == Split::COLS) {
            for (int c = q; c < m; c += 4) {
                T acc = Tt[a * LDM + c];
                for (int j = 0; j <= a; ++j) acc -= Lnext[j * LDS + a] * Lp[j * LDM + c];
                Tt[a * LDM + c] = acc;
            }
        } else {
            for (int c = 0; c < m; ++c) {
                T acc = T(0);
                for (int j = q; j <= a; j += 4) acc += Lnext[j * LDS + a] * Lp[j * LDM + c];
                acc = quad_sum(acc);
                if (q == 0) Tt[a * LDM + c] -= acc;
            }
        }
    }
    __syncthreads();
    if (S == Split::COLS) {
        for (int c = q; c < m; c += 4) {
            T acc = Tt[a * LDM + c];
            for (int j = a + 1; j < KB; ++j) acc += Lcur[j * LDS + a] * Tt[j * LDM + c];
            Lp[a * LDM + c] = acc;
        }
    } else {
        for (int c = 0; c < m; ++c) {
            T acc = T(0);
            for (int j = a + 1 + q; j < KB; j += 4) acc += Lcur[j * LDS + a] * Tt[j * LDM + c];
            acc = quad_sum(acc);
            if (q == 0) Lp[a * LDM + c] = Tt[a * LDM + c] + acc;
        }
    }
    __syncthreads();
}

// Copies a KB x KB row-major tile from global memory into shared memory with
// row stride LDS (KB + 1 avoids bank conflicts on column reads).
template <typename T, int KB>
__device__ __forceinline__ void load_tile(const T *__restrict__ g, T *s, int LDS) {
    for (int e = threadIdx.x; e < KB * KB; e += Geo<KB>::NT) s[(e / KB) * LDS + (e % KB)] = g[e];
}

}  // namespace lrs
