// Wide bands, 64 < k <= 1024 (the 2-D convection-diffusion systems of
// section 4, half-bandwidth = grid width).
//
// Every partition A_i is cut into blocks of W = 64 ceil(k/64) >= k rows, so it
// is block tridiagonal with W x W blocks; partitions are padded to NBW blocks
// with identity rows.  The block operations are dense contractions of order W
// (up to 1024), batched over the p partitions.  They run on the 5th-generation
// tensor cores (tc_gemm.cu; TF32 operands, or BF16 operands for
// LRSPIKE_MIXED_BF16, FP32 accumulation) or, in the FP64 and FP32 modes, as
// SIMT GEMMs in the working precision (k_simt_gemm):
//
//   factor, block step J (all partitions at once):
//     S_J = A_JJ - Y_{J-1} Z_{J-1};  S_J = L U with L^{-1}, U^{-1} by recursive
//     halving (64 x 64 base blocks in k_lu_inv64);
//     Z_J = L_JJ^{-1} A_{J,J+1} (= U_{J,J+1}),  Y_J = A_{J+1,J} U_JJ^{-1} (= L_{J+1,J})
//   compression: the randomized SVD the paper uses for wide bands (section
//     3.1, Halko-Martinsson-Tropp proto-algorithm) on each spike
//     T = A_i^{-1}[0; B_i] (eq. 'Veqn'; W_i = A_i^{-1}[C_i; 0] likewise),
//     never formed: its products are block solves with the factors on panels
//     of 2 lp columns, T X = A_i^{-1}[0; B_i X], T^T Q = B_i^T (A_i^{-T} Q)_bottom;
//       Y = T Omega;  Q = orth(Y);  q times: Y = T (T^T Q), Q = orth(Y);
//       B^T = T^T Q;  B B^T = U_B diag(sigma^2) U_B^T (cyclic Jacobi);
//       u = Q U_B,r,  P = U_B,r^T B = sigma_r V_r^T.
//     orth() is shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto
//     and Yanagisawa, 2020): three passes G = Y^T Y, G (+ s I) = R^T R,
//     Y <- Y R^{-1}, the first with the shift s = 11 (m l + l(l+1)) u ||Y||_F^2;
//     it spans the same subspace as the Householder QR of the oracle.
//   D-stage and its transpose: one cluster of CTAs per partition walks both
//     block recurrences (k_wide_dstage), reading only the nonzero triangles of
//     the factor tiles.
//
// Layouts: W x W tiles [p][NBW][W x W]; panels [p][PS x 2 lp] column-major
// with PS = NBW W rows (leading dimension PS).  A matrix that is a left factor of a
// tensor-core product is also kept row-major in the operand type, a right
// factor column-major in the operand type (K-contiguous operands for the MMA);
// the epilogue of the product that makes a matrix writes those copies.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrs {

namespace {

namespace cg = cooperative_groups;

constexpr int VP = 16;  // columns of the vector panels (max nrhs)

// A batch of matrices in the layouts products read; element (a, b) of entry i:
//   f    working precision, column-major  f[a + b ld + i s]
//   fr   working precision, row-major     fr[b + a ldr + i sr]
//   oc   operand type, column-major       oc[a + b ld + i s]
//   orow operand type, row-major          orow[b + a ldr + i sr]
// Absent layouts are NULL.  In TF32 mode the operand type is the working type
// and oc / orow alias f / fr.
struct WMat {
    void *f = nullptr, *fr = nullptr, *oc = nullptr, *orow = nullptr;
    int64_t ld = 0, s = 0, ldr = 0, sr = 0;
};

inline void *elem(void *base, int64_t e, size_t sz) {
    return base ? static_cast<void *>(static_cast<char *>(base) + e * (int64_t)sz) : nullptr;
}

WMat view(const Ctx *c, const WMat &m, int64_t a0, int64_t b0) {
    WMat v = m;
    v.f = elem(m.f, a0 + b0 * m.ld, c->tsize);
    v.oc = elem(m.oc, a0 + b0 * m.ld, c->osize);
    v.fr = elem(m.fr, b0 + a0 * m.ldr, c->tsize);
    v.orow = elem(m.orow, b0 + a0 * m.ldr, c->osize);
    return v;
}

WMat square(void *const (&arr)[4], int64_t W, int64_t stride) {
    WMat m;
    m.f = arr[0];
    m.fr = arr[1];
    m.oc = arr[2];
    m.orow = arr[3];
    m.ld = m.ldr = W;
    m.s = m.sr = stride;
    return m;
}

// ---------------------------------------------------------------------------
// SIMT GEMM (FP64 / FP32 modes):  C = alpha A' B'^T + beta C over the batch,
// A'(m, k) = A[m am + k ak + b as], B'(n, k) = B[n bn + k bk + b bs];
// C column-major (ldc, sc) and optionally a row-major copy Cr (ldr, sr).
// 64 x 64 tile per CTA, 16-deep K slabs in shared memory, 4 x 4 per thread.
template <typename T>
__global__ void __launch_bounds__(256)
    k_simt_gemm(int M, int N, int K, T alpha, T beta, const T *__restrict__ A, int64_t am, int64_t ak, int64_t as,
                const T *__restrict__ B, int64_t bn, int64_t bk, int64_t bs, T *C, int64_t ldc, int64_t sc,
                T *Cr, int64_t ldr, int64_t sr) {
    __shared__ T As[16][65], Bs[16][65];
    const int b = blockIdx.z, m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    A += b * as;
    B += b * bs;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const bool a1 = (ak == 1), b1 = (bk == 1);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int kk = a1 ? (e & 15) : (e >> 6), mm = a1 ? (e >> 4) : (e & 63);
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[gm * am + gk * ak] : T(0);
            kk = b1 ? (e & 15) : (e >> 6);
            const int nn = b1 ? (e >> 4) : (e & 63);
            const int gn = n0 + nn;
            gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < K) ? B[gn * bn + gk * bk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    // the reads of C (beta != 0) all before the first write of C
    T cin[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            cin[i][j] = (beta != T(0) && m < M && n < N) ? C[(int64_t)b * sc + m + (int64_t)n * ldc] : T(0);
        }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            if (m < M && n < N) {
                T v = alpha * acc[i][j];
                const int64_t ci = (int64_t)b * sc + m + (int64_t)n * ldc;
                if (beta != T(0)) v = fma(beta, cin[i][j], v);
                if (C) C[ci] = v;
                if (Cr) Cr[(int64_t)b * sr + n + (int64_t)m * ldr] = v;
            }
        }
}

// C = alpha op(X) op(Y) + beta C over the batch; op(X) is M x K, op(Y) K x N.
// rsplit / rss: the row-major operand copy of C splits its columns into
// blocks of rsplit placed rss apart (0 = no split).
bool gemm(Ctx *c, int M, int N, int K, double alpha, const WMat &X, bool tx, const WMat &Y, bool ty, double beta,
          const WMat &C, int batch, int rsplit = 0, int64_t rss = 0) {
    if (M <= 0 || N <= 0 || batch <= 0) return true;
    if (c->gpath == 0) {
        const int64_t am = tx ? X.ld : 1, ak = tx ? 1 : X.ld;
        const int64_t bn = ty ? 1 : Y.ld, bk = ty ? Y.ld : 1;
        const dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)batch);
        return launch(c, KID_WIDE_GEMM, [&] {
            if (c->fp64)
                k_simt_gemm<double><<<grid, 256, 0, c->stream>>>(
                    M, N, K, alpha, beta, (const double *)X.f, am, ak, X.s, (const double *)Y.f, bn, bk, Y.s,
                    (double *)C.f, C.ld, C.s, (double *)C.fr, C.ldr, C.sr);
            else
                k_simt_gemm<float><<<grid, 256, 0, c->stream>>>(
                    M, N, K, (float)alpha, (float)beta, (const float *)X.f, am, ak, X.s, (const float *)Y.f, bn, bk,
                    Y.s, (float *)C.f, C.ld, C.s, (float *)C.fr, C.ldr, C.sr);
        });
    }
    GemmOperand A, B;
    if (!tx) A = {X.orow, X.ldr, X.sr};
    else A = {X.oc, X.ld, X.s};
    if (!ty) B = {Y.oc, Y.ld, Y.s};
    else B = {Y.orow, Y.ldr, Y.sr};
    if (!A.p || !B.p) {
        c->err = "wide-band product: an operand layout is missing";
        return false;
    }
    GemmOutput o;
    o.f = static_cast<float *>(C.f);
    o.ldf = C.ld;
    o.sf = C.s;
    o.row = C.orow;
    o.ldr = C.ldr;
    o.sr = C.sr;
    o.rsplit = rsplit;
    o.rss = rss;
    o.col = (C.oc != C.f) ? C.oc : nullptr;
    o.ldc = C.ld;
    o.sc = C.s;
    o.frow = (C.fr != C.orow) ? static_cast<float *>(C.fr) : nullptr;
    std::string err;
    bool ok = true;
    const bool launched = launch(c, KID_WIDE_TC, [&] {
        ok = tc_gemm(c->stream, c->gpath == 2, M, N, K, batch, (float)alpha, A, B, (float)beta, o, c->gemm_err, &err);
    });
    if (!ok) {
        c->err = err;
        return false;
    }
    return launched;
}

// ---------------------------------------------------------------------------
template <typename O>
__device__ __forceinline__ O cvtd(double v) {
    if constexpr (sizeof(O) == 2) return __float2bfloat16_rn((float)v);
    else return (O)v;
}

// A_JJ (S), A_{J,J+1} (B), A_{J+1,J} (C) of every partition, W x W, in the
// layouts their products read (null pointers are skipped).  One CTA per
// 32 x 32 tile: it reads the tile along band diagonals (consecutive columns
// are consecutive band addresses) and writes it column by column (column-major
// layouts) and row by row (row-major layouts).
template <typename T, typename O>
__global__ void __launch_bounds__(256)
    k_wide_gather(const double *__restrict__ band, int64_t ld, int k, Parts P, int W, int J, T *Sf, T *Sfr, O *Soc,
                  O *Sor, T *Bf, O *Boc, T *Cf, O *Cor) {
    __shared__ double tile[32][33];
    const int which = blockIdx.z % 3, part = blockIdx.z / 3;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int64_t rb = (which == 2) ? (int64_t)(J + 1) * W : (int64_t)J * W;  // first local row
    const int64_t cb = (which == 1) ? (int64_t)(J + 1) * W : (int64_t)J * W;  // first local column
    for (int e = threadIdx.x; e < 63 * 32; e += 256) {
        const int dd = e / 32 - 31, b = e % 32, a = b + dd;
        if (a < 0 || a >= 32) continue;
        const int64_t lr = rb + a0 + a, lc = cb + b0 + b;
        double v = 0.0;
        if (lr < ni && lc < ni) {
            const int64_t d = k + lr - lc;
            if (d >= 0 && d <= 2 * k) v = band[d * ld + s + lc];
        } else if (which == 0 && lr == lc) {
            v = 1.0;  // padding rows carry the identity
        }
        tile[a][b] = v;
    }
    __syncthreads();
    const int64_t off = (int64_t)part * W * W;
    T *f = which == 0 ? Sf : which == 1 ? Bf : Cf;
    T *fr = which == 0 ? Sfr : nullptr;
    O *oc = which == 0 ? Soc : which == 1 ? Boc : nullptr;
    O *orow = which == 0 ? Sor : which == 2 ? Cor : nullptr;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int b = ty; b < 32; b += 8) {
        const int64_t ci = off + (int64_t)(b0 + b) * W + a0 + tx;   // column-major: column b0+b, row a0+tx
        const int64_t ri = off + (int64_t)(a0 + b) * W + b0 + tx;   // row-major: row a0+b, column b0+tx
        if (f) f[ci] = (T)tile[tx][b];
        if (oc) oc[ci] = cvtd<O>(tile[tx][b]);
        if (fr) fr[ri] = (T)tile[b][tx];
        if (orow) orow[ri] = cvtd<O>(tile[b][tx]);
    }
}

// Layout copies of the n x n leading view of each partition's matrix (f,
// leading dimension ld, stride s) into fr / oc / orow (nullable).
template <typename T, typename O>
__global__ void k_wide_layouts(const T *__restrict__ f, int n, int64_t ld, int64_t s, T *fr, O *oc, O *orow) {
    const int part = blockIdx.y;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int a = e % n, b = e / n;
        const T v = f[(int64_t)part * s + a + (int64_t)b * ld];
        if (oc) oc[(int64_t)part * s + a + (int64_t)b * ld] = cvtd<O>((double)v);
        if (fr) fr[(int64_t)part * s + b + (int64_t)a * ld] = v;
        if (orow) orow[(int64_t)part * s + b + (int64_t)a * ld] = cvtd<O>((double)v);
    }
}

// Spike right-hand sides on the zeroed panel X [PS x 2W]: [0; B_i] in columns
// 0..k-1 (rows n_i-k..n_i-1) and [C_i; 0] in columns W..W+k-1 (rows 0..k-1);
// Xc (nullable) is the operand-type copy.
template <typename T, typename O>
__global__ void k_wide_spike_rhs(const double *__restrict__ band, int64_t ld, int k, Parts P, int W, int64_t PS,
                                 T *__restrict__ X, O *Xc) {
    const int part = blockIdx.x;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t base = (int64_t)part * PS * 2 * W;
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int a = (int)(e % k), b = (int)(e / k);
        if (part < P.p - 1) {  // B_i[a][b] = A[s+n_i-k+a][s+n_i+b], nonzero for b <= a
            const int64_t sn = s + ni;
            const double v = (b <= a) ? band[(int64_t)(a - b) * ld + sn + b] : 0.0;
            const int64_t xi = base + (int64_t)b * PS + ni - k + a;
            X[xi] = (T)v;
            if (Xc) Xc[xi] = cvtd<O>(v);
        }
        if (part > 0) {  // C_i[a][b] = A[s+a][s-k+b], nonzero for a <= b
            const double v = (a <= b) ? band[(int64_t)(2 * k + a - b) * ld + s - k + b] : 0.0;
            const int64_t xi = base + (int64_t)(W + b) * PS + a;
            X[xi] = (T)v;
            if (Xc) Xc[xi] = cvtd<O>(v);
        }
    }
}

// Coupling blocks as W x W tiles, b = 2 i + side (zero beyond k and where the
// block does not exist): side 0 B_i[a][b] = A[s_{i+1}-k+a][s_{i+1}+b]
// (nonzero for b <= a, i < p-1), side 1 C_i[a][b] = A[s_i+a][s_i-k+b]
// (nonzero for a <= b, i > 0).  Threads walk the band along its diagonals
// (consecutive threads, consecutive band addresses); layouts as WMat.
template <typename T, typename O>
__global__ void k_wide_couple_gather(const double *__restrict__ band, int64_t ld, int k, Parts P, int W, T *f,
                                     O *oc, O *orow) {
    const int b = blockIdx.y, part = b / 2, side = b % 2;
    const bool live = side == 0 ? (part < P.p - 1) : (part > 0);
    const int64_t tile = (int64_t)b * W * W;
    const int64_t s = P.off[part], sn = P.off[part + 1];
    // entry e: diagonal d = e / k (0..k-1), position q = e % k
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(e / k), q = (int)(e % k);
        int a, c;
        double v = 0.0;
        if (side == 0) {  // a - c = d >= 0
            c = q;
            a = q + d;
            if (a < k && live) v = band[(int64_t)d * ld + sn + c];
        } else {          // c - a = d >= 0
            a = q;
            c = q + d;
            if (c < k && live) v = band[(int64_t)(2 * k - d) * ld + s - k + c];
        }
        if (a >= k || c >= k) continue;
        if (f) f[tile + a + (int64_t)c * W] = (T)v;
        if (oc) oc[tile + a + (int64_t)c * W] = cvtd<O>(v);
        if (orow) orow[tile + c + (int64_t)a * W] = cvtd<O>(v);
    }
}

// Tips of the 2 lp-column panels [p][PS x 2lp] as [2p][W x lp] tiles: side 0
// the last k rows of the first lp columns, side 1 the first k rows of the
// last lp columns (rows k..W-1 zero).
template <typename T, typename O>
__global__ void k_tips_gather(const T *__restrict__ Pf, Parts P, int k, int W, int64_t PS, int lp, T *Xf, O *Xoc) {
    const int b = blockIdx.y, part = b / 2, side = b % 2;
    const int64_t ni = P.off[part + 1] - P.off[part];
    const T *pan = Pf + (int64_t)part * PS * 2 * lp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < W * lp; e += gridDim.x * blockDim.x) {
        const int a = e % W, j = e / W;
        T v = T(0);
        if (a < k) v = side == 0 ? pan[(ni - k + a) + (int64_t)j * PS] : pan[a + (int64_t)(lp + j) * PS];
        Xf[(int64_t)b * W * lp + e] = v;
        if (Xoc) Xoc[(int64_t)b * W * lp + e] = cvtd<O>((double)v);
    }
}

// The reverse: [2p][W x lp] (first k rows) into the zeroed panels, side 0 at
// rows n_i-k.. of the first lp columns, side 1 at rows 0.. of the last lp
// (only where the spike exists).
template <typename T, typename O>
__global__ void k_tips_scatter(const T *__restrict__ Xf, Parts P, int k, int W, int64_t PS, int lp, T *Pf, O *Poc) {
    const int b = blockIdx.y, part = b / 2, side = b % 2;
    if (side == 0 ? part >= P.p - 1 : part == 0) return;
    const int64_t ni = P.off[part + 1] - P.off[part];
    const int64_t base = (int64_t)part * PS * 2 * lp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * lp; e += gridDim.x * blockDim.x) {
        const int a = e % k, j = e / k;
        const T v = Xf[(int64_t)b * W * lp + a + (int64_t)j * W];
        const int64_t pi = base + (side == 0 ? (ni - k + a) + (int64_t)j * PS : a + (int64_t)(lp + j) * PS);
        Pf[pi] = v;
        if (Poc) Poc[pi] = cvtd<O>((double)v);
    }
}

// SplitMix64 (Steele, Lea, Flood 2014): output i of the generator started at seed.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Gaussian sketches Omega_b (W x lp, column-major), b = 2 i + side: entry
// (a, j), a < k, j < ell, is the Box-Muller normal of SplitMix64 outputs 2c,
// 2c+1 at c = a ell + j with seed + b; zero elsewhere.
template <typename O>
__global__ void k_wide_sketch(O *__restrict__ Om, int W, int k, int ell, int lp, unsigned long long seed,
                              int nmat) {
    const int64_t per = (int64_t)W * lp, total = per * nmat;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const int64_t rem = e % per;
        const int j = (int)(rem / W), a = (int)(rem % W);
        double v = 0.0;
        if (a < k && j < ell) {
            const unsigned long long cidx = (unsigned long long)a * ell + j, sd = seed + (unsigned long long)b;
            const double u1 = ((double)(splitmix64(sd, 2 * cidx) >> 11) + 0.5) * 0x1p-53;
            const double u2 = (double)(splitmix64(sd, 2 * cidx + 1) >> 11) * 0x1p-53;
            v = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
        }
        Om[e] = cvtd<O>(v);
    }
}

// Gram matrices Y_m^T Y_m of the 2p sketch iterates (Y_m column-major,
// PS x lp, leading dimension PS) split over row chunks so that every SM has
// work: CTA (tile, c, m) forms the 64 x 64 output tile of the partial Gram of
// rows [c GRAM_ROWS, (c+1) GRAM_ROWS) (16-row slabs in shared memory, 4 x 4
// per thread); k_gram_sum adds the chunks in a fixed order in FP64.
constexpr int GRAM_ROWS = 1024;
inline int gram_chunks(int64_t PS) { return (int)((PS + GRAM_ROWS - 1) / GRAM_ROWS); }

template <typename T>
__global__ void __launch_bounds__(256)
    k_gram_part(const T *__restrict__ Y, int lp, int64_t PS, int64_t sY, T *__restrict__ part) {
    __shared__ T As[16][65], Bs[16][65];
    const int tiles = (lp + 63) / 64;
    const int m0 = (blockIdx.x % tiles) * 64, n0 = (blockIdx.x / tiles) * 64, ch = blockIdx.y, mat = blockIdx.z;
    const T *Ym = Y + (int64_t)mat * sY;
    const int64_t r0 = (int64_t)ch * GRAM_ROWS, r1 = min(PS, r0 + GRAM_ROWS);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int64_t k0 = r0; k0 < r1; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int kk = e & 15, mm = e >> 4;
            const int64_t gk = k0 + kk;
            As[kk][mm] = (gk < r1 && m0 + mm < lp) ? Ym[gk + (int64_t)(m0 + mm) * PS] : T(0);
            Bs[kk][mm] = (gk < r1 && n0 + mm < lp) ? Ym[gk + (int64_t)(n0 + mm) * PS] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    T *out = part + ((int64_t)mat * gridDim.y + ch) * lp * lp;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = m0 + tx + 16 * i, b = n0 + ty + 16 * j;
            if (a < lp && b < lp) out[a + (int64_t)b * lp] = acc[i][j];
        }
}

template <typename T>
__global__ void k_gram_sum(const T *__restrict__ part, int nch, int64_t sG, int64_t count, double *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mat = e / sG, idx = e % sG;
        const T *src = part + mat * nch * sG + idx;
        double s = 0.0;
        for (int c = 0; c < nch; ++c) s += (double)src[(int64_t)c * sG];
        out[e] = s;
    }
}

template <typename T>
__global__ void k_to_f64(const T *__restrict__ in, double *__restrict__ out, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (double)in[e];
}

template <typename T, typename O>
__global__ void k_to_op(const T *__restrict__ in, O *__restrict__ out, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = cvtd<O>((double)in[e]);
}

// One CholeskyQR pass on the n x n leading block of each Gram matrix G_b
// (FP64, lp x lp column-major): G (+ s I) = R^T R by right-looking Cholesky,
// then R^{-1} (upper triangular, in place, column by column) written as
// Rinv_b (working precision, lp x lp column-major, zero outside).  The shift
// (shifted = 1) is s = 11 (rows n + n (n+1)) u trace(G).  A pivot at or below
// n u max_j G_jj (after the shift) marks a direction that the columns already
// span: its row of R is set to the unit row and its row and column of R^{-1}
// to zero, so that column of Q = Y R^{-1} is zero and no other column uses it.
template <typename T>
__global__ void __launch_bounds__(256)
    k_chol_inv(const double *__restrict__ G, int lp, int n, int64_t rows, double u, int shifted, T *__restrict__ Rinv) {
    extern __shared__ double csm[];
    const int LD = n + 1;
    double *A = csm, *tmp = A + n * LD;
    __shared__ int dropped[128];
    __shared__ double s_shift, s_maxd;
    const int b = blockIdx.x;
    const double *g = G + (int64_t)b * lp * lp;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        A[i * LD + j] = g[i + (int64_t)j * lp];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) tr += A[i * LD + i];
        s_shift = shifted ? 11.0 * ((double)rows * n + (double)n * (n + 1)) * u * tr : 0.0;
        double md = 0.0;
        for (int i = 0; i < n; ++i) md = fmax(md, A[i * LD + i] + s_shift);
        s_maxd = md;
    }
    __syncthreads();
    if (threadIdx.x < n) A[threadIdx.x * LD + threadIdx.x] += s_shift;
    __syncthreads();
    const double tol = (double)n * u * s_maxd;
    for (int j = 0; j < n; ++j) {
        const double d = A[j * LD + j];
        const bool drop = !(d > tol);
        const double piv = drop ? 0.0 : sqrt(d);
        __syncthreads();
        for (int jj = j + 1 + threadIdx.x; jj < n; jj += blockDim.x) A[j * LD + jj] = drop ? 0.0 : A[j * LD + jj] / piv;
        if (threadIdx.x == 0) {
            A[j * LD + j] = drop ? 1.0 : piv;
            dropped[j] = drop;
        }
        __syncthreads();
        const int m = n - j - 1;  // trailing (i, i2), j < i <= i2
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e / m, i2 = j + 1 + e % m;
            if (i <= i2) A[i * LD + i2] -= A[j * LD + i] * A[j * LD + i2];
        }
        __syncthreads();
    }
    // R^{-1} in place: column j from the finished leading block
    for (int j = 0; j < n; ++j) {
        const double rjj = A[j * LD + j];
        for (int i = threadIdx.x; i < j; i += blockDim.x) tmp[i] = A[i * LD + j];
        __syncthreads();
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            double acc = 0.0;
            for (int l = i; l < j; ++l) acc += A[i * LD + l] * tmp[l];
            A[i * LD + j] = dropped[j] ? 0.0 : -acc / rjj;
        }
        __syncthreads();
        if (threadIdx.x == 0) A[j * LD + j] = dropped[j] ? 0.0 : 1.0 / rjj;
        __syncthreads();
    }
    T *out = Rinv + (int64_t)b * lp * lp;
    for (int e = threadIdx.x; e < lp * lp; e += blockDim.x) {
        const int i = e % lp, j = e / lp;
        out[e] = (i < n && j < n && i <= j) ? (T)A[i * LD + j] : T(0);
    }
}

// u-factors: Ucat[(s_i + row) 2r + side r + j] = sum_q Q_b[row, q] E_b[j, q]
// (b = 2 i + side, rows < n_i), E_b the leading eigenvectors (r x lp).
template <typename T>
__global__ void __launch_bounds__(128)
    k_wide_u(const T *__restrict__ Q, int64_t PS, int lp, const T *__restrict__ E, int r, Parts P, T *__restrict__ Ucat) {
    extern __shared__ __align__(16) unsigned char usm[];
    T *Es = reinterpret_cast<T *>(usm);  // r x lp
    const int b = blockIdx.y, part = b / 2, side = b % 2;
    for (int e = threadIdx.x; e < r * lp; e += blockDim.x) Es[e] = E[(int64_t)b * r * lp + e];
    __syncthreads();
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= ni) return;
    const T *q = Q + (int64_t)b * PS * lp + row;
    T *out = Ucat + (s + row) * 2 * r + side * r;
    for (int j0 = 0; j0 < r; j0 += 16) {
        T acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = T(0);
        for (int l = 0; l < lp; ++l) {
            const T qv = q[(int64_t)l * PS];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j0 + j < r) acc[j] = fma(qv, Es[(j0 + j) * lp + l], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j0 + j < r) out[j0 + j] = acc[j];
    }
}

// Vector panels: V[part][c][row] (leading dimension PS) <- r / |r|.
template <typename T>
__global__ void k_wide_pack(const double *__restrict__ rin, const double *__restrict__ inv, int64_t n, Parts P,
                            int64_t PS, int nrhs, T *__restrict__ V) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= PS) return;
    for (int c = 0; c < nrhs; ++c)
        V[((int64_t)part * VP + c) * PS + row] = (row < ni) ? (T)(rin[c * n + s + row] * inv[c]) : T(0);
}

// Transposed D-stage input: h / |h| minus V^T w at the partition tips
// (top rows: P_{i-1}^T w_zeta(i-1); bottom rows: Q_{i+1}^T w_omega(i)).
template <typename T>
__global__ void k_wide_pack_t(const double *__restrict__ hin, const double *__restrict__ inv,
                              const double *__restrict__ zr, const T *__restrict__ PQ, int W, Parts P, int k, int r,
                              int64_t n, int64_t PS, int nrhs, T *__restrict__ V) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= PS) return;
    const int n2 = 2 * r;
    for (int c = 0; c < nrhs; ++c) {
        double v = 0.0;
        if (row < ni) {
            v = hin[c * n + s + row] * inv[c];
            if (r > 0 && row < k && part >= 1) {
                const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * W;
                for (int j = 0; j < r; ++j)
                    v -= (double)Pm[(int64_t)j * W + row] * zr[((int64_t)(part - 1) * n2 + j) * nrhs + c];
            }
            if (r > 0 && row >= ni - k && part <= P.p - 2) {
                const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * W;
                const int64_t q = row - (ni - k);
                for (int j = 0; j < r; ++j)
                    v -= (double)Qm[(int64_t)j * W + q] * zr[((int64_t)part * n2 + r + j) * nrhs + c];
            }
        }
        V[((int64_t)part * VP + c) * PS + row] = (T)v;
    }
}

// g (n x nrhs, leading dimension n) <- the D-stage panel
template <typename T>
__global__ void k_wide_unpack(const T *__restrict__ V, int64_t n, Parts P, int64_t PS, int nrhs, T *__restrict__ Gv) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= ni) return;
    for (int c = 0; c < nrhs; ++c) Gv[c * n + s + row] = V[((int64_t)part * VP + c) * PS + row];
}

// x (+)= |h| * the transposed D-stage panel
template <typename T>
__global__ void k_wide_unpack_t(const T *__restrict__ V, const double *__restrict__ nrm, Parts P, int64_t PS,
                                int nrhs, double *__restrict__ x, int64_t ldx, int accumulate) {
    const int part = blockIdx.y;
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= ni) return;
    for (int c = 0; c < nrhs; ++c) {
        const double upd = nrm[c] * (double)V[((int64_t)part * VP + c) * PS + row];
        const int64_t xi = c * ldx + s + row;
        x[xi] = accumulate ? x[xi] + upd : upd;
    }
}

// psi_{i-1}[0:r] = P_{i-1} g_t,  psi_i[r:2r] = Q_{i+1} g_b  (FP64): one warp
// per (side, j, column) of a partition, lanes over the k tip rows (coalesced
// reads of the P / Q row and of g), partial sums added by a warp reduction.
constexpr int PSI_WARPS = 8;
template <typename T>
__global__ void __launch_bounds__(32 * PSI_WARPS)
    k_wide_psi(const T *__restrict__ Gv, const T *__restrict__ PQ, int W, Parts P, int k, int r, int64_t n,
               int nrhs, double *__restrict__ psi) {
    const int part = blockIdx.x, lane = threadIdx.x & 31;
    const int o = blockIdx.y * PSI_WARPS + (threadIdx.x >> 5);
    if (o >= 2 * r * nrhs) return;  // warp-uniform
    const int64_t s = P.off[part], ni = P.off[part + 1] - s;
    const int n2 = 2 * r;
    const int side = o / (r * nrhs), rem = o % (r * nrhs), j = rem / nrhs, c = rem % nrhs;
    if (side == 0 && part >= 1) {
        const T *Pm = PQ + ((int64_t)(part - 1) * 2 + 0) * r * W + (int64_t)j * W;
        double acc = 0.0;
        for (int q = lane; q < k; q += 32) acc += (double)Pm[q] * (double)Gv[c * n + s + q];
        acc = warp_sum(acc);
        if (lane == 0) psi[((int64_t)(part - 1) * n2 + j) * nrhs + c] = acc;
    } else if (side == 1 && part <= P.p - 2) {
        const T *Qm = PQ + ((int64_t)(part + 1) * 2 + 1) * r * W + (int64_t)j * W;
        double acc = 0.0;
        for (int q = lane; q < k; q += 32) acc += (double)Qm[q] * (double)Gv[c * n + s + ni - k + q];
        acc = warp_sum(acc);
        if (lane == 0) psi[((int64_t)part * n2 + r + j) * nrhs + c] = acc;
    }
}

// flag[d] = 1 when band row d holds a nonzero entry inside the matrix
__global__ void k_nonzero_diags(const double *__restrict__ band, int64_t ld, int64_t n, int k, int *__restrict__ flag) {
    const int d = blockIdx.y;
    const int64_t lo = std::max<int64_t>(0, k - d), hi = std::min<int64_t>(n, n + k - d);  // columns j with 0 <= j+d-k < n
    bool any = false;
    for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi; j += (int64_t)gridDim.x * blockDim.x)
        any = any || band[(int64_t)d * ld + j] != 0.0;
    if (__syncthreads_or(any) && threadIdx.x == 0) flag[d] = 1;
}

// ---------------------------------------------------------------------------
// D-stage (and its transpose) of the wide-band factors: one cluster of CS
// CTAs per partition walks the forward and the backward block recurrence
//   forward  t = b_J - Lo_{J-1} y_{J-1},  y_J = D_J t
//   backward t = y_J - Up_J x_{J+1},      x_J = E_J t
// (A: Lo = L_{J,J-1}, D = L_JJ^{-1}, Up = U_{J,J+1}, E = U_JJ^{-1};
//  A^T: Lo = U_{J-1,J}^T, D = U_JJ^{-T}, Up = L_{J+1,J}^T, E = L_JJ^{-T}).
// Every product is a set of dot products of "lines" of a factor tile with the
// gathered vector: rows of the row-major tiles (A) or columns of the
// column-major tiles (A^T), both contiguous in memory.  Line a of Lo and E
// holds its nonzeros in [a, W) ("tail"), of D and Up in [0, a] ("head").
//
// CTA c of a cluster owns lines a = c + CS t, sixteen at a time (a group).  A
// 4-D tensor map views each tile kind as [tile][t][phase c][column], so one
// TMA load (cp.async.bulk.tensor) brings a box of a group's 16 lines x
// BC columns (at most 1 KB per line) into a shared-memory slot; only the
// boxes that meet the group's nonzero columns are loaded (the rest of the
// triangle is never read; zeros inside a loaded box are multiplied as they
// are).  Warp DS_CONSUMERS (producer) streams the boxes of every product in
// order into a ring of slots, completion counted on the slot's mbarrier,
// running ahead of the consumers across products (the tiles do not depend on
// the vectors).  Warps 0..DS_CONSUMERS-1 (consumers) take (group, quarter)
// items in turn and their boxes in order (the four quarters of a box free its
// slot together): per box and
// quarter of the group (four lines), lanes over 4-entry pieces, the four lines
// at once so each vector entry read from shared memory serves four lines, and
// a butterfly reduce-scatter at the end.
// After each product the CTAs exchange their slices of the result through
// distributed shared memory (double-buffered, one cluster barrier per
// product).  Input b in V1, y in V2, result x in V1 (panel column c at c PS).
// Waits on the ring are bounded; one that runs out sets *err and the CTA
// keeps walking the barrier sequence without computing, so the cluster ends.
// Eight consumer warps and an 80 KB ring: two CTAs fit on an SM, so every SM
// interleaves the chains of two partitions (each product of a chain ends in
// a cluster barrier and an exchange, which one chain alone cannot hide; with
// sixteen consumer warps and one CTA per SM an application took 2.76 ms at
// the 1024^2 convection-diffusion size, 2.04 ms like this).
constexpr int DS_CONSUMERS = 8;
constexpr int DS_THREADS = 32 * (DS_CONSUMERS + 1);
constexpr int DS_GL = 16;  // lines per group (one TMA box)
constexpr long long kDsSpin = 1ll << 26;

__device__ __forceinline__ uint32_t ds_smem(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool ds_wait(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kDsSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(ds_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i >= 64) __nanosleep(32);
    }
    return false;
}
template <typename T>
struct V4 {
    T x, y, z, w;
};
// four consecutive shared-memory values (16-byte aligned), one vector load
template <typename T>
__device__ __forceinline__ V4<T> lds4(const T *p);
// four BF16 tile values (8-byte aligned) widened to FP32: a BF16 value is the
// high half of the FP32 value with the same bits, so the widening is exact
__device__ __forceinline__ V4<float> lds4(const __nv_bfloat16 *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    return {__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
            __uint_as_float(u.y & 0xffff0000u)};
}
template <typename T>
__device__ __forceinline__ V4<T> lds4(const T *p) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        return {v.x, v.y, v.z, v.w};
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        return {a.x, a.y, b.x, b.y};
    }
}
// Butterfly reduce-scatter of N values (N a power of two, 4 <= N <= 16) over
// the 32 lanes: at step o = 16, 8, .. each lane keeps the half of its values
// selected by bit o of its lane and adds the partner's copy of that half;
// N - 1 + log2(32 / N) shuffles leave in v[0] the warp sum of the value index
// returned, in every lane.
template <typename T, int N>
__device__ __forceinline__ int butterfly_reduce(T (&v)[N], int lane) {
    int j = 0;
#pragma unroll
    for (int half = N / 2, o = 16; half >= 1; half /= 2, o /= 2) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const T keep = up ? v[q + half] : v[q];
            const T send = up ? v[q] : v[q + half];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (up) j += half;
    }
#pragma unroll
    for (int o = 32 / N / 2; o >= 1; o /= 2) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return j;
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"r"(32 * DS_CONSUMERS) : "memory"); }

// Product k of the 4 NB products: forward J = k/2 (sub 0: Lo_{J-1}, sub 1:
// D_J), backward J = NB-1-(k-2NB)/2 (sub 0: Up_J, sub 1: E_J).  Products 0
// and 2NB read no tile (they copy b_0 and y_{NB-1}).  kind: 0 Lo, 1 D, 2 Up, 3 E.
struct DsProduct {
    int J, sub, kind, blk;
    bool fwd, tile, head;
};
__device__ __forceinline__ DsProduct ds_product(int k, int NB) {
    DsProduct d;
    d.fwd = k < 2 * NB;
    const int q = d.fwd ? k : k - 2 * NB;
    d.sub = q & 1;
    d.J = d.fwd ? q / 2 : NB - 1 - q / 2;
    d.tile = !(q == 0);
    d.head = d.fwd ? (d.sub == 1) : (d.sub == 0);
    d.kind = d.fwd ? d.sub : 2 + d.sub;
    d.blk = (d.fwd && d.sub == 0) ? d.J - 1 : d.J;
    return d;
}
// first and one-past-last box column index of group g (boxes of BC columns)
__device__ __forceinline__ void ds_boxes(bool head, int cr, int CS, int g, int W, int BC, int &b0, int &b1) {
    if (head) {
        b0 = 0;
        b1 = (cr + CS * (DS_GL * g + DS_GL - 1)) / BC + 1;  // through the last line's diagonal
    } else {
        b0 = (cr + CS * (DS_GL * g)) / BC;
        b1 = (W + BC - 1) / BC;
    }
}

struct DsMaps {
    CUtensorMap m[4];
};

// T: vectors and accumulation; TT: factor tiles (T, or BF16 with BF16 factors)
template <typename T, typename TT, int NR>
__global__ void __launch_bounds__(DS_THREADS, 2)
    k_wide_dstage(const __grid_constant__ DsMaps maps, int W, int NB, int64_t PS, int c0, int S, int BC, T *V1,
                  T *V2, int *err) {
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    const int part = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int owned = W / CS, G = owned / DS_GL, nprod = 4 * NB, nbc = (W + BC - 1) / BC;
    extern __shared__ __align__(128) unsigned char dsm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(dsm), *empty = full + S;
    // boxes the producer has posted (byte count on the slot's barrier): a
    // consumer waits for its box to be posted before it waits on the slot's
    // phase, so the parity it tests cannot belong to an older use of the slot
    volatile long long *posted = reinterpret_cast<volatile long long *>(empty + S);
    int *pre = reinterpret_cast<int *>(dsm + 2 * S * 8 + 8);  // box prefix per group: head G+1, tail G+1
    // TMA box destinations: 128-byte aligned slots after the header
    TT *ring = reinterpret_cast<TT *>((reinterpret_cast<uintptr_t>(dsm) + 2 * S * 8 + 8 + 8 * (G + 1) + 1023) &
                                      ~(uintptr_t)1023);
    T *vin = reinterpret_cast<T *>(ring + (int64_t)S * DS_GL * BC);  // NR columns of W
    T *slice0 = vin + (int64_t)W * NR, *slice1 = slice0 + (int64_t)owned * NR;
    T *v1 = V1 + ((int64_t)part * VP + c0) * PS, *v2 = V2 + ((int64_t)part * VP + c0) * PS;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ds_smem(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(ds_smem(&empty[s])) : "memory");
        }
        *posted = 0;
        for (int h = 0; h < 2; ++h) {
            int acc = 0;
            for (int g = 0; g < G; ++g) {
                pre[h * (G + 1) + g] = acc;
                int b0, b1;
                ds_boxes(h == 0, cr, CS, g, W, BC, b0, b1);
                acc += b1 - b0;
            }
            pre[h * (G + 1) + G] = acc;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    (void)nbc;

    if (warp == DS_CONSUMERS) {
        // producer (lane 0): the boxes of every product in order, then the
        // product's barrier (whole warp)
        bool ok = true;
        int64_t seq = 0;
        for (int k = 0; k < nprod; ++k) {
            const DsProduct d = ds_product(k, NB);
            if (d.tile && lane == 0) {
                const CUtensorMap *map = &maps.m[d.kind];
                const int tix = part * NB + d.blk;
                for (int g = 0; g < G; ++g) {
                    int b0, b1;
                    ds_boxes(d.head, cr, CS, g, W, BC, b0, b1);
                    for (int bx = b0; bx < b1; ++bx, ++seq) {
                        if (!ok) continue;
                        const int slot = (int)(seq % S);
                        const uint32_t par = (uint32_t)((seq / S) & 1);
                        if (!ds_wait(&empty[slot], par ^ 1u)) {
                            ok = false;
                            atomicExch(err, 1);
                            continue;
                        }
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                         ds_smem(&full[slot])),
                                     "r"((uint32_t)(DS_GL * BC * sizeof(TT)))
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                            "[%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(ds_smem(ring + (int64_t)slot * DS_GL * BC)),
                            "l"(reinterpret_cast<uint64_t>(map)), "r"(ds_smem(&full[slot])), "r"(bx * BC), "r"(cr),
                            "r"(DS_GL * g), "r"(tix)
                            : "memory");
                        __threadfence_block();
                        *posted = seq + 1;
                    }
                }
            }
            __syncwarp();
            if (k > 0) cluster_wait();
            cluster_arrive();
        }
        // every copy issued has landed before the CTA may leave (bounded)
        if (lane == 0)
            for (int64_t q = (seq > S ? seq - S : 0); q < seq; ++q) ds_wait(&full[q % S], (uint32_t)((q / S) & 1));
        __syncwarp();
        cluster_wait();
        return;
    }

    // consumers
    bool ok = true;
    int64_t base = 0;  // sequence number of the first box of this product
    for (int k = 0; k < nprod; ++k) {
        const DsProduct d = ds_product(k, NB);
        T *sl = (k & 1) ? slice1 : slice0;
        const int64_t rowJ = (int64_t)d.J * W;
        if (!d.tile) {
            const T *src = d.fwd ? v1 : v2;
            for (int e = threadIdx.x; e < owned * NR; e += 32 * DS_CONSUMERS) {
                const int t = e / NR, c = e % NR;
                sl[e] = src[(int64_t)c * PS + rowJ + cr + CS * t];
            }
        } else {
            const int *pf = pre + (d.head ? 0 : G + 1);
            const T *bsrc = (d.sub == 0) ? (d.fwd ? v1 : v2) + rowJ : nullptr;
            T *gout = (d.sub == 1) ? (d.fwd ? v2 : v1) + rowJ : nullptr;
            // work items (group g, quarter q = four of its lines), round-robin
            // over the warps; the four quarters of a box free its slot together
            for (int item = warp; item < 4 * G; item += DS_CONSUMERS) {
                const int g = item >> 2, q = item & 3;
                int b0, b1;
                ds_boxes(d.head, cr, CS, g, W, BC, b0, b1);
                T acc[4 * NR];
#pragma unroll
                for (int j = 0; j < 4 * NR; ++j) acc[j] = T(0);
                int64_t s = base + pf[g];
                for (int bx = b0; bx < b1; ++bx, ++s) {
                    const int slot = (int)(s % S);
                    const uint32_t par = (uint32_t)((s / S) & 1);
                    bool ready = ok;
                    if (ready && lane == 0) {
                        long long i = 0;
                        while (*posted <= s && i < kDsSpin)
                            if (++i >= 64) __nanosleep(32);
                        ready = *posted > s;
                        __threadfence_block();
                    }
                    ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
                    ready = ready && ds_wait(&full[slot], par);
                    ready = __all_sync(0xffffffffu, ready);
                    if (!ready) {
                        if (ok && lane == 0) atomicExch(err, 1);
                        ok = false;
                        continue;
                    }
                    const TT *buf = ring + (int64_t)slot * DS_GL * BC + (int64_t)(4 * q) * BC;
                    const int col0 = bx * BC, len = min(BC, W - col0);
                    for (int e = 4 * lane; e < len; e += 128) {
                        V4<T> v[NR];
#pragma unroll
                        for (int c = 0; c < NR; ++c) v[c] = lds4(vin + (int64_t)c * W + col0 + e);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const V4<T> m = lds4(buf + i * BC + e);
#pragma unroll
                            for (int c = 0; c < NR; ++c) {
                                T t = acc[i * NR + c];
                                t = fma(m.x, v[c].x, t);
                                t = fma(m.y, v[c].y, t);
                                t = fma(m.z, v[c].z, t);
                                t = fma(m.w, v[c].w, t);
                                acc[i * NR + c] = t;
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ds_smem(&empty[slot]))
                                     : "memory");
                }
                // reduce-scatter of the 4 NR sums over the warp
                const int j = butterfly_reduce<T, 4 * NR>(acc, lane);
                if ((lane & (32 / (4 * NR) - 1)) == 0) {
                    const int i = j / NR, c = j % NR;
                    const int t = DS_GL * g + 4 * q + i, ai = cr + CS * t;
                    T val = acc[0];
                    if (bsrc) val = bsrc[(int64_t)c * PS + ai] - val;
                    sl[t * NR + c] = val;
                    if (gout) gout[(int64_t)c * PS + ai] = val;
                }
            }
            base += pf[G];
        }
        // exchange: every CTA's slice of this product into vin (line a = r' + CS t)
        cluster_arrive();
        cluster_wait();
        if (k + 1 < nprod) {
            constexpr int U = 4;
            for (int a0 = threadIdx.x; a0 < W; a0 += U * 32 * DS_CONSUMERS) {
                T buf[U][NR];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int a = a0 + u * 32 * DS_CONSUMERS;
                    if (a < W) {
                        const T *remote = cl.map_shared_rank(sl, a % CS) + (a / CS) * NR;
#pragma unroll
                        for (int c = 0; c < NR; ++c) buf[u][c] = remote[c];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int a = a0 + u * 32 * DS_CONSUMERS;
                    if (a < W)
#pragma unroll
                        for (int c = 0; c < NR; ++c) vin[(int64_t)c * W + a] = buf[u][c];
                }
            }
            consumers_sync();
        }
    }
}

template <typename T, typename TT, int NR>
size_t dstage_smem(int W, int cs, int S, int BC) {
    const int G = W / cs / DS_GL;
    // header, alignment of the ring to 1024 bytes, ring, vector, two slices
    return (2 * (size_t)S * 8 + 8 + 8 * (G + 1)) + 1024 + (size_t)S * DS_GL * BC * sizeof(TT) +
           (size_t)W * NR * sizeof(T) + 2 * (size_t)(W / cs) * NR * sizeof(T);
}

// Cluster size: the largest CS <= 8 (16-line groups) for which all p
// clusters are resident at once; otherwise the one that keeps the most CTAs
// resident.
template <typename T, typename TT, int NR>
int dstage_cluster(Ctx *c, int S, int BC) {
    int best = 0, fallback = 0;
    int64_t fallback_ctas = 0;
    for (int cs = 1; cs <= 8; cs *= 2) {
        if (c->W % (DS_GL * cs)) break;
        const size_t smem = dstage_smem<T, TT, NR>(c->W, cs, S, BC);
        if (smem > (227u << 10)) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cs, (unsigned)c->p, 1);
        cfg.blockDim = dim3(DS_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, k_wide_dstage<T, TT, NR>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (active >= c->p) best = cs;
        if (active > 0 && (int64_t)std::min(active, c->p) * cs > fallback_ctas) {
            fallback_ctas = (int64_t)std::min(active, c->p) * cs;
            fallback = cs;
        }
    }
    return best ? best : fallback;
}

// 4-D view of a tile kind for the D-stage's boxes: [tile][t][phase][column]
// with line a = phase + CS t; box 16 lines (t) x BC columns.
bool dstage_map(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int64_t es, int W, int CS,
                int64_t ntiles, int BC, std::string *err) {
    cuuint64_t dims[4] = {(cuuint64_t)W, (cuuint64_t)CS, (cuuint64_t)(W / CS), (cuuint64_t)ntiles};
    cuuint64_t strides[3] = {(cuuint64_t)(W * es), (cuuint64_t)(CS * W * es), (cuuint64_t)((int64_t)W * W * es)};
    cuuint32_t box[4] = {(cuuint32_t)BC, 1u, (cuuint32_t)DS_GL, 1u};
    cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return encode_tensor_map(map, dt, 4, base, dims, strides, box, estr, err);
}

template <typename TT> constexpr CUtensorMapDataType tile_dtype() {
    return sizeof(TT) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
           : sizeof(TT) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

template <typename T, typename TT, int NR>
bool launch_dstage(Ctx *c, bool trans, int c0) {
    const int W = c->W;
    // box columns: at most 1 KB per line and 256 elements (the TMA box limit)
    const int BC = std::min(std::min(W, 256), (int)(1024 / sizeof(TT)));
    // A: row-major tiles (lines = rows); A^T: column-major tiles (lines = columns);
    // BF16 factors: the operand-type copies the tensor-core products wrote
    const bool bft = sizeof(TT) == 2;
    void *const *src = trans ? (bft ? c->WFoc : c->WF) : (bft ? c->WFor : c->WFr);
    const void *kinds[4] = {trans ? src[2] : src[3],   // Lo: U_{J-1,J}^T / L_{J,J-1}
                            trans ? src[1] : src[0],   // D: U_JJ^{-T} / L_JJ^{-1}
                            trans ? src[3] : src[2],   // Up: L_{J+1,J}^T / U_{J,J+1}
                            trans ? src[0] : src[1]};  // E: L_JJ^{-T} / U_JJ^{-1}
    // ring slots: 80 KB of boxes, so that two CTAs share an SM
    const int S = (int)std::min<size_t>(16, (80u << 10) / ((size_t)DS_GL * BC * sizeof(TT)));
    cudaFuncSetAttribute(k_wide_dstage<T, TT, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 << 10);
    const int CS = dstage_cluster<T, TT, NR>(c, S, BC);
    if (CS == 0) {
        c->err = "no cluster shape of the wide D-stage fits on this GPU";
        return false;
    }
    DsMaps maps;
    for (int q = 0; q < 4; ++q)
        if (!dstage_map(&maps.m[q], kinds[q], tile_dtype<TT>(), (int64_t)sizeof(TT), W, CS, (int64_t)c->p * c->NBW,
                        BC, &c->err))
            return false;
    const size_t smem = dstage_smem<T, TT, NR>(W, CS, S, BC);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CS, (unsigned)c->p, 1);
    cfg.blockDim = dim3(DS_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    c->dcs = CS;
    cudaError_t e = cudaSuccess;
    const bool ok = launch(c, KID_WIDE_DSTAGE, [&] {
        e = cudaLaunchKernelEx(&cfg, k_wide_dstage<T, TT, NR>, maps, W, c->NBW, c->PS, c0, S, BC, (T *)c->WV1,
                               (T *)c->WV2, c->gemm_err);
    });
    if (e != cudaSuccess) {
        c->err = std::string("cluster launch of the wide D-stage failed: ") + cudaGetErrorString(e);
        return false;
    }
    return ok;
}

template <typename T, typename TT>
bool dstage_chain_tt(Ctx *c, int nrhs, bool trans) {
    for (int c0 = 0; c0 < nrhs; c0 += 4) {
        // three columns run as four: the fourth panel column is independent of
        // the others and never read back
        const int nc = std::min(4, nrhs - c0);
        const bool ok = nc == 1   ? launch_dstage<T, TT, 1>(c, trans, c0)
                        : nc == 2 ? launch_dstage<T, TT, 2>(c, trans, c0)
                                  : launch_dstage<T, TT, 4>(c, trans, c0);
        if (!ok) return false;
    }
    return true;
}

// BF16 factors: the D-stage streams the BF16 copies of the factor tiles (half
// the bytes of the FP32 tiles) and accumulates in FP32
template <typename T>
bool run_dstage_chain(Ctx *c, int nrhs, bool trans) {
    if constexpr (sizeof(T) == 4)
        if (c->gpath == 2) return dstage_chain_tt<T, __nv_bfloat16>(c, nrhs, trans);
    return dstage_chain_tt<T, T>(c, nrhs, trans);
}

// ---------------------------------------------------------------------------
// In-place recursive LU with both inverses of the n x n leading view of S
// (n a multiple of 64): Li = L^{-1}, Ui = U^{-1}; Tm is workspace.  Split
// n = h + n2 with h = 64 ceil(n / 128):
//   A11 = L11 U11;  U12 = L11^{-1} A12;  L21 = A21 U11^{-1};
//   A22 -= L21 U12 = L22 U22;  (L^{-1})_21 = -L22^{-1} (L21 L11^{-1}),
//   (U^{-1})_12 = -U11^{-1} (U12 U22^{-1}).
// The zero triangles of Li, Ui must be zero on entry.  Every product writes
// the layouts its consumers read.
bool luinv(Ctx *c, const WMat &S, const WMat &Li, const WMat &Ui, const WMat &Tm, int n, int64_t row0) {
    const int p = c->p;
    if (n % 64 != 0 || n < 64) {
        c->err = "wide-band block LU: block order is not a multiple of 64";
        return false;
    }
    if (n == 64) {
        if (!run_lu_inv64(c, S.f, (int)S.ld, S.s, Li.f, Ui.f, (int)Li.ld, Li.s, row0)) return false;
        // the other layouts of the two 64 x 64 inverses (row-major working copy
        // for the D-stage, operand copies for the products)
        const dim3 grid(8, p);
        return launch(c, KID_WIDE_VEC, [&] {
            for (const WMat *m : {&Li, &Ui}) {
                if (c->gpath == 2)
                    k_wide_layouts<float, __nv_bfloat16><<<grid, 256, 0, c->stream>>>(
                        (const float *)m->f, 64, m->ld, m->s, (float *)m->fr, (__nv_bfloat16 *)m->oc,
                        (__nv_bfloat16 *)m->orow);
                else if (c->gpath == 1)  // TF32: oc / orow alias f / fr
                    k_wide_layouts<float, float><<<grid, 256, 0, c->stream>>>((const float *)m->f, 64, m->ld, m->s,
                                                                            (float *)m->fr, nullptr, nullptr);
                else if (c->fp64)
                    k_wide_layouts<double, double><<<grid, 256, 0, c->stream>>>(
                        (const double *)m->f, 64, m->ld, m->s, (double *)m->fr, nullptr, nullptr);
                else
                    k_wide_layouts<float, float><<<grid, 256, 0, c->stream>>>((const float *)m->f, 64, m->ld, m->s,
                                                                            (float *)m->fr, nullptr, nullptr);
            }
        });
    }
    const int h = 64 * ((n / 64 + 1) / 2), n2 = n - h;
    auto q12 = [&](const WMat &m) { return view(c, m, 0, h); };
    auto q21 = [&](const WMat &m) { return view(c, m, h, 0); };
    auto q22 = [&](const WMat &m) { return view(c, m, h, h); };
    if (!luinv(c, S, Li, Ui, Tm, h, row0)) return false;
    return gemm(c, h, n2, h, 1.0, Li, false, q12(S), false, 0.0, q12(Tm), p) &&           // U12 = L11^{-1} A12
           gemm(c, n2, h, h, 1.0, q21(S), false, Ui, false, 0.0, q21(Tm), p) &&           // L21 = A21 U11^{-1}
           gemm(c, n2, n2, h, -1.0, q21(Tm), false, q12(Tm), false, 1.0, q22(S), p) &&    // A22 -= L21 U12
           luinv(c, q22(S), q22(Li), q22(Ui), q22(Tm), n2, row0 + h) &&
           gemm(c, n2, h, h, 1.0, q21(Tm), false, Li, false, 0.0, q21(S), p) &&           // L21 L11^{-1}
           gemm(c, n2, h, n2, -1.0, q22(Li), false, q21(S), false, 0.0, q21(Li), p) &&
           gemm(c, h, n2, n2, 1.0, q12(Tm), false, q22(Ui), false, 0.0, q12(S), p) &&     // U12 U22^{-1}
           gemm(c, h, n2, h, -1.0, Ui, false, q12(S), false, 0.0, q12(Ui), p);
}

// Orthonormal basis of the columns of the 2p iterates in Y (PS x lp, first
// ell columns live) by shifted CholeskyQR3; the result lands in Qout.
template <typename T>
bool cholqr3(Ctx *c, void *Y, void *Qout) {
    const int lp = c->lp, ell = c->ell, nm = 2 * c->p;
    const int64_t PS = c->PS, sY = PS * lp, sG = (int64_t)lp * lp;
    const double u = c->fp64 ? 0x1p-53 : 0x1p-24;
    const size_t smem = ((size_t)ell * (ell + 1) + ell) * sizeof(double);
    cudaFuncSetAttribute(k_chol_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int pass = 0; pass < 3; ++pass) {
        // pass 0: Y -> Qout (shifted); 1: Qout -> Y; 2: Y -> Qout
        void *src = (pass == 1) ? Qout : Y, *dst = (pass == 1) ? Y : Qout;
        const int tiles = (lp + 63) / 64, nch = gram_chunks(PS);
        const dim3 gg((unsigned)(tiles * tiles), (unsigned)nch, (unsigned)nm);
        const dim3 gq((unsigned)((PS + 63) / 64), (unsigned)((lp + 63) / 64), (unsigned)nm);
        const bool ok =
            launch(c, KID_WIDE_CHOLQR, [&] {
                k_gram_part<T><<<gg, 256, 0, c->stream>>>((const T *)src, lp, PS, sY, (T *)c->WGp);
            }) &&
            launch(c, KID_WIDE_CHOLQR, [&] {
                k_gram_sum<T><<<256, 256, 0, c->stream>>>((const T *)c->WGp, nch, sG, nm * sG, c->WGd);
            }) &&
            launch(c, KID_WIDE_CHOLQR, [&] {
                k_chol_inv<T><<<nm, 256, smem, c->stream>>>(c->WGd, lp, ell, PS, u, pass == 0 ? 1 : 0, (T *)c->WRi);
            }) &&
            launch(c, KID_WIDE_CHOLQR, [&] {
                k_simt_gemm<T><<<gq, 256, 0, c->stream>>>((int)PS, lp, lp, T(1), T(0), (const T *)src, 1, PS, sY,
                                                          (const T *)c->WRi, lp, 1, sG, (T *)dst, PS, sY, nullptr, 0,
                                                          0);
            });
        if (!ok) return false;
    }
    return true;
}

template <typename T>
bool wide_compress_t(Ctx *c);

template <typename T>
bool wide_factor_t(Ctx *c) {
    const int W = c->W, NB = c->NBW, p = c->p;
    const int64_t WW = (int64_t)W * W, sF = NB * WW;
    const bool tc = c->gpath != 0, bf = c->gpath == 2;
    Parts P{c->off_d, c->boff_d, p};
    if (cudaMemsetAsync(c->gemm_err, 0, sizeof(int), c->stream) != cudaSuccess) {
        c->err = "cudaMemsetAsync failed";
        return false;
    }
    // the zero triangles of the diagonal-block inverses (every layout)
    for (int kind = 0; kind < 2; ++kind) {
        void *arrs[4] = {c->WF[kind], c->WFr[kind], c->WFoc[kind], c->WFor[kind]};
        const size_t szs[4] = {c->tsize, c->tsize, c->osize, c->osize};
        for (int l = 0; l < 4; ++l)
            if (arrs[l] && cudaMemsetAsync(arrs[l], 0, (size_t)p * sF * szs[l], c->stream) != cudaSuccess) {
                c->err = "cudaMemsetAsync failed";
                return false;
            }
    }
    WMat S = square(c->WSm, W, WW), Bm = square(c->WBm, W, WW), Cm = square(c->WCm, W, WW),
         Tm = square(c->WTm, W, WW);
    auto tile = [&](int kind, int J) {  // factor tile J of the given kind, all partitions
        return WMat{elem(c->WF[kind], J * WW, c->tsize), elem(c->WFr[kind], J * WW, c->tsize),
                    elem(c->WFoc[kind], J * WW, c->osize), elem(c->WFor[kind], J * WW, c->osize), W, sF, W, sF};
    };
    for (int J = 0; J < NB; ++J) {
        if (!launch(c, KID_WIDE_GATHER, [&] {
                const dim3 grid(W / 32, W / 32, 3 * p);
                if (bf)
                    k_wide_gather<float, __nv_bfloat16><<<grid, 256, 0, c->stream>>>(
                        c->band, c->ld, c->k, P, W, J, (float *)S.f, nullptr, (__nv_bfloat16 *)S.oc,
                        (__nv_bfloat16 *)S.orow, (float *)Bm.f, (__nv_bfloat16 *)Bm.oc, (float *)Cm.f,
                        (__nv_bfloat16 *)Cm.orow);
                else if (tc)
                    k_wide_gather<float, float><<<grid, 256, 0, c->stream>>>(
                        c->band, c->ld, c->k, P, W, J, (float *)S.f, nullptr, nullptr, (float *)S.orow, (float *)Bm.f,
                        nullptr, (float *)Cm.f, (float *)Cm.orow);
                else
                    k_wide_gather<T, T><<<grid, 256, 0, c->stream>>>(c->band, c->ld, c->k, P, W, J, (T *)S.f,
                                                                     nullptr, nullptr, nullptr, (T *)Bm.f, nullptr,
                                                                     (T *)Cm.f, nullptr);
            }))
            return false;
        const WMat Li = tile(0, J), Ui = tile(1, J), Z = tile(2, J), Y = tile(3, J);
        if (J > 0 && !gemm(c, W, W, W, -1.0, tile(3, J - 1), false, tile(2, J - 1), false, 1.0, S, p)) return false;
        if (!luinv(c, S, Li, Ui, Tm, W, (int64_t)J * W)) return false;
        if (!gemm(c, W, W, W, 1.0, Li, false, Bm, false, 0.0, Z, p) ||
            !gemm(c, W, W, W, 1.0, Cm, false, Ui, false, 0.0, Y, p))
            return false;
    }
    if (p < 2 || c->r == 0) return true;

    return wide_compress_t<T>(c);
}

// Rank-r truncation of every spike by the HMT proto-algorithm (section 3.1)
// without forming the spikes: with T = A_i^{-1}[0; B_i] and W = A_i^{-1}[C_i; 0]
// every product the range finder needs is a block solve with the factors on
// a panel of 2 lp columns (T side, W side):
//   T X   = A_i^{-1} [0; B_i X],        W X   = A_i^{-1} [C_i X; 0]
//   T^T Q = B_i^T (A_i^{-T} Q)_bottom,   W^T Q = C_i^T (A_i^{-T} Q)_top
// Y = T Omega, Q = orth(Y); q times Y = T (T^T Q), Q = orth(Y); B^T = T^T Q;
// then the eigenvectors U_B of B B^T, u = Q U_B,r and P = U_B,r^T B as before.
template <typename T>
bool wide_compress_t(Ctx *c) {
    const int W = c->W, NB = c->NBW, p = c->p, lp = c->lp, ell = c->ell, r = c->r, nm = 2 * p;
    const int64_t WW = (int64_t)W * W, sF = NB * WW, PS = c->PS, sP = PS * 2 * lp, sQ = PS * lp,
                  sZ = (int64_t)W * lp;
    const bool tc = c->gpath != 0, bf = c->gpath == 2;
    const size_t tz = c->tsize, oz = c->osize;
    Parts P{c->off_d, c->boff_d, p};
    auto tile = [&](int kind, int J) {
        return WMat{elem(c->WF[kind], J * WW, tz), elem(c->WFr[kind], J * WW, tz), elem(c->WFoc[kind], J * WW, oz),
                    elem(c->WFor[kind], J * WW, oz), W, sF, W, sF};
    };
    // panel rows of block J (both sides), column-major PS x 2lp
    auto pv = [&](void *f, void *oc, int64_t J) {
        WMat m;
        m.f = elem(f, J * W, tz);
        m.oc = bf ? elem(oc, J * W, oz) : m.f;
        m.ld = PS;
        m.s = sP;
        return m;
    };
    // P1 <- A^{-1} P1 (or A^{-T} P1): forward then backward block recurrence
    auto solve = [&](bool trans) {
        for (int J = 0; J < NB; ++J) {
            const WMat x1 = pv(c->WP1, c->WP1c, J), x2 = pv(c->WP2, c->WP2c, J);
            if (J > 0 && !gemm(c, W, 2 * lp, W, -1.0, tile(trans ? 2 : 3, J - 1), trans,
                               pv(c->WP2, c->WP2c, J - 1), false, 1.0, x1, p))
                return false;
            if (!gemm(c, W, 2 * lp, W, 1.0, tile(trans ? 1 : 0, J), trans, x1, false, 0.0, x2, p)) return false;
        }
        for (int J = NB - 1; J >= 0; --J) {
            const WMat x2 = pv(c->WP2, c->WP2c, J), x1 = pv(c->WP1, c->WP1c, J);
            if (J < NB - 1 && !gemm(c, W, 2 * lp, W, -1.0, tile(trans ? 3 : 2, J), trans,
                                    pv(c->WP1, c->WP1c, J + 1), false, 1.0, x2, p))
                return false;
            if (!gemm(c, W, 2 * lp, W, 1.0, tile(trans ? 0 : 1, J), trans, x2, false, 0.0, x1, p)) return false;
        }
        return true;
    };
    const WMat Cpl = square(c->WCpl, W, WW);
    WMat Om;
    Om.f = Om.oc = c->WOm;
    Om.ld = W;
    Om.s = sZ;
    WMat Tip;
    Tip.f = c->WTip;
    Tip.oc = bf ? c->WTipc : c->WTip;
    Tip.ld = W;
    Tip.s = sZ;
    WMat Zk;
    Zk.f = c->WZk;
    Zk.oc = bf ? c->WZc : c->WZk;
    Zk.ld = W;
    Zk.s = sZ;
    const size_t panel_bytes = (size_t)p * sP;
    auto clear_panel = [&]() {
        return cudaMemsetAsync(c->WP1, 0, panel_bytes * tz, c->stream) == cudaSuccess &&
               (!bf || cudaMemsetAsync(c->WP1c, 0, panel_bytes * oz, c->stream) == cudaSuccess);
    };
    // P1 <- the right-hand sides [0; B_i X_T | C_i X_W; 0]
    auto couple = [&](const WMat &X) {
        if (!clear_panel() || !gemm(c, W, lp, W, 1.0, Cpl, false, X, false, 0.0, Tip, nm)) return false;
        return launch(c, KID_WIDE_VEC, [&] {
            const dim3 g(64, nm);
            if (bf)
                k_tips_scatter<float, __nv_bfloat16><<<g, 256, 0, c->stream>>>(
                    (const float *)c->WTip, P, c->k, W, PS, lp, (float *)c->WP1, (__nv_bfloat16 *)c->WP1c);
            else
                k_tips_scatter<T, T><<<g, 256, 0, c->stream>>>((const T *)c->WTip, P, c->k, W, PS, lp,
                                                               (T *)c->WP1, nullptr);
        });
    };
    // Zk <- [B_i^T (P1)_bottom | C_i^T (P1)_top]
    auto couple_t = [&]() {
        if (!launch(c, KID_WIDE_VEC, [&] {
                const dim3 g(64, nm);
                if (bf)
                    k_tips_gather<float, __nv_bfloat16><<<g, 256, 0, c->stream>>>(
                        (const float *)c->WP1, P, c->k, W, PS, lp, (float *)c->WTip, (__nv_bfloat16 *)c->WTipc);
                else
                    k_tips_gather<T, T><<<g, 256, 0, c->stream>>>((const T *)c->WP1, P, c->k, W, PS, lp,
                                                                  (T *)c->WTip, nullptr);
            }))
            return false;
        return gemm(c, W, lp, W, 1.0, Cpl, true, Tip, false, 0.0, Zk, nm);
    };
    // Q <- orth(Y) for the Y in P1 (2p matrices PS x lp); Q stays in WQk and is
    // copied back into P1 (and its operand copy) for the next solve
    auto orth = [&]() {
        if (!cholqr3<T>(c, c->WP1, c->WQk)) return false;
        if (cudaMemcpyAsync(c->WP1, c->WQk, (size_t)nm * sQ * tz, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return false;
        if (!bf) return true;
        return launch(c, KID_WIDE_VEC, [&] {
            k_to_op<float, __nv_bfloat16><<<1024, 256, 0, c->stream>>>((const float *)c->WQk, (__nv_bfloat16 *)c->WP1c,
                                                                      (int64_t)nm * sQ);
        });
    };
    // coupling tiles and the sketches
    if (!launch(c, KID_WIDE_GATHER, [&] {
            const dim3 g((unsigned)std::min<int64_t>(1024, ((int64_t)c->k * c->k + 255) / 256), nm);
            for (int l = 0; l < 4; ++l) {
                void *q = c->WCpl[l];
                const size_t sz = (l < 2) ? tz : oz;
                if (q) cudaMemsetAsync(q, 0, (size_t)nm * WW * sz, c->stream);
            }
            if (bf)
                k_wide_couple_gather<float, __nv_bfloat16><<<g, 256, 0, c->stream>>>(
                    c->band, c->ld, c->k, P, W, (float *)Cpl.f, (__nv_bfloat16 *)Cpl.oc, (__nv_bfloat16 *)Cpl.orow);
            else if (tc)
                k_wide_couple_gather<float, float><<<g, 256, 0, c->stream>>>(c->band, c->ld, c->k, P, W,
                                                                           (float *)Cpl.f, nullptr, (float *)Cpl.orow);
            else
                k_wide_couple_gather<T, T><<<g, 256, 0, c->stream>>>(c->band, c->ld, c->k, P, W, (T *)Cpl.f, nullptr,
                                                                   nullptr);
            if (bf)
                k_wide_sketch<__nv_bfloat16><<<1024, 256, 0, c->stream>>>((__nv_bfloat16 *)c->WOm, W, c->k, ell, lp,
                                                                         c->opt.seed, nm);
            else
                k_wide_sketch<T><<<1024, 256, 0, c->stream>>>((T *)c->WOm, W, c->k, ell, lp, c->opt.seed, nm);
        }))
        return false;
    if (!couple(Om) || !solve(false) || !orth()) return false;
    for (int it = 0; it < c->opt.power_iters; ++it)
        if (!solve(true) || !couple_t() || !couple(Zk) || !solve(false) || !orth()) return false;
    // B^T = T^T Q (W x lp); H = B B^T = Z^T Z (FP64 for the eigensolver)
    if (!solve(true) || !couple_t()) return false;
    const dim3 gg((unsigned)((lp + 63) / 64), (unsigned)((lp + 63) / 64), (unsigned)nm);
    if (!launch(c, KID_WIDE_CHOLQR, [&] {
            k_simt_gemm<T><<<gg, 256, 0, c->stream>>>(lp, lp, W, T(1), T(0), (const T *)c->WZk, W, 1, sZ,
                                                      (const T *)c->WZk, W, 1, sZ, (T *)c->WG, lp, (int64_t)lp * lp,
                                                      nullptr, 0, 0);
        }) ||
        !launch(c, KID_WIDE_VEC, [&] {
            k_to_f64<T><<<64, 256, 0, c->stream>>>((const T *)c->WG, c->WGd, (int64_t)nm * lp * lp);
        }) ||
        !run_jacobi_batch(c, lp, c->WGd, nm, r, c->opt.rank_tol, c->WE, c->sigma))
        return false;
    // P_b^T = Z_b U_B,r (W x r, leading dimension W): PQ holds P row-major r x W
    const dim3 gp((unsigned)((W + 63) / 64), (unsigned)((r + 63) / 64), (unsigned)nm);
    if (!launch(c, KID_WIDE_VEC, [&] {
            k_simt_gemm<T><<<gp, 256, 0, c->stream>>>(W, r, lp, T(1), T(0), (const T *)c->WZk, 1, W, sZ,
                                                      (const T *)c->WE, lp, 1, (int64_t)r * lp, (T *)c->PQ, W,
                                                      (int64_t)r * W, nullptr, 0, 0);
        }))
        return false;
    // u_b = Q_b U_B,r into Ucat
    const size_t usm = (size_t)r * lp * sizeof(T);
    cudaFuncSetAttribute(k_wide_u<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usm);
    return launch(c, KID_WIDE_VEC, [&] {
        k_wide_u<T><<<dim3((unsigned)((PS + 127) / 128), nm), 128, usm, c->stream>>>((const T *)c->WQk, PS, lp,
                                                                                     (const T *)c->WE, r, P,
                                                                                     (T *)c->Ucat);
    });
}

}  // namespace

bool wide_setup(Ctx *c) {
    const int k = c->k, p = c->p, r = c->r;
    c->W = 64 * ((k + 63) / 64);
    int64_t nbw = 0;
    for (int i = 0; i < p; ++i) nbw = std::max<int64_t>(nbw, (c->off_h[i + 1] - c->off_h[i] + c->W - 1) / c->W);
    c->NBW = (int)nbw;
    c->PS = nbw * c->W;
    c->ell = std::min(k, r + c->opt.oversample);
    c->lp = c->ell <= 16 ? 16 : c->ell <= 32 ? 32 : c->ell <= 64 ? 64 : 128;
    c->gpath = (c->opt.precision == LRSPIKE_MIXED_TF32) ? 1 : (c->opt.precision == LRSPIKE_MIXED_BF16) ? 2 : 0;
    c->osize = (c->gpath == 2) ? 2 : c->tsize;
    const size_t tz = c->tsize, oz = c->osize, W = c->W, WW = W * W, NB = c->NBW, PS = c->PS, lp = c->lp;
    const bool tc = c->gpath != 0, bf = c->gpath == 2;
    auto al = [&](void **ptr, size_t bytes) { return cudaMalloc(ptr, bytes) == cudaSuccess; };
    bool ok = true;
    // factor tiles: f and fr always (the D-stage reads fr for A, f for A^T);
    // operand copies in BF16 mode (TF32: they alias f / fr), which the BF16
    // D-stage reads instead
    for (int kind = 0; kind < 4 && ok; ++kind) {
        ok = al(&c->WF[kind], p * NB * WW * tz) && al(&c->WFr[kind], p * NB * WW * tz);
        if (ok && bf) ok = al(&c->WFoc[kind], p * NB * WW * oz) && al(&c->WFor[kind], p * NB * WW * oz);
        if (ok && !bf && tc) {
            c->WFoc[kind] = c->WF[kind];
            c->WFor[kind] = c->WFr[kind];
        }
    }
    // block-step work: f always; operand layouts in the tensor-core modes
    void **work[4] = {c->WSm, c->WBm, c->WCm, c->WTm};
    for (int w = 0; w < 4 && ok; ++w) {
        ok = al(&work[w][0], p * WW * tz);
        if (ok && tc) {
            if (bf) ok = al(&work[w][2], p * WW * oz) && al(&work[w][3], p * WW * oz);
            else {
                work[w][2] = work[w][0];
                ok = al(&work[w][3], p * WW * oz);
            }
        }
    }
    ok = ok && al(&c->WV1, p * PS * VP * tz) && al(&c->WV2, p * PS * VP * tz) &&
         al((void **)&c->diag_list, (2 * k + 1) * sizeof(int)) && al((void **)&c->gemm_err, sizeof(int));
    if (ok && p > 1 && r > 0) {
        const size_t WL = W * lp, panel = p * PS * 2 * lp;
        ok = al(&c->WP1, panel * tz) && al(&c->WP2, panel * tz) && al(&c->WTip, 2 * p * WL * tz) &&
             al(&c->WOm, 2 * p * WL * (tc ? oz : tz)) && al(&c->WQk, 2 * p * PS * lp * tz) &&
             al(&c->WZk, 2 * p * WL * tz) && al(&c->WG, 2 * p * lp * lp * tz) &&
             al(&c->WGp, 2 * p * (size_t)gram_chunks(PS) * lp * lp * tz) &&
             al((void **)&c->WGd, 2 * p * lp * lp * 8) && al(&c->WRi, 2 * p * lp * lp * tz) &&
             al(&c->WE, 2 * p * (size_t)std::max(r, 1) * lp * tz) && al(&c->WCpl[0], 2 * p * WW * tz);
        if (ok && tc) {
            if (bf) ok = al(&c->WCpl[2], 2 * p * WW * oz) && al(&c->WCpl[3], 2 * p * WW * oz);
            else {
                c->WCpl[2] = c->WCpl[0];
                ok = al(&c->WCpl[3], 2 * p * WW * oz);
            }
        }
        if (ok && bf)
            ok = al(&c->WP1c, panel * oz) && al(&c->WP2c, panel * oz) && al(&c->WTipc, 2 * p * WL * oz) &&
                 al(&c->WZc, 2 * p * WL * oz);
    }
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    return true;
}

void wide_free(Ctx *c) {
    std::vector<void *> ptrs;
    for (int kind = 0; kind < 4; ++kind) {
        ptrs.push_back(c->WF[kind]);
        ptrs.push_back(c->WFr[kind]);
        if (c->WFoc[kind] != c->WF[kind]) ptrs.push_back(c->WFoc[kind]);
        if (c->WFor[kind] != c->WFr[kind]) ptrs.push_back(c->WFor[kind]);
        c->WF[kind] = c->WFr[kind] = c->WFoc[kind] = c->WFor[kind] = nullptr;
    }
    void **work[4] = {c->WSm, c->WBm, c->WCm, c->WTm};
    for (auto w : work) {
        ptrs.push_back(w[0]);
        ptrs.push_back(w[1]);
        if (w[2] != w[0]) ptrs.push_back(w[2]);
        ptrs.push_back(w[3]);
        w[0] = w[1] = w[2] = w[3] = nullptr;
    }
    ptrs.push_back(c->WCpl[0]);
    if (c->WCpl[2] != c->WCpl[0]) ptrs.push_back(c->WCpl[2]);
    ptrs.push_back(c->WCpl[3]);
    c->WCpl[0] = c->WCpl[1] = c->WCpl[2] = c->WCpl[3] = nullptr;
    for (void *q : {c->WP1, c->WP2, c->WP1c, c->WP2c, c->WTip, c->WTipc, c->WOm, c->WQk, c->WZk, c->WZc, c->WG, c->WGp,
                    (void *)c->WGd, c->WRi, c->WE, c->WV1, c->WV2, (void *)c->diag_list, (void *)c->gemm_err})
        ptrs.push_back(q);
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (c->wgraph) cudaGraphExecDestroy(c->wgraph);
    if (c->wcap) cudaStreamDestroy(c->wcap);
    c->wgraph = nullptr;
    c->wcap = nullptr;
}

// Everything a factorisation enqueues: the block factorisation, the spikes
// and their truncation, the reduced system, and the flags of the band rows
// holding a nonzero (the FP64 residual visits only those).
static bool wide_factor_device(Ctx *c) {
    const bool ok = c->fp64 ? wide_factor_t<double>(c) : wide_factor_t<float>(c);
    if (!ok) return false;
    if (c->p > 1 && c->r > 0 && !(run_reduced_build_ld(c, c->W) && run_reduced_factor(c))) return false;
    const int nd = 2 * c->k + 1;
    if (cudaMemsetAsync(c->diag_list, 0, nd * sizeof(int), c->stream) != cudaSuccess) return false;
    return launch(c, KID_DIAGS, [&] {
        k_nonzero_diags<<<dim3(64, nd), 256, 0, c->stream>>>(c->band, c->ld, c->n, c->k, c->diag_list);
    });
}

// The factorisation's few thousand launches (the block products of the
// recursive LU are small) as one graph launch: captured on the handle's
// private stream the first time (and again when the band moves), replayed on
// the handle's stream afterwards.
static bool wide_factor_graph(Ctx *c) {
    if (!c->wgraph || c->wgraph_band != c->band || c->wgraph_ld != c->ld) {
        if (c->wgraph) cudaGraphExecDestroy(c->wgraph);
        c->wgraph = nullptr;
        if (!c->wcap && cudaStreamCreateWithFlags(&c->wcap, cudaStreamNonBlocking) != cudaSuccess) {
            c->err = "capture stream creation failed";
            return false;
        }
        const int64_t l0 = c->launches;
        cudaStream_t own = c->stream;
        c->stream = c->wcap;
        if (cudaStreamBeginCapture(c->wcap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            c->stream = own;
            c->err = "stream capture of the factorisation failed to start";
            return false;
        }
        const bool ok = wide_factor_device(c);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->wcap, &g);
        c->stream = own;
        if (!ok || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (c->err.empty()) c->err = std::string("capture of the factorisation failed: ") + cudaGetErrorString(e);
            return false;
        }
        const cudaError_t ei = cudaGraphInstantiate(&c->wgraph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->wgraph = nullptr;
            c->err = std::string("graph instantiation failed: ") + cudaGetErrorString(ei);
            return false;
        }
        c->wgraph_band = c->band;
        c->wgraph_ld = c->ld;
        c->wgraph_launches = c->launches - l0;
        c->launches = l0;
    }
    if (cudaGraphLaunch(c->wgraph, c->stream) != cudaSuccess) {
        c->err = "graph launch of the factorisation failed";
        return false;
    }
    c->launches += c->wgraph_launches;
    return true;
}

bool run_wide_factor(Ctx *c) {
    // profiling brackets every kernel with events on the handle's stream, so
    // it runs the launches one by one; so does a handle whose capture failed
    bool ok;
    if (c->profile || c->wgraph_failed) {
        ok = wide_factor_device(c);
    } else {
        ok = wide_factor_graph(c);
        if (!ok && !c->wgraph) {  // nothing was launched: run the same work eagerly
            c->wgraph_failed = true;
            c->err.clear();
            ok = wide_factor_device(c);
        }
    }
    if (!ok) return false;
    const int nd = 2 * c->k + 1;
    std::vector<int> flag(nd), list;
    int gerr = 0;
    if (cudaMemcpyAsync(flag.data(), c->diag_list, nd * sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&gerr, c->gemm_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return false;
    if (gerr) {
        c->err = "a tensor-core block product gave up waiting on its pipeline";
        return false;
    }
    for (int d = 0; d < nd; ++d)
        if (flag[d]) list.push_back(d);
    if (list.empty()) list.push_back(c->k);
    c->ndiag = (int)list.size();
    return cudaMemcpyAsync(c->diag_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice,
                           c->stream) == cudaSuccess &&
           cudaStreamSynchronize(c->stream) == cudaSuccess;
}

// inv: the column scale factors of the input (rin / |rin| enters the solve)
template <typename T>
static bool wide_dstage_t(Ctx *c, const double *rin, int nrhs, bool trans, double *x, int64_t ldx, bool acc,
                          const double *inv) {
    const int W = c->W, p = c->p;
    const int64_t PS = c->PS;
    Parts P{c->off_d, c->boff_d, p};
    const dim3 grid((unsigned)((PS + 255) / 256), p);
    if (!launch(c, KID_WIDE_VEC, [&] {
            if (trans)
                k_wide_pack_t<T><<<grid, 256, 0, c->stream>>>(rin, inv, c->zr, (const T *)c->PQ, W, P, c->k, c->r,
                                                              c->n, PS, nrhs, (T *)c->WV1);
            else
                k_wide_pack<T><<<grid, 256, 0, c->stream>>>(rin, inv, c->n, P, PS, nrhs, (T *)c->WV1);
        }))
        return false;
    if (!run_dstage_chain<T>(c, nrhs, trans)) return false;
    if (trans)
        return launch(c, KID_WIDE_VEC, [&] {
            k_wide_unpack_t<T><<<grid, 256, 0, c->stream>>>((const T *)c->WV1, c->nrm + c->opt.max_nrhs, P, PS, nrhs,
                                                            x, ldx, acc ? 1 : 0);
        });
    if (!launch(c, KID_WIDE_VEC, [&] {
            k_wide_unpack<T><<<grid, 256, 0, c->stream>>>((const T *)c->WV1, c->n, P, PS, nrhs, (T *)c->Gv);
        }))
        return false;
    if (p < 2 || c->r == 0) return true;
    return launch(c, KID_WIDE_VEC, [&] {
        const dim3 grid((unsigned)p, (unsigned)((2 * c->r * nrhs + PSI_WARPS - 1) / PSI_WARPS));
        k_wide_psi<T><<<grid, 32 * PSI_WARPS, 0, c->stream>>>((const T *)c->Gv, (const T *)c->PQ, W, P, c->k, c->r,
                                                               c->n, nrhs, c->psi);
    });
}

bool run_wide_dstage_inv(Ctx *c, const double *rin, int nrhs, const double *inv) {
    return c->fp64 ? wide_dstage_t<double>(c, rin, nrhs, false, nullptr, 0, false, inv)
                   : wide_dstage_t<float>(c, rin, nrhs, false, nullptr, 0, false, inv);
}

bool run_wide_dstage(Ctx *c, const double *rin, int nrhs) {
    return run_wide_dstage_inv(c, rin, nrhs, c->nrm + 2 * c->opt.max_nrhs);
}

bool run_wide_dstage_t(Ctx *c, const double *hin, double *x, int64_t ldx, int nrhs, bool accumulate) {
    const double *inv = c->nrm + 2 * c->opt.max_nrhs;
    return c->fp64 ? wide_dstage_t<double>(c, hin, nrhs, true, x, ldx, accumulate, inv)
                   : wide_dstage_t<float>(c, hin, nrhs, true, x, ldx, accumulate, inv);
}

}  // namespace lrs
