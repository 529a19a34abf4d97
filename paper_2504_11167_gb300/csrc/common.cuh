// Shared device-side helpers of the LR-SPIKE CUDA library (sm_103a).
//
// Block geometry.  Every partition A_i is processed in square blocks of KB rows,
// KB in {8, 16, 32, 64} the smallest block that is >= the half-bandwidth k.
// Blocks of >= k rows make A_i block tridiagonal, so the banded LU becomes a
// chain of KB x KB block steps.  A partition of n_i rows holds
// nb_i = ceil(n_i / KB) blocks; rows n_i .. nb_i*KB-1 are padding rows that
// carry the identity and zero right-hand sides, so every kernel works on full
// tiles.  A CTA of NT = 4*KB threads serves one tile; tile rows map to
// groups of four consecutive lanes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lrs {

template <int KB> struct Geo {
    static constexpr int NT = 4 * KB;  // threads per CTA for tile work
    static constexpr int W = 2 * KB;   // window of one LU block step
    // LU window thread grid TY x TX, each thread owning RY x RX window entries
    static constexpr int TX = (KB >= 64) ? 16 : 8;
    static constexpr int TY = NT / TX;
    static constexpr int RY = W / TY;
    static constexpr int RX = W / TX;
};

// Partition geometry passed to kernels (device arrays of p+1 entries).
struct Parts {
    const int64_t *off;   // row offset s_i of partition i, off[p] = n
    const int64_t *boff;  // first global block index of partition i, boff[p] = NB
    int p;
};

__device__ __forceinline__ int part_of_block(const Parts &P, int64_t blk) {
    int lo = 0, hi = P.p - 1;
    while (lo < hi) {  // last i with boff[i] <= blk
        int mid = (lo + hi + 1) >> 1;
        if (P.boff[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T> __device__ __forceinline__ T to(double v) { return (T)v; }

__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }

// Reduction over the 4 lanes that share a tile row (lanes 4q..4q+3 of a warp).
template <typename T> __device__ __forceinline__ T quad_sum(T v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A[i][j] of partition-local indices from the diagonal-major band, with the
// identity on the padding rows.  s: row offset of the partition, ni: its size.
__device__ __forceinline__ double band_local(const double *__restrict__ band, int64_t ld, int k,
                                             int64_t s, int64_t ni, int64_t i, int64_t j) {
    if (i < 0 || j < 0) return 0.0;
    if (i >= ni || j >= ni) return (i == j) ? 1.0 : 0.0;
    int64_t d = (int64_t)k + i - j;
    if (d < 0 || d > 2 * k) return 0.0;
    return band[d * ld + s + j];
}

// Pivot reciprocal: the hardware approximate reciprocal; in FP64 refined by
// two Newton-Raphson steps r <- r (2 - v r) (each squares the relative error,
// from about 2^-22 to below 2^-53).  A pivot below the smallest normal number
// counts as singular.
template <typename T> __device__ __forceinline__ T fast_rcp(T v);
template <> __device__ __forceinline__ float fast_rcp<float>(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
template <> __device__ __forceinline__ double fast_rcp<double>(double v) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
    r = r * (2.0 - v * r);
    r = r * (2.0 - v * r);
    return r;
}
template <typename T> __device__ __forceinline__ bool usable_pivot(T v);
template <> __device__ __forceinline__ bool usable_pivot<float>(float v) { return fabsf(v) >= 1.17549435e-38f && isfinite(v); }
template <> __device__ __forceinline__ bool usable_pivot<double>(double v) { return fabs(v) >= 2.2250738585072014e-308 && isfinite(v); }

// FP64 -> FP32, round to nearest even, in integer arithmetic.  GB300 runs the
// hardware conversion on its FP64 units, at a small fraction of the FP32
// rate.  Derived from the IEEE 754 binary64 and binary32 layouts:
//   - round the binary64 encoding at bit 29 (ties to even; a carry into the
//     exponent is correct by construction);
//   - keep the low 9 exponent bits and the top 23 mantissa bits;
//   - rebias the exponent: for binary64 exponents of normal binary32 numbers
//     (897..1150, i.e. 2^-126 <= |v| < 2^128), e - 896 equals the low 8 bits
//     of e with the top bit flipped.
// Branch-free (selects only, so no predicated FP64 instruction is issued):
// magnitudes below 2^-126 become signed zero, 2^128 and above (Inf, NaN
// included) become signed infinity.
__device__ __forceinline__ float d2f_rn(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), mag = hi & 0x7FFFFFFFu, sign = hi & 0x80000000u;
    b += 0x0FFFFFFFull + ((b >> 29) & 1ull);
    const unsigned bits = __funnelshift_l((unsigned)b, (unsigned)(b >> 32), 3);
    unsigned r = ((bits ^ 0x40000000u) & 0x7FFFFFFFu) | sign;
    r = (mag < 0x38100000u) ? sign : r;
    r = (mag >= 0x47F00000u) ? (sign | 0x7F800000u) : r;
    return __int_as_float((int)r);
}
template <typename T> __device__ __forceinline__ T from_f64(double v);
template <> __device__ __forceinline__ float from_f64<float>(double v) { return d2f_rn(v); }
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }

}  // namespace lrs
