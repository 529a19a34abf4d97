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

}  // namespace lrs
