// lrspike_fp64_fma_probe: the FP64 fused multiply-add rate of the current
// GPU, measured with one kernel and CUDA events.  The roofline of the FP64
// residual (the only FP64 arithmetic on the mixed-precision path) divides by
// this measured rate.
//
// Every thread runs 16 independent FMA chains x <- x * a + b (a slightly
// below 1, b small: the values stay bounded, no denormals) for `iters`
// iterations; the grid fills every SM with 8 CTAs of 256 threads, enough
// independent chains to cover the FP64 pipe latency.  A sink write that never
// happens (the flag is zero) keeps the chains live.
#include <string>

#include "internal.h"

namespace {

static __device__ double g_fma_sink[16];

__global__ void __launch_bounds__(256) k_fp64_fma(int64_t iters, double a, double b, int flag) {
    double x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = fma(x[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s += x[j];
    if (flag == 1 && s == 12345.0) g_fma_sink[threadIdx.x & 15] = s;
}

}  // namespace

extern "C" lrspike_status lrspike_fp64_fma_probe(int64_t iters, double *tflops, void *cuda_stream) {
    if (!tflops || iters < 1) {
        lrs::set_handleless_error("need iters >= 1 and an output pointer");
        return LRSPIKE_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        lrs::set_handleless_error("no usable current CUDA device");
        return LRSPIKE_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        lrs::set_handleless_error("event creation failed");
        return LRSPIKE_ERR_CUDA;
    }
    const int blocks = 8 * sms;
    k_fp64_fma<<<blocks, 256, 0, st>>>(iters / 8 + 1, 0.999999, 1e-6, 0);  // warm-up
    cudaEventRecord(e0, st);
    k_fp64_fma<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-6, 0);
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.0f) {
        cudaGetLastError();
        lrs::set_handleless_error(std::string("FMA probe failed: ") + cudaGetErrorString(e));
        return LRSPIKE_ERR_CUDA;
    }
    const double flops = 2.0 * 16.0 * 256.0 * (double)blocks * (double)iters;
    *tflops = flops / (ms * 1e-3) / 1e12;
    lrs::set_handleless_error("");
    return LRSPIKE_OK;
}
