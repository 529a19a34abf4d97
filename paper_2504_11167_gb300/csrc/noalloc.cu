// lrspike_residual_noalloc: the FP64 band residual r = f - A x with its
// per-column 2-norms, for callers that must not allocate device memory.
//
// The residual kernel needs scratch beyond its inputs and outputs: one
// partial sum per CTA and column, and a ticket counter for the last-CTA
// reduction.  Here that scratch is a fixed file-scope device array, so the
// call performs no cudaMalloc / cudaFree and no allocating library call.
// Every call on a device shares the array; calls that overlap on the GPU
// (different streams, or different host threads) race on it.
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr int kMaxDevices = 64;
// 65536 partial sums: ceil(n / 256) * nrhs must not exceed this.
constexpr int64_t kPartials = LRSPIKE_NOALLOC_MAX_PARTIALS;

static __device__ __align__(256) double g_partial[kPartials];
static __device__ __align__(256) unsigned int g_counter[64];

struct DeviceScratch {
    bool ready = false;
    double *partial = nullptr;
    unsigned int *counter = nullptr;
};

std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];
lrspike_status err(lrspike_status st, const std::string &m) {
    lrs::set_handleless_error(m);
    return st;
}

// Device memory of GPU `dev` (the current device), or managed memory (which
// every device can reach).  Device memory of another GPU is refused: the
// kernel runs on the current device and would reach it only through peer
// access, if at all.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" lrspike_status lrspike_residual_noalloc(const double *band, int64_t ld_band, int64_t n, int32_t k,
                                                   const double *f, const double *x, double *r,
                                                   int32_t nrhs, int64_t ld, double *norms,
                                                   void *cuda_stream) {
    if (!band || !f || !x || !r || !norms) return err(LRSPIKE_ERR_INVALID_ARG, "NULL pointer argument");
    if (n < 1 || k < 0 || ld < n || ld_band < n || nrhs < 1 || nrhs > 16)
        return err(LRSPIKE_ERR_INVALID_ARG, "need n >= 1, k >= 0, ld >= n, ld_band >= n, 1 <= nrhs <= 16");
    const int64_t ctas = (n + 255) / 256;
    if (ctas * nrhs > kPartials)
        return err(LRSPIKE_ERR_INVALID_ARG,
                   "ceil(n/256) * nrhs exceeds the static scratch of LRSPIKE_NOALLOC_MAX_PARTIALS partial sums");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return err(LRSPIKE_ERR_CUDA, "no usable current CUDA device");
    }
    if (!on_device(band, dev) || !on_device(f, dev) || !on_device(x, dev) || !on_device(r, dev) ||
        !on_device(norms, dev))
        return err(LRSPIKE_ERR_INVALID_ARG,
                   "band, f, x, r and norms must be device memory of the current device (or managed memory)");
    DeviceScratch sc;
    {
        // once per device, with that device current: the device addresses of
        // the static arrays (their host-side names are not device addresses)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_dev[dev].ready) {
            void *pp = nullptr, *pc = nullptr;
            cudaError_t e1 = cudaGetSymbolAddress(&pp, g_partial);
            cudaError_t e2 = cudaGetSymbolAddress(&pc, g_counter);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                cudaGetLastError();
                return err(LRSPIKE_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") +
                                                 cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
            }
            // the ticket counter must start at zero; the last CTA of every
            // launch puts it back to zero, so it is cleared here once, on the
            // first call's stream (the static array starts zeroed at module
            // load as well)
            if (cudaMemsetAsync(pc, 0, sizeof(unsigned int), (cudaStream_t)cuda_stream) != cudaSuccess) {
                cudaGetLastError();
                return err(LRSPIKE_ERR_CUDA, "counter reset failed");
            }
            g_dev[dev].partial = static_cast<double *>(pp);
            g_dev[dev].counter = static_cast<unsigned int *>(pc);
            g_dev[dev].ready = true;
        }
        sc = g_dev[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!lrs::launch_residual_raw(band, ld_band, k, n, f, x, ld, nrhs, r, sc.partial, sc.counter, norms, st))
        return err(LRSPIKE_ERR_CUDA, "residual kernel launch failed");
    lrs::set_handleless_error("");
    return LRSPIKE_OK;
}
