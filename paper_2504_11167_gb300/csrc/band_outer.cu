// The band-restricted outer product of the adjoint (gradient) of a solve:
// for x = A^{-1} f, dL/dA = -lambda x^T with A^T lambda = dL/dx, of which only
// the band entries are parameters.  One thread per (band row d, column j):
// consecutive threads take consecutive columns, so the reads of x, lambda and
// the band write are coalesced; HBM-bound ((2k+1) n 8 bytes written).
#include <string>

#include "internal.h"

namespace lrs {

namespace {

template <int NR>
__global__ void __launch_bounds__(256)
    k_band_outer(const double *__restrict__ lam, const double *__restrict__ x, int nrhs, int64_t ld, int64_t n,
                 int k, double alpha, double *__restrict__ g, int64_t ldg) {
    const int d = blockIdx.y;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = j + d - k;  // A[i][j] = band[(k + i - j) ld + j]
        double v = 0.0;
        if (i >= 0 && i < n) {
#pragma unroll
            for (int q = 0; q < NR; ++q)
                if (q < nrhs) v += lam[q * ld + i] * x[q * ld + j];
            v *= alpha;
        }
        g[(int64_t)d * ldg + j] = v;
    }
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lrspike_status err(lrspike_status st, const std::string &m) {
    set_handleless_error(m);
    return st;
}

}  // namespace

}  // namespace lrs

using lrs::err;

extern "C" lrspike_status lrspike_band_outer(const double *lam, const double *x, int32_t nrhs, int64_t ld, int64_t n,
                                             int32_t k, double alpha, double *grad_band, int64_t ld_band,
                                             void *cuda_stream) {
    if (!lam || !x || !grad_band) return err(LRSPIKE_ERR_INVALID_ARG, "NULL pointer argument");
    if (n < 1 || k < 0 || k > 1024 || nrhs < 1 || nrhs > 16 || ld < n || ld_band < n)
        return err(LRSPIKE_ERR_INVALID_ARG, "need n >= 1, 0 <= k <= 1024, 1 <= nrhs <= 16, ld >= n, ld_band >= n");
    if (!lrs::on_device(lam) || !lrs::on_device(x) || !lrs::on_device(grad_band))
        return err(LRSPIKE_ERR_INVALID_ARG, "lam, x and grad_band must be device memory");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 1024), 2 * k + 1);
    switch (nrhs <= 1 ? 1 : nrhs <= 4 ? 4 : 16) {
        case 1: lrs::k_band_outer<1><<<grid, 256, 0, st>>>(lam, x, nrhs, ld, n, k, alpha, grad_band, ld_band); break;
        case 4: lrs::k_band_outer<4><<<grid, 256, 0, st>>>(lam, x, nrhs, ld, n, k, alpha, grad_band, ld_band); break;
        default: lrs::k_band_outer<16><<<grid, 256, 0, st>>>(lam, x, nrhs, ld, n, k, alpha, grad_band, ld_band); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(LRSPIKE_ERR_CUDA, std::string("band_outer launch failed: ") + cudaGetErrorString(e));
    lrs::set_handleless_error("");
    return LRSPIKE_OK;
}
