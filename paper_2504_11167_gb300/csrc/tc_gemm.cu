// Batched block products of the wide-band path on the 5th-generation tensor
// cores (tcgen05, sm_103a):
//
//   C_b = alpha * A'_b B'_b^T + beta * C_b,   b = 0..batch-1
//
// A'_b (M x K) and B'_b (N x K) are both K-contiguous ("K-major"): element
// (m, k) of A'_b is at A + b sA + m lda + k.  The wide-band factorisation keeps
// every matrix that enters a product in the layout its product needs (a
// row-major copy for a left factor, the column-major array for a right
// factor), written by the epilogue of the product that made it.
//
// One CTA per 128 x 128 output tile and batch entry, 192 threads:
//   warp 0, one lane : TMA producer.  Per k-block it loads a 128-row x
//                      128-byte slab of A' and of B' (32 TF32 or 64 BF16
//                      values of K per row) with cp.async.bulk.tensor into a
//                      three-deep shared-memory ring, 128-byte swizzled (the
//                      canonical K-major layout of the MMA), out-of-range rows
//                      and K columns zero-filled by the TMA unit;
//   warp 1           : allocates 128 TMEM columns (the FP32 accumulator,
//                      128 lanes x 128 columns); one lane issues
//                      tcgen05.mma (M = 128, N = 128, K = 8 TF32 / 16 BF16 per
//                      instruction) from shared-memory descriptors and frees a
//                      ring slot with tcgen05.commit once its MMAs are done;
//   warps 2..5       : epilogue.  Warp w reads TMEM lanes 32 (w mod 4) ..
//                      +31 (rows of the tile) with tcgen05.ld, applies
//                      alpha / beta and writes the requested outputs: the
//                      FP32 column-major C (beta reads it), a row-major copy
//                      and a column-major copy in the operand type (for
//                      products that use the result as a left or right factor).
// Two CTAs fit on one SM (99 KB of shared memory, 128 TMEM columns each), so
// one CTA's epilogue overlaps the other's main loop.
//
// Every wait on an mbarrier is bounded (about four seconds); a wait that runs
// out sets *err, the CTA waits (again bounded) for its copies and MMAs in
// flight, frees its TMEM and returns.  The host reports *err != 0 as a CUDA
// error of the factorisation.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace lrs {

namespace {

constexpr int TBM = 128, TBN = 128;      // output tile
constexpr int TKB = 128;                 // bytes of K per stage (one swizzle row)
constexpr int TSTAGES = 3;
constexpr int TTHREADS = 192;
constexpr uint32_t TMEM_COLS = 128;
constexpr int A_BYTES = TBM * TKB, B_BYTES = TBN * TKB;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr size_t TSMEM = 1024 + (size_t)TSTAGES * STAGE_BYTES + 256;
constexpr long long kSpinLimit = 1ll << 26;

struct TcParams {
    int M, N, K, nkb;
    float alpha, beta;
    float *f;
    int64_t ldf, sf;
    void *row;
    int64_t ldr, sr;
    int rsplit;
    int64_t rss;
    void *col;
    int64_t ldc, sc;
    float *frow;  // FP32 row-major copy (same index map as row)
    int vec_row;  // 1: the row-major copies may be written with 16-byte stores
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity to complete; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kSpinLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i >= 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzling:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused for this layout, descriptor version 1, layout 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of the same format
// (TF32 = 2, BF16 = 1), both K-major, N = TBN, M = TBM.
template <bool BF16>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) | ((uint32_t)(TBN >> 3) << 17) |
           ((uint32_t)(TBM >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if constexpr (BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

template <typename OpT>
__device__ __forceinline__ OpT to_op(float v);
template <>
__device__ __forceinline__ float to_op<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_op<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Columns nb .. nb+nv-1 of row m (values v) into a row-major copy:
// dst[(n % rsplit) + (n / rsplit) rss + m ldr + b sr].
template <typename OutT>
__device__ __forceinline__ void store_row(OutT *base, const TcParams &P, int b, int m, int nb, int nv,
                                          const float (&v)[32]) {
    OutT *rp = base + (int64_t)b * P.sr + (int64_t)m * P.ldr;
    if (P.vec_row && nv == 32) {
        OutT *dst = rp + (nb % P.rsplit) + (int64_t)(nb / P.rsplit) * P.rss;
        if constexpr (sizeof(OutT) == 2) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                __nv_bfloat162 h0 = __floats2bfloat162_rn(v[j], v[j + 1]);
                __nv_bfloat162 h1 = __floats2bfloat162_rn(v[j + 2], v[j + 3]);
                __nv_bfloat162 h2 = __floats2bfloat162_rn(v[j + 4], v[j + 5]);
                __nv_bfloat162 h3 = __floats2bfloat162_rn(v[j + 6], v[j + 7]);
                uint4 u;
                u.x = *reinterpret_cast<uint32_t *>(&h0);
                u.y = *reinterpret_cast<uint32_t *>(&h1);
                u.z = *reinterpret_cast<uint32_t *>(&h2);
                u.w = *reinterpret_cast<uint32_t *>(&h3);
                *reinterpret_cast<uint4 *>(dst + j) = u;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4 *>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < nv) {
                const int n = nb + j;
                rp[(n % P.rsplit) + (int64_t)(n / P.rsplit) * P.rss] = to_op<OutT>(v[j]);
            }
    }
}

template <bool BF16>
__global__ void __launch_bounds__(TTHREADS, 2)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const TcParams P) {
    using OpT = typename std::conditional<BF16, __nv_bfloat16, float>::type;
    constexpr int KELEM = TKB / (int)sizeof(OpT);  // K values per stage
    constexpr int KSTEP = BF16 ? 16 : 8;           // K per MMA instruction (32 bytes)
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base, *sB = base + TSTAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(base + TSTAGES * STAGE_BYTES);
    uint64_t *empty = full + TSTAGES, *accum = empty + TSTAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN, b = blockIdx.z;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nkb = P.nkb;

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
            int issued = 0;
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % TSTAGES;
                const uint32_t ph = (uint32_t)(kb / TSTAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_3d(sA + s * A_BYTES, &mapA, &full[s], kb * KELEM, m0, b);
                tma_load_3d(sB + s * B_BYTES, &mapB, &full[s], kb * KELEM, n0, b);
                ++issued;
            }
            if (!ok) {
                atomicExch(P.err, 1);
                // the loads still in flight land before the CTA leaves
                for (int kb = issued > TSTAGES ? issued - TSTAGES : 0; kb < issued; ++kb)
                    mbar_wait(&full[kb % TSTAGES], (uint32_t)(kb / TSTAGES) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc<BF16>();
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % TSTAGES;
                const uint32_t ph = (uint32_t)(kb / TSTAGES) & 1u;
                if (!mbar_wait(&full[s], ph)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
                for (int kk = 0; kk < KELEM / KSTEP; ++kk)
                    mma_issue<BF16>(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                                    (kb | kk) != 0 ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            // completes once every MMA issued above has (also after a failed wait)
            mma_commit(accum);
            if (!ok) atomicExch(P.err, 1);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int m = m0 + 32 * q + lane;
        bool ok = mbar_wait(accum, 0);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) atomicExch(P.err, 1);
        } else {
            tc_fence_after();
            const bool mrow = m < P.M;
            const int ncb = min(TBN, P.N - n0);
            for (int c = 0; c < TBN / 32; ++c) {
                if (c * 32 >= ncb) break;  // warp-uniform
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * 32), v);
                if (!mrow) continue;
                const int nb = n0 + c * 32;
                const int nv = min(32, P.N - nb);
                if (P.f) {
                    float *fp = P.f + (int64_t)b * P.sf + m;
                    if (P.beta != 0.0f) {
                        // all 32 reads of C before the first write of the
                        // same array, so they are in flight together
                        float cin[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) cin[j] = (j < nv) ? fp[(int64_t)(nb + j) * P.ldf] : 0.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaf(P.beta, cin[j], P.alpha * v[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] *= P.alpha;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j < nv) fp[(int64_t)(nb + j) * P.ldf] = v[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] *= P.alpha;
                }
                if (P.row) store_row<OpT>(reinterpret_cast<OpT *>(P.row), P, b, m, nb, nv, v);
                if (P.frow) store_row<float>(P.frow, P, b, m, nb, nv, v);
                if (P.col) {
                    OpT *cp = reinterpret_cast<OpT *>(P.col) + (int64_t)b * P.sc + m;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j < nv) cp[(int64_t)(nb + j) * P.ldc] = to_op<OpT>(v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // every MMA has completed once accum has (the epilogue waited on it; a
        // failed epilogue wait is repeated here, bounded)
        if (lane == 0) mbar_wait(accum, 0);
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a K-major operand: dims {K, rows, batch}, box {128 bytes of K, 128 rows, 1}.
bool make_map(CUtensorMap *map, bool bf16, const GemmOperand &o, int K, int rows, int batch, std::string *err) {
    const int64_t es = bf16 ? 2 : 4;
    auto fn = encode_fn();
    if (!fn) {
        *err = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    const int64_t sb = (batch > 1) ? o.s : o.ld * rows;
    if ((reinterpret_cast<uintptr_t>(o.p) & 15) || (o.ld * es) % 16 || (sb * es) % 16 || o.ld < K) {
        *err = "tensor-core GEMM operand is not 16-byte aligned or its leading dimension is below K";
        return false;
    }
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(o.ld * es), (cuuint64_t)(sb * es)};
    cuuint32_t box[3] = {(cuuint32_t)(TKB / es), (cuuint32_t)TBM, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r =
        fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(o.p),
           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed with status " + std::to_string((int)r);
        return false;
    }
    return true;
}

}  // namespace

bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                       const cuuint64_t *strides, const cuuint32_t *box, const cuuint32_t *estr, std::string *err) {
    auto fn = encode_fn();
    if (!fn) {
        *err = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    if (reinterpret_cast<uintptr_t>(base) & 15) {
        *err = "tensor map base is not 16-byte aligned";
        return false;
    }
    const CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed with status " + std::to_string((int)r);
        return false;
    }
    return true;
}

bool tc_gemm(cudaStream_t st, bool bf16, int M, int N, int K, int batch, float alpha, const GemmOperand &A,
             const GemmOperand &B, float beta, const GemmOutput &C, int *err_dev, std::string *err) {
    if (M <= 0 || N <= 0 || batch <= 0) return true;
    if (K <= 0 || (beta != 0.0f && !C.f) || batch > 65535 || (N + TBN - 1) / TBN > 65535) {
        *err = "tensor-core GEMM: bad arguments";
        return false;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, bf16, A, K, M, batch, err) || !make_map(&mb, bf16, B, K, N, batch, err)) return false;
    const int64_t es = bf16 ? 2 : 4;
    TcParams P{};
    P.M = M;
    P.N = N;
    P.K = K;
    P.nkb = (int)((K * es + TKB - 1) / TKB);
    P.alpha = alpha;
    P.beta = beta;
    P.f = C.f;
    P.ldf = C.ldf;
    P.sf = C.sf;
    P.row = C.row;
    P.ldr = C.ldr;
    P.sr = C.sr;
    P.rsplit = C.rsplit > 0 ? C.rsplit : (1 << 30);
    P.rss = C.rss;
    P.col = C.col;
    P.ldc = C.ldc;
    P.sc = C.sc;
    P.frow = C.frow;
    // 16-byte row stores need every row start 16-byte aligned in both copies
    auto vec_ok = [&](const void *ptr, int64_t e) {
        return !ptr || ((reinterpret_cast<uintptr_t>(ptr) & 15) == 0 && (C.ldr * e) % 16 == 0 && (C.sr * e) % 16 == 0 &&
                        (C.rsplit <= 0 || (C.rsplit % 32 == 0 && (C.rss * e) % 16 == 0)));
    };
    P.vec_row = (vec_ok(C.row, es) && vec_ok(C.frow, 4)) ? 1 : 0;
    P.err = err_dev;
    const dim3 grid((unsigned)((M + TBM - 1) / TBM), (unsigned)((N + TBN - 1) / TBN), (unsigned)batch);
    // the shared-memory opt-in is a per-device attribute of each kernel
    static std::mutex mu;
    static bool ready[2][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64 && !ready[bf16][dev]) {
            cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TSMEM);
            cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TSMEM);
            ready[bf16][dev] = true;
        }
    }
    if (bf16)
        k_tc_gemm<true><<<grid, TTHREADS, TSMEM, st>>>(ma, mb, P);
    else
        k_tc_gemm<false><<<grid, TTHREADS, TSMEM, st>>>(ma, mb, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("tensor-core GEMM launch failed: ") + cudaGetErrorString(e);
        return false;
    }
    return true;
}

}  // namespace lrs
