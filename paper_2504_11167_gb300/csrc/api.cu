// Host side of the C ABI declared in lrspike.h: option checks, workspace
// sizing, the factorisation pipeline, and the FP64 outer iteration that uses
// the LR-SPIKE operator as its preconditioner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace lrs {

const char *const kKernelNames[KID_COUNT] = {
    "band_lu",      "spike_rhs",   "spike_sweep", "gram",
    "gram_reduce",  "coupling_gram", "jacobi",      "make_u",      "reduced_build",
    "reduced_factor", "norm",        "residual",    "dstage",      "reduced_solve",
    "retrieve",     "project_t",     "dstage_t",    "bicgstab_vector", "matvec",
    "wide_gather",  "wide_gemm_simt", "wide_lu64",  "wide_vector", "wide_gemm_tc", "wide_cholqr", "wide_dstage",
    "nonzero_diagonals", "band_lu_inv", "otf"};

static cudaEvent_t take_event(Ctx *c) {
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool begin_launch(Ctx *c, int kid, cudaEvent_t *ev_end) {
    *ev_end = nullptr;
    if (c->profile) {
        cudaEvent_t a = take_event(c), b = take_event(c);
        cudaEventRecord(a, c->stream);
        c->pending.push_back({kid, a, b});
        *ev_end = b;
    }
    return true;
}

bool end_launch(Ctx *c, int kid, cudaEvent_t ev_end) {
    const cudaError_t e = cudaGetLastError();
    if (ev_end) cudaEventRecord(ev_end, c->stream);
    c->launches++;
    c->kcount[kid]++;
    if (e != cudaSuccess) {
        c->err = std::string("launch of ") + kKernelNames[kid] + " failed: " + cudaGetErrorString(e);
        return false;
    }
    return true;
}

static void drain_profile(Ctx *c) {
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &pd : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pd.a, pd.b) == cudaSuccess) c->kms[pd.kid] += ms;
        c->free_events.push_back(pd.a);
        c->free_events.push_back(pd.b);
    }
    c->pending.clear();
}

}  // namespace lrs

using namespace lrs;

static thread_local std::string g_err;
static const int64_t kNoStatus = INT64_MAX;
static const int64_t kReducedSingular = INT64_MAX - 1;

void lrs::set_handleless_error(const std::string &msg) { g_err = msg; }

static lrspike_status fail(Ctx *c, lrspike_status st, const std::string &msg) {
    if (c) c->err = msg;
    else g_err = msg;
    return st;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename P>
static bool dalloc(P **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return true;
    return cudaMalloc((void **)ptr, bytes) == cudaSuccess;
}

static void free_all(Ctx *c) {
    void *ptrs[] = {c->off_d, c->boff_d, c->LT,   c->UT,  c->DI,   c->X,     c->Ucat,
                    c->PQ,    c->Gram,   c->Gpart, c->sigma, c->E, c->F,    c->Gs,    c->Rinv,
                    c->rv,     c->Yv,   c->Gv,  c->psi,  c->zr,   c->wr,    c->nrm,
                    c->partial, c->counter, c->status, c->stopf, c->band_own, c->io_f, c->io_x, c->dots,
                    c->bpartial, c->PF, c->PIVP, c->ocv, c->og, c->orv, c->osc, c->oone, c->xalt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (double *p : c->bv)
        if (p) cudaFree(p);
    for (auto &b : c->bcr)
        for (double *p : {b.E, b.F, b.G, b.Einv, b.al, b.be})
            if (p) cudaFree(p);
    wide_free(c);
    if (c->host) cudaFreeHost(c->host);
    for (auto &pd : c->pending) {
        cudaEventDestroy(pd.a);
        cudaEventDestroy(pd.b);
    }
    for (auto e : c->free_events) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    for (auto e : c->grp_ev) cudaEventDestroy(e);
    for (auto st : c->grp_streams) cudaStreamDestroy(st);
    if (c->ev_up) cudaEventDestroy(c->ev_up);
    if (c->ev_strips) cudaEventDestroy(c->ev_strips);
    if (c->up) cudaStreamDestroy(c->up);
}

// A host band is uploaded in groups of partitions overlapped with the band LU
// when the LU is the column kernel (unpivoted, FP32 / FP64 working precision,
// k <= 64) and there are partitions to overlap.
static bool upload_pipelined(const Ctx *c) {
    // (a profiling handle times every launch on the handle's stream: one LU)
    return !c->wide && !c->opt.pivoting && c->opt.precision != LRSPIKE_MIXED_TF32 && c->p >= 2 && !c->profile;
}

static int upload_groups(const Ctx *c) { return std::min(c->p, 16); }

static bool upload_setup(Ctx *c) {
    if (c->up) return true;
    const int G = upload_groups(c);
    bool ok = cudaStreamCreateWithFlags(&c->up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->ev_up, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->ev_strips, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; ok && g < G; ++g) {
        cudaStream_t st = nullptr;
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) c->grp_streams.push_back(st);
    }
    for (int e = 0; ok && e < 2 * G; ++e) {
        cudaEvent_t ev = nullptr;
        ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) c->grp_ev.push_back(ev);
    }
    return ok;
}

// Enqueues the upload of a host band into band_own on the upload stream (after
// the handle's earlier work): with a coupling branch first the 2k columns
// around every interface (B_i, C_i; event ev_strips), then the partition
// groups' columns, each followed by its event grp_ev[2g].  Every column range
// is a pitched copy of the 2k+1 band rows.  The group copies rewrite the
// interface columns with the same bytes.
static bool upload_band(Ctx *c, const double *band, int64_t ld) {
    const int G = upload_groups(c), rows = 2 * c->k + 1;
    auto copy_cols = [&](int64_t c0, int64_t c1) {
        return c1 <= c0 || cudaMemcpy2DAsync(c->band_own + c0, ld * 8, band + c0, ld * 8, (size_t)(c1 - c0) * 8,
                                             rows, cudaMemcpyHostToDevice, c->up) == cudaSuccess;
    };
    if (cudaEventRecord(c->ev_up, c->stream) != cudaSuccess || cudaStreamWaitEvent(c->up, c->ev_up, 0) != cudaSuccess)
        return false;
    if (c->side) {
        for (int i = 1; i < c->p; ++i) {
            const int64_t e = c->off_h[i];
            if (!copy_cols(std::max<int64_t>(0, e - c->k), std::min<int64_t>(c->n, e + c->k))) return false;
        }
        if (cudaEventRecord(c->ev_strips, c->up) != cudaSuccess) return false;
    }
    for (int g = 0; g < G; ++g) {
        const int g0 = (int)((int64_t)g * c->p / G), g1 = (int)((int64_t)(g + 1) * c->p / G);
        if (!copy_cols(c->off_h[g0], c->off_h[g1]) || cudaEventRecord(c->grp_ev[2 * g], c->up) != cudaSuccess)
            return false;
    }
    return true;
}

// The band LU of each partition group, then its triangular inverses, on the
// group's own stream after the group's upload; the handle's stream waits for
// all of them.  (A device band keeps one LU launch over all partitions:
// sixteen concurrent group launches of the same CTAs measured slower.)
static bool band_lu_grouped(Ctx *c) {
    const int G = upload_groups(c);
    cudaStream_t own = c->stream;
    bool ok = true;
    for (int g = 0; ok && g < G; ++g) {
        cudaStream_t st = c->grp_streams[g];
        c->lu_g0 = (int)((int64_t)g * c->p / G);
        c->lu_g1 = (int)((int64_t)(g + 1) * c->p / G);
        ok = cudaStreamWaitEvent(st, c->grp_ev[2 * g], 0) == cudaSuccess;
        c->stream = st;
        ok = ok && run_band_lu(c);
        c->stream = own;
        ok = ok && cudaEventRecord(c->grp_ev[2 * g + 1], st) == cudaSuccess &&
             cudaStreamWaitEvent(own, c->grp_ev[2 * g + 1], 0) == cudaSuccess;
    }
    c->lu_g0 = 0;
    c->lu_g1 = -1;
    return ok;
}

extern "C" lrspike_status lrspike_options_default(lrspike_options *o, int64_t n, int32_t k, int32_t p,
                                                  int32_t r) {
    if (!o) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "options pointer is NULL");
    std::memset(o, 0, sizeof(*o));
    o->n = n;
    o->k = k;
    o->p = p;
    o->r = r;
    o->precision = LRSPIKE_FP64;
    o->pivoting = 0;
    o->compress = LRSPIKE_COMPRESS_SPIKE;
    o->reduced = LRSPIKE_REDUCED_FULL;
    o->outer = LRSPIKE_OUTER_IR;
    o->max_iter = 50;
    o->tol = 1e-12;
    o->rank_tol = 1e-13;
    o->max_nrhs = 16;
    o->profile = 0;
    o->oversample = r;
    o->power_iters = 2;
    o->seed = 0x4C52535049ull;
    o->graph_safe = 0;
    o->block = 0;
    o->otf_tol = 1e-8;
    o->otf_max_iter = 100;
    return LRSPIKE_OK;
}

extern "C" lrspike_status lrspike_create(const lrspike_options *opt, void *stream, lrspike_handle *out) {
    if (!opt || !out) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "NULL options or output pointer");
    *out = nullptr;
    const lrspike_options &o = *opt;
    if (o.n < 1) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "n must be >= 1");
    if (o.k < 0 || o.k > 1024) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "k must be in 0..1024");
    if (o.p < 1 || o.p > o.n) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "p must be in 1..n");
    if (o.r < 0 || o.r > o.k) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "r must be in 0..k");
    if (o.max_nrhs < 1 || o.max_nrhs > 16)
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "max_nrhs must be in 1..16");
    if (o.precision < LRSPIKE_FP64 || o.precision > LRSPIKE_MIXED_BF16 || o.compress < 0 || o.compress > 1 ||
        o.reduced < 0 || o.reduced > 2 || o.outer < 0 || o.outer > 2 || o.pivoting < 0 || o.pivoting > 1)
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "unknown enum value in options");
    if (o.max_iter < 0 || !(o.tol >= 0.0) || !(o.rank_tol >= 0.0))
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "max_iter, tol and rank_tol must be >= 0");
    const bool wide = o.k > 64;
    if (o.graph_safe && (o.outer == LRSPIKE_OUTER_BICGSTAB || wide))
        return fail(nullptr, LRSPIKE_ERR_UNSUPPORTED, "graph_safe supports outer IR or NONE with k <= 64");
    if (o.graph_safe && o.profile)
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "graph_safe handles cannot profile (no host reads)");
    if (o.block != 0 && (wide || (o.block != 8 && o.block != 16 && o.block != 32 && o.block != 64) || o.block < o.k))
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "block must be 8, 16, 32 or 64 and >= k (k <= 64)");
    if (wide && (o.pivoting || o.compress != LRSPIKE_COMPRESS_SPIKE))
        return fail(nullptr, LRSPIKE_ERR_UNSUPPORTED, "k > 64 supports SPIKE compression without pivoting");
    if (wide && (o.oversample < 0 || o.power_iters < 0))
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "oversample and power_iters must be >= 0");
    if (wide && o.p > 1 && o.r > 0 &&
        std::min(o.k, o.r + o.oversample) > (o.precision == LRSPIKE_FP64 ? 64 : 128))
        return fail(nullptr, LRSPIKE_ERR_UNSUPPORTED,
                    "min(k, r + oversample) sketch columns beyond 64 (FP64) / 128 (mixed) is not built");
    if (!wide && o.precision == LRSPIKE_MIXED_BF16)
        return fail(nullptr, LRSPIKE_ERR_UNSUPPORTED, "BF16 operands are built for the wide-band path (k > 64)");
    // reduced-system blocks of 2r x 2r: up to 64 (every path), up to 128 for
    // wide bands with the truncated reduced system
    if (o.r > 32 && !(wide && o.r <= 64 && o.reduced == LRSPIKE_REDUCED_TRUNCATED))
        return fail(nullptr, LRSPIKE_ERR_UNSUPPORTED,
                    "r > 32 is built for k > 64 with the truncated reduced system (r <= 64)");
    if (o.reduced == LRSPIKE_REDUCED_OTF) {
        if (o.p < 2 || o.r < 1)
            return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "the OTF reduced system needs p >= 2 and r >= 1");
        if (o.pivoting || o.graph_safe || o.outer == LRSPIKE_OUTER_BICGSTAB)
            return fail(nullptr, LRSPIKE_ERR_UNSUPPORTED,
                        "OTF is built without pivoting, for outer IR or NONE, not graph_safe");
    }
    if (!(o.otf_tol > 0.0) || o.otf_max_iter < 1)
        return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "otf_tol must be > 0 and otf_max_iter >= 1");

    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return fail(nullptr, LRSPIKE_ERR_OOM, "host allocation failed");
    c->opt = o;
    if (o.reduced == LRSPIKE_REDUCED_OTF) {  // factorised as TRUNCATED (its preconditioner)
        c->otf = true;
        c->opt.reduced = LRSPIKE_REDUCED_TRUNCATED;
    }
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    c->n = o.n;
    c->k = o.k;
    c->p = o.p;
    c->r = (o.p > 1) ? o.r : 0;  // one partition has no spikes and no reduced system
    c->KB = 8;
    while (c->KB < o.k) c->KB *= 2;
    c->wide = wide;
    if (wide) c->KB = 64 * ((o.k + 63) / 64);  // W, the wide-band block size
    if (o.block > c->KB) c->KB = o.block;
    c->fp64 = (o.precision == LRSPIKE_FP64);
    c->tsize = c->fp64 ? 8 : 4;
    c->profile = o.profile != 0;
    // partitions (first n mod p get one extra row) and their blocks
    c->off_h.resize(c->p + 1);
    c->boff_h.resize(c->p + 1);
    c->off_h[0] = 0;
    c->boff_h[0] = 0;
    const int64_t base = c->n / c->p, extra = c->n % c->p;
    int64_t minnb = INT64_MAX;
    for (int i = 0; i < c->p; ++i) {
        const int64_t ni = base + (i < extra ? 1 : 0);
        if (c->p > 1 && ni <= c->k) {
            delete c;
            return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "every partition needs n_i > k (use fewer partitions)");
        }
        c->off_h[i + 1] = c->off_h[i] + ni;
        const int64_t nb = (ni + c->KB - 1) / c->KB;
        c->boff_h[i + 1] = c->boff_h[i] + nb;
        c->maxni = std::max(c->maxni, ni);
        minnb = std::min(minnb, nb);
    }
    c->NB = c->boff_h[c->p];
    const bool spikes = (c->p > 1 && c->r > 0);
    // spike panel columns: a multiple of 16 (the register-tiled sweep's column
    // groups); T_i in the first half, W_i in the second half
    c->m = spikes ? (o.compress == LRSPIKE_COMPRESS_COUPLING ? 16 * ((2 * c->r + 15) / 16) : 2 * c->KB) : 0;
    if (wide) c->m = 0;
    if (c->m == 48) c->m = 64;  // column groups of 1, 2, 4 or 8
    c->gram_chunks = (int)std::max<int64_t>(1, std::min<int64_t>(32, minnb));
    const size_t T = c->tsize, KB = c->KB, NB = c->NB, mx = o.max_nrhs;
    const size_t n2 = 2 * c->r, ni = (size_t)std::max(0, c->p - 1);
    const int64_t rb = (c->n + 255) / 256;
    const bool piv = o.pivoting != 0;
    bool ok = dalloc(&c->off_d, (c->p + 1) * 8) && dalloc(&c->boff_d, (c->p + 1) * 8) &&
              (wide ? true
               : piv ? dalloc(&c->PF, NB * 5 * KB * KB * T) && dalloc(&c->PIVP, NB * 2 * KB)
                     : dalloc(&c->LT, NB * KB * KB * T) && dalloc(&c->UT, NB * KB * KB * T) &&
                           dalloc(&c->DI, NB * KB * T)) &&
              dalloc(&c->rv, (size_t)c->n * mx * 8) && dalloc(&c->Yv, (size_t)c->n * mx * T) &&
              dalloc(&c->Gv, (size_t)c->n * mx * T) && dalloc(&c->nrm, 4 * mx * 8) &&
              dalloc(&c->partial, (size_t)rb * mx * 8) && dalloc(&c->counter, 64) && dalloc(&c->status, 64) &&
              dalloc(&c->stopf, 16);
    if (ok && spikes) {
        ok = (wide ? true
                   : dalloc(&c->X, NB * KB * c->m * T) && dalloc(&c->Gram, (size_t)c->p * 2 * KB * KB * 8) &&
                         dalloc(&c->Gpart, (size_t)c->p * c->gram_chunks * 2 * KB * KB * 8)) &&
             dalloc(&c->Ucat, (size_t)c->n * n2 * T) && dalloc(&c->PQ, (size_t)c->p * 2 * c->r * KB * T) &&
             dalloc(&c->sigma, (size_t)c->p * 2 * c->r * 8) && dalloc(&c->E, ni * n2 * n2 * 8) &&
             dalloc(&c->F, ni * n2 * n2 * 8) && dalloc(&c->Gs, ni * n2 * n2 * 8) &&
             dalloc(&c->Rinv, ni * n2 * n2 * 8) &&
             dalloc(&c->psi, ni * n2 * mx * 8) && dalloc(&c->zr, ni * n2 * mx * 8) &&
             dalloc(&c->wr, ni * n2 * mx * 8);
    }
    if (ok && spikes && o.reduced == LRSPIKE_REDUCED_FULL)
        for (int t = 0; t < 2 && ok; ++t)
            for (double **q : {&c->bcr[t].E, &c->bcr[t].F, &c->bcr[t].G, &c->bcr[t].Einv, &c->bcr[t].al, &c->bcr[t].be})
                ok = ok && dalloc(q, ni * n2 * n2 * 8);
    if (ok && o.outer == LRSPIKE_OUTER_BICGSTAB) ok = bicgstab_alloc(c);
    if (ok && c->otf) ok = otf_alloc(c);
    // fused retrieval + residual in the IR loop: rows of one CTA (256) and its
    // 2k halo rows may span at most two partitions
    if (ok && !wide && !piv && !c->otf && !o.graph_safe && o.outer == LRSPIKE_OUTER_IR &&
        c->n / c->p >= 256 + 2 * (int64_t)c->k)
        ok = dalloc(&c->xalt, (size_t)c->n * 8);
    if (ok && wide) ok = wide_setup(c);
    if (ok) ok = cudaMallocHost((void **)&c->host, (8 * mx + 8) * 8) == cudaSuccess;
    if (ok && spikes && !wide && o.compress == LRSPIKE_COMPRESS_COUPLING)
        ok = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return fail(nullptr, LRSPIKE_ERR_OOM, "device or pinned allocation failed");
    }
    cudaMemcpy(c->off_d, c->off_h.data(), (c->p + 1) * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(c->boff_d, c->boff_h.data(), (c->p + 1) * 8, cudaMemcpyHostToDevice);
    cudaMemset(c->counter, 0, 64);
    cudaMemset(c->stopf, 0, 16);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(nullptr, LRSPIKE_ERR_CUDA, std::string("CUDA error at create: ") + cudaGetErrorString(e));
    }
    *out = reinterpret_cast<lrspike_handle>(c);
    return LRSPIKE_OK;
}

static Ctx *ctx(lrspike_handle h) { return reinterpret_cast<Ctx *>(h); }

static lrspike_status cuda_fail(Ctx *c, const char *what) {
    const cudaError_t e = cudaGetLastError();
    return fail(c, LRSPIKE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

__global__ void k_set_status(int64_t *s, int64_t v) { *s = v; }

extern "C" lrspike_status lrspike_factor(lrspike_handle h, const double *band, int64_t ld) {
    Ctx *c = ctx(h);
    if (!c) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "NULL handle");
    c->err.clear();
    if (!band || ld < c->n) return fail(c, LRSPIKE_ERR_INVALID_ARG, "band is NULL or ld < n");
    cudaSetDevice(c->device);
    c->factored = false;
    const bool gs = c->opt.graph_safe != 0;  // enqueue only: no host reads, no synchronisation
    bool piped = false;  // host band uploaded in groups beside the band LU
    if (gs || is_device_ptr(band)) {
        c->band = band;
    } else {
        const size_t bytes = (size_t)(2 * c->k + 1) * ld * 8;
        if (c->band_own_bytes < bytes) {
            if (c->band_own) cudaFree(c->band_own);
            c->band_own = nullptr;
            c->band_own_bytes = 0;
            if (!dalloc(&c->band_own, bytes)) return fail(c, LRSPIKE_ERR_OOM, "band copy allocation failed");
            c->band_own_bytes = bytes;
        }
        piped = upload_pipelined(c);
        if (piped) {
            if (!upload_setup(c)) return cuda_fail(c, "upload stream creation");
        } else if (cudaMemcpyAsync(c->band_own, band, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            return cuda_fail(c, "band host-to-device copy");
        }
        c->band = c->band_own;
    }
    c->ld = ld;
    if (gs) {
        k_set_status<<<1, 1, 0, c->stream>>>(c->status, kNoStatus);
        if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, "status reset");
    } else {
        *(int64_t *)c->host = kNoStatus;
        if (cudaMemcpyAsync(c->status, c->host, 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return cuda_fail(c, "status reset");
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_fail(c, "stream sync");
    }
    if (piped && !upload_band(c, band, ld)) return cuda_fail(c, "band host-to-device copy");
    bool ok;
    if (c->side) {
        // Coupling compression: the Gram matrices of B_i and C_i, their
        // eigenvectors and the spike right-hand sides need the band only, so
        // they run on the side stream while the band LU (one CTA per
        // partition, SMs not full) runs on the handle's stream; the spike
        // sweep waits for both.  The LU is enqueued first.
        // (a host band: the side stream starts once the interface columns have
        // landed, the LU per partition group as its columns land)
        if (piped)
            ok = band_lu_grouped(c) && cudaStreamWaitEvent(c->side, c->ev_strips, 0) == cudaSuccess;
        else
            ok = cudaEventRecord(c->ev_fork, c->stream) == cudaSuccess && run_band_lu(c) &&
                 cudaStreamWaitEvent(c->side, c->ev_fork, 0) == cudaSuccess;
        if (ok) {
            cudaStream_t own = c->stream;
            c->stream = c->side;
            ok = run_coupling_gram(c) && run_jacobi(c) && run_spike_rhs(c);
            c->stream = own;
            ok = ok && cudaEventRecord(c->ev_join, c->side) == cudaSuccess &&
                 cudaStreamWaitEvent(c->stream, c->ev_join, 0) == cudaSuccess;
        }
        ok = ok && run_sweep(c) && run_make_u(c) && run_reduced_build(c) && run_reduced_factor(c);
    } else {
        ok = c->wide ? run_wide_factor(c) : piped ? band_lu_grouped(c) : run_band_lu(c);
        if (ok && !c->wide && c->p > 1 && c->r > 0) {
            if (c->opt.compress == LRSPIKE_COMPRESS_COUPLING)
                ok = run_coupling_gram(c) && run_jacobi(c) && run_spike_rhs(c) && run_sweep(c) && run_make_u(c);
            else
                ok = run_spike_rhs(c) && run_sweep(c) && run_gram(c) && run_jacobi(c) && run_make_u(c);
            ok = ok && run_reduced_build(c) && run_reduced_factor(c);
        }
    }
    if (!ok) return fail(c, LRSPIKE_ERR_CUDA, c->err);
    c->bcr_t_ready = gs;  // also after a replayed factorisation graph
    if (gs) {  // the status is read by lrspike_finish
        c->factored = true;
        c->last_nrhs = 0;
        return LRSPIKE_OK;
    }
    if (cudaMemcpyAsync(c->host, c->status, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return cuda_fail(c, "factorisation");
    const int64_t st = *(int64_t *)c->host;
    if (st == kReducedSingular) return fail(c, LRSPIKE_ERR_SINGULAR, "singular reduced system block");
    if (st != kNoStatus) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "zero or non-finite pivot at global row %lld", (long long)st);
        return fail(c, LRSPIKE_ERR_SINGULAR, buf);
    }
    c->factored = true;
    return LRSPIKE_OK;
}

static lrspike_status solve_common(Ctx *c, const double *f, double *x, int nrhs, int64_t ld,
                                   lrspike_info *info, bool trans) {
    if (!c) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "NULL handle");
    c->err.clear();
    if (!c->factored) return fail(c, LRSPIKE_ERR_STATE, "solve called without a successful factor");
    if (!f || !x || nrhs < 1 || nrhs > c->opt.max_nrhs || ld < c->n)
        return fail(c, LRSPIKE_ERR_INVALID_ARG, "bad f/x pointer, nrhs or ld");
    const size_t span = (size_t)((nrhs - 1) * ld + c->n) * 8;
    if ((const char *)x < (const char *)f + span && (const char *)f < (const char *)x + span)
        return fail(c, LRSPIKE_ERR_INVALID_ARG, "x must not alias f");
    cudaSetDevice(c->device);
    if (c->opt.graph_safe) {
        // device buffers; exactly max_iter refinement steps (NONE: one application);
        // the final residual stays on the device for lrspike_finish
        // up to max_iter steps enqueued; with outer IR the residual that meets
        // tol raises a device flag and the kernels of the remaining steps
        // return at entry (the norms of that residual stay for lrspike_finish)
        const bool none = c->opt.outer == LRSPIKE_OUTER_NONE;
        const int steps = none ? 1 : c->opt.max_iter;
        struct Reset {  // the rule is enqueue-time state of this call only
            Ctx *c;
            ~Reset() { c->stop = StopRule(); c->skip = nullptr; }
        } reset{c};
        if (cudaMemset2DAsync(x, ld * 8, 0, c->n * 8, nrhs, c->stream) != cudaSuccess) return cuda_fail(c, "x reset");
        if (cudaMemsetAsync(c->stopf, 0, 2 * sizeof(int), c->stream) != cudaSuccess) return cuda_fail(c, "flag reset");
        if (!run_norms(c, f, ld, nrhs, c->nrm)) return fail(c, LRSPIKE_ERR_CUDA, c->err);
        if (!none) {
            c->stop.flag = c->stopf;
            c->stop.fnrm = c->nrm;
            c->stop.tol = c->opt.tol;
            c->stop.count = 1;
            c->skip = c->stopf;
        }
        for (int it = 0; it < steps; ++it)
            if (!run_residual(c, f, x, ld, nrhs, trans, it == 0) ||
                !apply_precond(c, c->rv, x, ld, nrhs, trans, true))
                return fail(c, LRSPIKE_ERR_CUDA, c->err);
        c->stop.count = 0;
        if (!run_residual(c, f, x, ld, nrhs, trans, false)) return fail(c, LRSPIKE_ERR_CUDA, c->err);
        c->last_nrhs = nrhs;
        if (info) {
            info->iterations = steps;
            info->converged = 0;
            info->max_rel_residual = NAN;
        }
        return LRSPIKE_OK;
    }
    c->otf_iters = 0;
    const bool fdev = is_device_ptr(f), xdev = is_device_ptr(x);
    if (fdev != xdev) return fail(c, LRSPIKE_ERR_INVALID_ARG, "f and x must both be device or both host");
    const double *fd = f;
    double *xd = x;
    int64_t ldd = ld;
    if (!fdev) {
        const size_t bytes = (size_t)c->n * nrhs * 8;
        if (c->io_bytes < bytes) {
            if (c->io_f) cudaFree(c->io_f);
            if (c->io_x) cudaFree(c->io_x);
            c->io_f = c->io_x = nullptr;
            c->io_bytes = 0;
            if (!dalloc(&c->io_f, bytes) || !dalloc(&c->io_x, bytes))
                return fail(c, LRSPIKE_ERR_OOM, "solve staging allocation failed");
            c->io_bytes = bytes;
        }
        if (cudaMemcpy2DAsync(c->io_f, c->n * 8, f, ld * 8, c->n * 8, nrhs, cudaMemcpyHostToDevice,
                              c->stream) != cudaSuccess)
            return cuda_fail(c, "f host-to-device copy");
        fd = c->io_f;
        xd = c->io_x;
        ldd = c->n;
    }
    const int mx = c->opt.max_nrhs;
    if (cudaMemset2DAsync(xd, ldd * 8, 0, c->n * 8, nrhs, c->stream) != cudaSuccess)
        return cuda_fail(c, "x reset");
    const int outer = c->opt.outer;
    double *hf = c->host, *hr = c->host + mx;
    // |f|: BiCGStab reads it before its first step; the IR loop takes it from
    // its first residual (x = 0: r = f, the same reduction)
    if (outer == LRSPIKE_OUTER_BICGSTAB) {
        if (!run_norms(c, fd, ldd, nrhs, c->nrm)) return fail(c, LRSPIKE_ERR_CUDA, c->err);
        if (cudaMemcpyAsync(hf, c->nrm, nrhs * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return cuda_fail(c, "norm read");
    }
    const int max_it = (outer == LRSPIKE_OUTER_NONE) ? 1 : c->opt.max_iter;
    std::vector<double> hist;
    int it = 0;
    bool converged = false, stalled = false;
    std::vector<double> rel(nrhs, 0.0);
    if (outer == LRSPIKE_OUTER_BICGSTAB) {
        BicgResult br;
        br.rel.assign(nrhs, 0.0);
        if (!run_bicgstab(c, fd, xd, ldd, nrhs, trans, br)) {
            if (c->err.empty()) return cuda_fail(c, "BiCGStab iteration");
            return fail(c, LRSPIKE_ERR_CUDA, c->err);
        }
        it = br.iterations;
        rel = br.rel;
        double worst = 0.0;
        bool nan = false;
        for (int q = 0; q < nrhs; ++q) {
            if (!(rel[q] == rel[q])) nan = true;
            worst = std::max(worst, rel[q]);
        }
        hist.push_back(nan ? NAN : worst);
        converged = !nan && worst <= c->opt.tol;
        stalled = br.breakdown;
    }
    // With fused_retrieve_ok an application's retrieval waits for the next
    // residual (one kernel); the iterate alternates between xd and xalt.
    const bool fuse = outer == LRSPIKE_OUTER_IR && fused_retrieve_ok(c, nrhs, trans);
    double *xcur = xd;
    bool pending = false;
    for (; outer != LRSPIKE_OUTER_BICGSTAB; ++it) {
        if (pending) {
            double *xnext = (xcur == xd) ? c->xalt : xd;
            if (!run_residual_retrieve(c, fd, xcur, xnext)) return fail(c, LRSPIKE_ERR_CUDA, c->err);
            xcur = xnext;
            pending = false;
        } else if (!run_residual(c, fd, xd, ldd, nrhs, trans, it == 0)) {
            return fail(c, LRSPIKE_ERR_CUDA, c->err);
        }
        if (outer == LRSPIKE_OUTER_NONE) {
            if (!apply_precond(c, c->rv, xd, ldd, nrhs, trans, true)) return fail(c, LRSPIKE_ERR_CUDA, c->err);
            it = 1;
            break;
        }
        if (cudaMemcpyAsync(hr, c->nrm + mx, nrhs * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return cuda_fail(c, "outer iteration");
        if (it == 0)
            for (int q = 0; q < nrhs; ++q) hf[q] = hr[q];
        double worst = 0.0;
        bool nan = false;
        for (int q = 0; q < nrhs; ++q) {
            rel[q] = (hf[q] > 0.0) ? hr[q] / hf[q] : 0.0;
            if (!(rel[q] == rel[q])) nan = true;
            worst = std::max(worst, rel[q]);
        }
        hist.push_back(worst);
        if (nan) { stalled = true; break; }
        if (worst <= c->opt.tol) { converged = true; break; }
        if (it >= max_it) break;
        if (it >= 3 && worst > 0.9 * hist[it - 3]) { stalled = true; break; }
        if (fuse) {
            if (!apply_precond_deferred(c, c->rv, nrhs)) return fail(c, LRSPIKE_ERR_CUDA, c->err);
            pending = true;
        } else if (!apply_precond(c, c->rv, xd, ldd, nrhs, trans, true)) {
            return fail(c, LRSPIKE_ERR_CUDA, c->err);
        }
    }
    if (xcur != xd && cudaMemcpyAsync(xd, xcur, (size_t)c->n * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return cuda_fail(c, "iterate copy");
    if (!fdev) {
        if (cudaMemcpy2DAsync(x, ld * 8, xd, ldd * 8, c->n * 8, nrhs, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess)
            return cuda_fail(c, "x device-to-host copy");
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_fail(c, "solve");
    if (outer == LRSPIKE_OUTER_NONE) converged = true;
    if (info) {
        info->iterations = it;
        info->converged = converged ? 1 : 0;
        info->reduced_iterations = c->otf_iters;
        info->max_rel_residual = hist.empty() ? NAN : hist.back();
        if (info->rel_residual)
            for (int q = 0; q < nrhs; ++q) info->rel_residual[q] = hist.empty() ? NAN : rel[q];
    }
    if (!converged) {
        char buf[200];
        std::snprintf(buf, sizeof buf, "%s after %d iterations, worst relative residual %.3e",
                      stalled ? (outer == LRSPIKE_OUTER_BICGSTAB ? "BiCGStab breakdown" : "outer iteration stagnated")
                              : "max_iter reached",
                      it,
                      hist.empty() ? NAN : hist.back());
        return fail(c, LRSPIKE_ERR_NOT_CONVERGED, buf);
    }
    return LRSPIKE_OK;
}

extern "C" lrspike_status lrspike_solve(lrspike_handle h, const double *f, double *x, int32_t nrhs, int64_t ld,
                                        lrspike_info *info) {
    return solve_common(ctx(h), f, x, nrhs, ld, info, false);
}

extern "C" lrspike_status lrspike_solve_transpose(lrspike_handle h, const double *hv, double *lam, int32_t nrhs,
                                                  int64_t ld, lrspike_info *info) {
    return solve_common(ctx(h), hv, lam, nrhs, ld, info, true);
}

extern "C" lrspike_status lrspike_finish(lrspike_handle h, lrspike_info *info) {
    Ctx *c = ctx(h);
    if (!c) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "NULL handle");
    c->err.clear();
    if (!c->opt.graph_safe) return fail(c, LRSPIKE_ERR_STATE, "lrspike_finish is for graph_safe handles");
    cudaSetDevice(c->device);
    int64_t st = kNoStatus;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(&st, c->status, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(c, "finish");
    if (st == kReducedSingular) return fail(c, LRSPIKE_ERR_SINGULAR, "singular reduced system block");
    if (st != kNoStatus) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "zero or non-finite pivot at global row %lld", (long long)st);
        return fail(c, LRSPIKE_ERR_SINGULAR, buf);
    }
    const int nrhs = c->last_nrhs, mx = c->opt.max_nrhs;
    if (nrhs == 0) return fail(c, LRSPIKE_ERR_STATE, "no solve since the last factor");
    std::vector<double> nf(nrhs), nr(nrhs);
    int flag[2] = {0, 0};
    if (cudaMemcpy(nf.data(), c->nrm, nrhs * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nr.data(), c->nrm + mx, nrhs * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(flag, c->stopf, sizeof flag, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(c, "residual read");
    double worst = 0.0;
    bool ok = true;
    for (int q = 0; q < nrhs; ++q) {
        const double rel = (nf[q] > 0.0) ? nr[q] / nf[q] : 0.0;
        if (info && info->rel_residual) info->rel_residual[q] = rel;
        ok = ok && rel <= c->opt.tol;
        worst = std::max(worst, (rel == rel) ? rel : INFINITY);
    }
    // outer IR: the preconditioner applications that ran before the residual
    // met tol (the rest of the enqueued steps returned at entry)
    const int steps = c->opt.outer == LRSPIKE_OUTER_NONE ? 1 : flag[1];
    if (info) {
        info->iterations = steps;
        info->converged = ok ? 1 : 0;
        info->max_rel_residual = worst;
    }
    if (!ok) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "worst relative residual %.3e after %d steps", worst, steps);
        return fail(c, LRSPIKE_ERR_NOT_CONVERGED, buf);
    }
    return LRSPIKE_OK;
}

extern "C" lrspike_status lrspike_destroy(lrspike_handle h) {
    Ctx *c = ctx(h);
    if (!c) return LRSPIKE_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return LRSPIKE_OK;
}

extern "C" const char *lrspike_last_error(lrspike_handle h) {
    Ctx *c = ctx(h);
    return c ? c->err.c_str() : g_err.c_str();
}

extern "C" int64_t lrspike_launch_count(lrspike_handle h) {
    Ctx *c = ctx(h);
    return c ? c->launches : 0;
}

extern "C" lrspike_status lrspike_profile_get(lrspike_handle h, int32_t id, const char **name, int64_t *launches,
                                              double *total_ms) {
    Ctx *c = ctx(h);
    if (!c || id < 0 || id >= KID_COUNT) return fail(c, LRSPIKE_ERR_INVALID_ARG, "bad handle or kernel id");
    drain_profile(c);
    if (name) *name = kKernelNames[id];
    if (launches) *launches = c->kcount[id];
    if (total_ms) *total_ms = c->kms[id];
    return LRSPIKE_OK;
}

extern "C" lrspike_status lrspike_profile_reset(lrspike_handle h) {
    Ctx *c = ctx(h);
    if (!c) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "NULL handle");
    drain_profile(c);
    for (int i = 0; i < KID_COUNT; ++i) {
        c->kcount[i] = 0;
        c->kms[i] = 0.0;
    }
    c->launches = 0;
    return LRSPIKE_OK;
}

extern "C" lrspike_status lrspike_get_reduced(lrspike_handle h, double *sigma, double *R) {
    Ctx *c = ctx(h);
    if (!c) return fail(nullptr, LRSPIKE_ERR_INVALID_ARG, "NULL handle");
    if (!c->factored) return fail(c, LRSPIKE_ERR_STATE, "no successful factor");
    cudaSetDevice(c->device);
    const int r = c->r, n2 = 2 * r, ni = c->p - 1;
    const bool spikes = (c->p > 1 && r > 0);
    if (sigma) {
        const size_t cnt = (size_t)c->p * 2 * c->opt.r;
        if (spikes) {
            if (cudaMemcpy(sigma, c->sigma, cnt * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                return cuda_fail(c, "sigma copy");
        } else {
            std::fill(sigma, sigma + cnt, 0.0);
        }
    }
    if (R && spikes) {
        const size_t nz = (size_t)n2 * ni, nn = (size_t)n2 * n2;
        std::vector<double> E(ni * nn), F(ni * nn), G(ni * nn);
        if (cudaMemcpy(E.data(), c->E, ni * nn * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(F.data(), c->F, ni * nn * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(G.data(), c->Gs, ni * nn * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_fail(c, "reduced copy");
        std::fill(R, R + nz * nz, 0.0);
        const bool full = (c->opt.reduced == LRSPIKE_REDUCED_FULL);
        for (int i = 0; i < ni; ++i)
            for (int a = 0; a < n2; ++a)
                for (int b = 0; b < n2; ++b) {
                    const size_t row = (size_t)i * n2 + a;
                    R[row * nz + (size_t)i * n2 + b] = E[i * nn + a * n2 + b];
                    if (full && i + 1 < ni) R[row * nz + (size_t)(i + 1) * n2 + b] = F[i * nn + a * n2 + b];
                    if (full && i >= 1) R[row * nz + (size_t)(i - 1) * n2 + b] = G[i * nn + a * n2 + b];
                }
    }
    return LRSPIKE_OK;
}
