// C ABI of libfmm (include/fmm.h): argument checks, context state, host/device staging and the
// order of the evaluation steps.  No C++ exception crosses this boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fmm_internal.h"

using namespace fmm;

namespace fmm {

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};
std::atomic<size_t> g_alloc_cap{SIZE_MAX};   // fmm_set_alloc_limit
}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (bytes > g_alloc_cap.load()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    if (bytes > g_alloc_cap.load()) return cudaErrorMemoryAllocation;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&g_pool[dev], &props)) != cudaSuccess) {
                g_pool[dev] = nullptr;
                return e;
            }
            uint64_t keep = UINT64_MAX;
            if ((e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
                return e;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_trim() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool[dev]) cudaMemPoolTrimTo(g_pool[dev], 0);
}
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace fmm

namespace {

fmm_status fail(fmm_ctx *ctx, fmm_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

fmm_status cuda_fail(fmm_ctx *ctx, cudaError_t e, const char *where) {
    cudaGetLastError();   // clear a non-sticky error
    return fail(ctx, e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA,
                std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of pinned (page-locked, mapped) host memory; nullptr for any other pointer
void *mapped_host(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

size_t elem_size(const fmm_ctx *ctx) { return ctx->fp64 ? sizeof(double) : sizeof(float); }

template <typename P>
void free_async(P *&p, cudaStream_t s) {
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

}  // namespace

namespace fmm {

void free_workspace(fmm_ctx *ctx) {
    cudaStream_t s = ctx->stream;
    if (ctx->masks_ev) cudaStreamWaitEvent(s, ctx->masks_ev, 0);   // the side stream's mask kernels
    free_async(ctx->Uc, s), free_async(ctx->Dc, s), free_async(ctx->Ut, s), free_async(ctx->Ct, s);
    free_async(ctx->UtP, s), free_async(ctx->Uscale, s);
    free_async(ctx->UpP, s), free_async(ctx->DnP, s), free_async(ctx->CtP, s);
    free_async(ctx->Ups, s), free_async(ctx->Dns, s), free_async(ctx->Cts, s);
    free_async(ctx->Yc, s), free_async(ctx->Dq, s), free_async(ctx->Cmean, s);
    free_async(ctx->near_phi, s), free_async(ctx->near_grad, s);
    free_async(ctx->far_phi, s), free_async(ctx->far_grad, s), free_async(ctx->pts_qi, s);
    free_async(ctx->stage_in, s), free_async(ctx->stage_out, s), free_async(ctx->stage_grad, s);
    for (int l = 0; l <= kMaxDepth; ++l)
        for (TileSet *ts : {&ctx->tiles_plain[l], &ctx->tiles_cls[l]}) {
            free_async(ts->tiles, s), free_async(ts->masks, s);
            ts->host.clear();
            ts->ntiles = 0;
        }
    ctx->have_ws = false;
    ctx->ws_bytes = 0;
}

// The workspaces outlive the tree: a new tree reuses them when it fits (see ensure_workspace).
void free_tree(fmm_ctx *ctx) {
    cudaStream_t s = ctx->stream;
    free_async(ctx->pts, s), free_async(ctx->perm, s), free_async(ctx->leaf_off, s), free_async(ctx->inv_perm, s);
    free_async(ctx->u_off, s), free_async(ctx->u_idx, s), free_async(ctx->p2p_order, s);
    for (int l = 0; l <= kMaxDepth; ++l) {
        LevelTables &L = ctx->lev[l];
        free_async(L.keys, s), free_async(L.parent, s), free_async(L.child, s);
        free_async(L.dense, s);
        if (!ctx->cls_all) free_async(L.cls_rows, s);
        L = LevelTables{};
    }
    free_async(ctx->cls_all, s);
    ctx->have_tree = false;
    ctx->tiles_ok = false;
    ctx->last_far = false;
    ctx->n = 0;
    ctx->nleaf = 0;
}

void free_ops(fmm_ctx *ctx) {
    cudaStreamSynchronize(ctx->stream);
    for (void *p : ctx->op_allocs) cudaFree(p);
    ctx->op_allocs.clear();
    tc_free(ctx);
    for (int l = 0; l <= kMaxDepth; ++l) {
        ctx->fwd[l] = OpSet{};
        ctx->adj[l] = OpSet{};
        ctx->host_ops[l] = nullptr;
    }
    ctx->grid_dev = nullptr;
    ctx->have_ops = false;
}

// Workspaces sized for the current tree, kept across trees while they fit (rows of levels 0
// and 1 and padding columns are zeroed once when allocated and never written or read by the
// passes); the tiles of the VLI and the level sweeps are rebuilt for every tree.
fmm_status ensure_workspace(fmm_ctx *ctx) {
    const int64_t need_rows = ctx->total_rows, need_nl = ctx->nleaf, need_n = ctx->n;
    if (ctx->have_ws && (need_rows > ctx->ws_rows || need_nl > ctx->ws_nleaf || need_n > ctx->ws_n))
        free_workspace(ctx);
    if (ctx->have_ws) {
        if (!ctx->tiles_ok) {
            cudaError_t e = build_tiles(ctx, ctx->tensor ? 128 : 64);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "tile construction");
            ctx->tiles_ok = true;
        }
        return FMM_OK;
    }
    cudaStream_t s = ctx->stream;
    const size_t es = elem_size(ctx);
    const int nsp = ctx->nsp;
    const OpSet &o = ctx->fwd[ctx->opt.depth];   // every level has the same shapes
    const int kw = std::max(std::max(o.kinp, o.koutp), 16);
    ctx->ws_kw = kw;
    const int64_t rows = need_rows, nl = need_nl, n = need_n;
    const int vc = ctx->cplx ? 2 : 1;   // values per point (complex outputs)
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {&ctx->Uc, (size_t)rows * nsp * es},   {&ctx->Dc, (size_t)rows * nsp * es},
        // tensor-core modes hand the compressed vectors over as split planes (UtP) instead
        {&ctx->Ut, ctx->tensor ? (size_t)16 : (size_t)rows * kw * es},
        {&ctx->Ct, (size_t)rows * kw * es},
        {&ctx->Yc, (size_t)nl * o.rclp * es},
        {&ctx->Dq, (size_t)nl * nsp * es},     {&ctx->Cmean, (size_t)rows * sizeof(double)},
        {&ctx->near_phi, (size_t)n * vc * es},
        {&ctx->near_grad, (size_t)n * 3 * vc * es}, {&ctx->far_phi, (size_t)n * vc * es},
        {&ctx->far_grad, (size_t)n * 3 * vc * es}, {&ctx->pts_qi, ctx->cplx ? (size_t)n * es : (size_t)16},
    };
    if (ctx->tensor) {
        const int np = ctx->opt.precision == FMM_BF16X6 ? 3 : 2;
        const size_t pesz = ctx->opt.precision == FMM_TF32X3 ? 4 : 2;
        ctx->utp_plane = (long long)((size_t)rows * kw * pesz + 256) / 256 * 256;
        if (ctx->opt.precision == FMM_FP16X3) {
            // every contraction reads FP16 planes: the upward- and downward-side rows, the
            // compressed vectors (UtP) and the stencil output, each with its row scales
            ctx->upp_plane = (long long)((size_t)rows * nsp * 2 + 256) / 256 * 256;
            ctx->ctp_plane = ctx->utp_plane;
            const size_t ns_chunks = (size_t)rows * ((nsp + 63) / 64) * sizeof(float) + 16;
            const size_t kw_chunks = (size_t)rows * ((kw + 63) / 64) * sizeof(float) + 16;
            bool okp = pool_alloc((void **)&ctx->Uscale, kw_chunks, s) == cudaSuccess &&
                       pool_alloc((void **)&ctx->Cts, kw_chunks, s) == cudaSuccess &&
                       pool_alloc((void **)&ctx->Ups, ns_chunks, s) == cudaSuccess &&
                       pool_alloc((void **)&ctx->Dns, ns_chunks, s) == cudaSuccess &&
                       pool_alloc(&ctx->UpP, (size_t)ctx->upp_plane * 2, s) == cudaSuccess &&
                       pool_alloc(&ctx->DnP, (size_t)ctx->upp_plane * 2, s) == cudaSuccess &&
                       pool_alloc(&ctx->CtP, (size_t)ctx->ctp_plane * 2, s) == cudaSuccess;
            if (!okp) {
                cudaGetLastError();
                free_workspace(ctx);
                return fail(ctx, FMM_ENOMEM, "workspace allocation failed (FP16 planes)");
            }
        }
        if (pool_alloc(&ctx->UtP, (size_t)ctx->utp_plane * np, s) != cudaSuccess) {
            cudaGetLastError();
            free_workspace(ctx);
            return fail(ctx, FMM_ENOMEM, "workspace allocation failed (split planes)");
        }
    }
    size_t total = 0;
    for (auto &a : allocs) {
        cudaError_t e = pool_alloc(a.p, std::max<size_t>(a.bytes, 16), s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_workspace(ctx);
            return fail(ctx, FMM_ENOMEM, "workspace allocation of " + std::to_string(a.bytes) + " bytes failed");
        }
        total += a.bytes;
    }
    // rows that no step writes (levels 0-1, unused padding) must read as zero
    for (void **p : {&ctx->Uc, &ctx->Dc, &ctx->Ut, &ctx->Ct}) {
        size_t b = (p == &ctx->Uc || p == &ctx->Dc) ? (size_t)rows * nsp * es : (size_t)rows * kw * es;
        if (p == &ctx->Ut && ctx->tensor) b = 16;
        cudaMemsetAsync(*p, 0, b, s);
    }
    cudaError_t e = build_tiles(ctx, ctx->tensor ? 128 : 64);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile construction");
    ctx->tiles_ok = true;
    ctx->ws_bytes = total;
    ctx->ws_rows = rows, ctx->ws_nleaf = nl, ctx->ws_n = n;
    ctx->have_ws = true;
    return FMM_OK;
}

}  // namespace fmm

namespace {

// device view of a caller array: either the pointer itself or a staging buffer
struct Staged {
    void *dev = nullptr;
    bool host = false;
};

fmm_status stage(fmm_ctx *ctx, const void *p, size_t bytes, bool copy_in, void **slot, Staged *out) {
    out->host = !is_device_ptr(p);
    if (!out->host) {
        out->dev = const_cast<void *>(p);
        return FMM_OK;
    }
    if (!*slot) {
        if (pool_alloc(slot, std::max<size_t>(bytes, 16), ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FMM_ENOMEM, "staging allocation failed");
        }
    }
    out->dev = *slot;
    if (copy_in) {
        cudaError_t e = cudaMemcpyAsync(*slot, p, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copy");
    }
    return FMM_OK;
}

template <typename T>
fmm_status run_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad, int parts, bool adjoint) {
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n;
    const int64_t vn = ctx->cplx ? 2 * n : n;   // values of a density or potential array
    Staged sq, sphi, sgrad;
    fmm_status st;
    if ((st = stage(ctx, q, vn * sizeof(T), true, &ctx->stage_in, &sq)) != FMM_OK) return st;
    // outputs in pinned host memory (all of them) are written by the output gather straight over
    // the host link, in the caller's order: no staging buffer and no separate copy
    const bool want_grad = grad && !adjoint;
    void *phi_map = (!ctx->cplx && phi) ? mapped_host(phi) : nullptr;
    void *grad_map = (!ctx->cplx && want_grad) ? mapped_host(grad) : nullptr;
    const bool direct = !ctx->cplx && (phi || want_grad) && (!phi || phi_map) && (!want_grad || grad_map);
    if (!direct) {
        if (phi && (st = stage(ctx, phi, vn * sizeof(T), false, &ctx->stage_out, &sphi)) != FMM_OK) return st;
        if (grad && (st = stage(ctx, grad, 3 * vn * sizeof(T), false, &ctx->stage_grad, &sgrad)) != FMM_OK) return st;
    } else if (!ctx->inv_perm) {
        if (pool_alloc((void **)&ctx->inv_perm, std::max<int64_t>(n, 1) * sizeof(int), s) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FMM_ENOMEM, "inverse permutation");
        }
        cudaError_t ei = launch_invert_perm(ctx->perm, n, ctx->inv_perm, s);
        if (ei != cudaSuccess) return cuda_fail(ctx, ei, "inverse permutation");
    }
    cudaError_t e;
    cudaEventRecord(ctx->ev[0], s);
    e = ctx->cplx ? launch_gather_points_c<T>((const T *)sq.dev, ctx->perm, ctx->pts, (T *)ctx->pts_qi, n, s)
                  : launch_gather_points<T>((const T *)sq.dev, ctx->perm, ctx->pts, n, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather");
    cudaEventRecord(ctx->ev[7], s);
    const bool near = parts & FMM_PART_NEAR;
    const bool far = (parts & FMM_PART_FAR) && ctx->opt.depth >= 2;
    T *ng = (grad && !adjoint) ? (T *)ctx->near_grad : nullptr;
    T *fg = (grad && !adjoint) ? (T *)ctx->far_grad : nullptr;
    // the near field (ULI) and the far field run on two side streams, concurrently
    cudaStream_t ns = ctx->aux[kMaxDepth + 1], fs = ctx->aux[0];
    cudaStreamWaitEvent(ns, ctx->ev[7], 0);
    cudaStreamWaitEvent(fs, ctx->ev[7], 0);
    if (far) {
        e = run_far<T>(ctx, adjoint, phi ? (T *)ctx->far_phi : nullptr, fg, fs);
        if (e == cudaErrorNotSupported)
            return fail(ctx, FMM_EUNSUPPORTED, "tensor-core contractions are not available in this library");
        if (e != cudaSuccess) return cuda_fail(ctx, e, "far field");
    } else {
        cudaEventRecord(ctx->ev[2], fs), cudaEventRecord(ctx->ev[3], fs), cudaEventRecord(ctx->ev[4], fs);
    }
    cudaEventRecord(ctx->ev[5], fs);
    if (near) {
        T *np = phi ? (T *)ctx->near_phi : nullptr;
        e = ctx->adaptive_eval ? adaptive_uli<T>(ctx, np, ng, ns) : launch_p2p<T>(ctx, np, ng, ns);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "near field");
    }
    cudaEventRecord(ctx->ev[1], ns);
    cudaStreamWaitEvent(s, ctx->ev[5], 0);   // join the far field
    cudaStreamWaitEvent(s, ctx->ev[1], 0);   // join the near field
    if (direct) {
        e = launch_gather_out<T>(near && phi ? (const T *)ctx->near_phi : nullptr, near ? ng : nullptr,
                                 far && phi ? (const T *)ctx->far_phi : nullptr, far ? fg : nullptr, ctx->inv_perm,
                                 (T *)phi_map, (T *)grad_map, n, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "output gather");
        cudaEventRecord(ctx->ev[6], s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
        ctx->last_adjoint = adjoint;
        ctx->last_far = far;
        return FMM_OK;
    }
    {
        const T *a = near && phi ? (const T *)ctx->near_phi : nullptr, *b = near ? ng : nullptr;
        const T *c = far && phi ? (const T *)ctx->far_phi : nullptr, *d = far ? fg : nullptr;
        T *go = (grad && !adjoint) ? (T *)sgrad.dev : nullptr;
        e = ctx->cplx ? launch_scatter_c<T>(a, b, c, d, ctx->perm, (T *)sphi.dev, go, n, s)
                      : launch_scatter<T>(a, b, c, d, ctx->perm, (T *)sphi.dev, go, n, s);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scatter");
    cudaEventRecord(ctx->ev[6], s);
    if (phi && sphi.host && (e = cudaMemcpyAsync(phi, sphi.dev, vn * sizeof(T), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "device-to-host copy");
    if (grad && !adjoint && sgrad.host &&
        (e = cudaMemcpyAsync(grad, sgrad.dev, 3 * vn * sizeof(T), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "device-to-host copy");
    if (sq.host || (phi && sphi.host) || (grad && sgrad.host)) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    }
    ctx->last_adjoint = adjoint;
    ctx->last_far = far;
    return FMM_OK;
}

// `out`: the output that must be present (the potentials, or for a gradient-only evaluation the
// gradients)
template <typename T>
fmm_status run_partition(fmm_ctx *ctx, const void *q, void *phi, void *grad) {
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n;
    Staged sq, sphi, sgrad;
    fmm_status st;
    if ((st = stage(ctx, q, n * sizeof(T), true, &ctx->stage_in, &sq)) != FMM_OK) return st;
    if (phi && (st = stage(ctx, phi, n * sizeof(T), false, &ctx->stage_out, &sphi)) != FMM_OK) return st;
    if (grad && (st = stage(ctx, grad, 3 * n * sizeof(T), false, &ctx->stage_grad, &sgrad)) != FMM_OK) return st;
    st = split_run<T>(ctx, (const T *)sq.dev, (T *)sphi.dev, (T *)sgrad.dev);
    if (st != FMM_OK) return st;
    cudaError_t e;
    if (phi && sphi.host && (e = cudaMemcpyAsync(phi, sphi.dev, n * sizeof(T), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "device-to-host copy");
    if (grad && sgrad.host &&
        (e = cudaMemcpyAsync(grad, sgrad.dev, 3 * n * sizeof(T), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "device-to-host copy");
    if (sq.host || (phi && sphi.host) || (grad && sgrad.host)) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    }
    return FMM_OK;
}

fmm_status check_ready(fmm_ctx *ctx, const void *q, const void *out) {
    if (!ctx) return FMM_EINVAL;
    if (!ctx->have_tree) return fail(ctx, FMM_ESTATE, "fmm_build_tree has not been called");
    if (!ctx->have_ops) return fail(ctx, FMM_ESTATE, "fmm_precompute has not been called");
    if (!q || !out) return fail(ctx, FMM_EINVAL, "null density or output pointer");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    return ensure_workspace(ctx);
}

}  // namespace

extern "C" {

fmm_status fmm_default_options(fmm_options *opt) {
    if (!opt) return FMM_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->order_p = 6;
    opt->depth = 4;
    opt->precision = FMM_FP32;
    opt->svd_rtol = 1e-6;
    opt->pinv_rtol = 1e-7;
    opt->with_gradient = 1;
    opt->has_domain = 0;
    opt->side = 1.0;
    opt->mean_free = 0;
    return FMM_OK;
}

fmm_status fmm_create(const fmm_options *opt, void *cuda_stream, fmm_ctx **out) {
    if (!opt || !out) return FMM_EINVAL;
    *out = nullptr;
    if (opt->order_p < 2 || opt->order_p > 10) return FMM_EINVAL;
    if (opt->depth < 0 || opt->depth > kMaxDepth) return FMM_EINVAL;
    if (opt->precision < FMM_FP32 || opt->precision > FMM_FP16X3) return FMM_EINVAL;
    if (!(opt->svd_rtol > 0 && opt->svd_rtol < 1) || !(opt->pinv_rtol > 0 && opt->pinv_rtol < 1))
        return FMM_EINVAL;
    // the FP16 planes of FMM_FP16X3 carry the downward rows as produced, before a mean is taken off
    if (opt->mean_free && opt->precision == FMM_FP16X3) return FMM_EUNSUPPORTED;
    if (opt->kernel != FMM_LAPLACE && opt->kernel != FMM_YUKAWA && opt->kernel != FMM_HELMHOLTZ) return FMM_EINVAL;
    if (opt->kernel != FMM_LAPLACE) {
        if (!(std::isfinite(opt->kappa) && opt->kappa > 0)) return FMM_EINVAL;
        // the operators depend on the physical box sizes (no homogeneity), and the means that
        // mean_free carries down the tree are exact for Laplace only
        if (!opt->has_domain || opt->mean_free) return FMM_EUNSUPPORTED;
    }
    if (opt->m2l != FMM_M2L_DENSE && opt->m2l != FMM_M2L_FFT) return FMM_EINVAL;
    if (opt->m2l == FMM_M2L_FFT) {
        if (opt->order_p < 4) return FMM_EINVAL;   // the lattice surfaces of boxes 2 apart would touch
        if ((opt->precision != FMM_FP32 && opt->precision != FMM_FP64) || opt->kernel != FMM_LAPLACE ||
            opt->mean_free)
            return FMM_EUNSUPPORTED;
    }
    if (opt->has_domain) {
        if (!(std::isfinite(opt->side) && opt->side > 0)) return FMM_EINVAL;
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(opt->origin[a])) return FMM_EINVAL;
    }
    fmm_ctx *ctx = new (std::nothrow) fmm_ctx();
    if (!ctx) return FMM_ENOMEM;
    ctx->opt = *opt;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->fp64 = opt->precision == FMM_FP64;
    ctx->tensor = opt->precision == FMM_TF32X3 || opt->precision == FMM_BF16X3 || opt->precision == FMM_BF16X6 ||
                  opt->precision == FMM_FP16X3;
    ctx->npts = 6 * (opt->order_p - 1) * (opt->order_p - 1) + 2;
    ctx->cplx = opt->kernel == FMM_HELMHOLTZ;
    ctx->fft = opt->m2l == FMM_M2L_FFT;
    ctx->ns = ctx->cplx ? 2 * ctx->npts : ctx->npts;   // real and imaginary parts of complex values
    ctx->nsp = round_up(ctx->ns, 16);
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return FMM_ECUDA;
    }
    bool okc = true;
    for (auto &e : ctx->ev) okc = okc && cudaEventCreate(&e) == cudaSuccess;
    for (cudaEvent_t *e : {&ctx->masks_fork_ev, &ctx->masks_ev})
        okc = okc && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    // Far-field streams (aux[0] for the level sweeps, aux[2..] for the VLI of each level) at
    // the highest priority, the near field (aux[kMaxDepth + 1]) at the lowest: the far field's
    // dependent chain of small launches then takes SMs first and the near-field kernel fills
    // whatever it leaves idle.
    int prio_lo = 0, prio_hi = 0;
    okc = okc && cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) == cudaSuccess;
    for (int k = 0; k < kMaxDepth + 2; ++k) {
        const int prio = k == kMaxDepth + 1 ? prio_lo : prio_hi;
        okc = okc && cudaStreamCreateWithPriority(&ctx->aux[k], cudaStreamNonBlocking, prio) == cudaSuccess;
        okc = okc && cudaEventCreateWithFlags(&ctx->fork_ev[k], cudaEventDisableTiming) == cudaSuccess;
        okc = okc && cudaEventCreateWithFlags(&ctx->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!okc) {
        cudaGetLastError();
        fmm_destroy(ctx);
        return FMM_ECUDA;
    }
    *out = ctx;
    return FMM_OK;
}

fmm_status fmm_build_tree(fmm_ctx *ctx, const void *xyz, int64_t n) {
    if (!ctx) return FMM_EINVAL;
    if (!xyz) return fail(ctx, FMM_EINVAL, "null coordinate pointer");
    if (n <= 0 || n > 2147483647LL) return fail(ctx, FMM_EINVAL, "n must be in [1, 2^31 - 1]");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    split_free(ctx);   // a partition belongs to the tree it was built on
    adaptive_free(ctx);
    free_tree(ctx);
    ctx->n = n;
    const size_t bytes = (size_t)n * 3 * elem_size(ctx);
    void *dev = const_cast<void *>(xyz);
    void *tmp = nullptr;
    if (!is_device_ptr(xyz)) {
        if (pool_alloc(&tmp, bytes, ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FMM_ENOMEM, "staging allocation failed");
        }
        cudaError_t e = cudaMemcpyAsync(tmp, xyz, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copy");
        dev = tmp;
    }
    cudaError_t e = build_tree(ctx, dev);
    if (tmp) cudaFreeAsync(tmp, ctx->stream);
    if (e == cudaErrorInvalidValue) {
        free_tree(ctx);
        return fail(ctx, FMM_EINVAL, "non-finite coordinate");
    }
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        free_tree(ctx);
        return fail(ctx, FMM_ENOMEM, "tree allocation failed");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tree build");
    ctx->have_tree = true;
    return FMM_OK;
}

fmm_status fmm_precompute(fmm_ctx *ctx) {
    if (!ctx) return FMM_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    if (ctx->have_ops) return FMM_OK;
    std::string err;
    // Laplace: one set for every level.  Modified Helmholtz: one per level that a step uses
    // (2..d, or d alone for d < 2: U2U, VLI and D2D run on levels >= 2, the closing on d), with
    // kappa in units of that level's half-width side / 2^(l+1); the other levels alias the
    // coarsest built one and are never read.
    const int d = ctx->opt.depth;
    const bool lap = ctx->opt.kernel == FMM_LAPLACE;
    const int lo = !lap ? (d < 2 ? d : 2) : 0;
    std::vector<double> ku;
    for (int l = lo; l <= d; ++l) ku.push_back(!lap ? ctx->opt.kappa * std::ldexp(ctx->opt.side, -(l + 1)) : 0.0);
    if (lap) ku.resize(1);
    std::vector<const HostOps *> hs;
    try {
        hs = host_operator_levels(ctx->opt.order_p, ctx->opt.pinv_rtol, ctx->opt.svd_rtol, ctx->opt.kernel, ku, &err,
                                  ctx->fft);
    } catch (const std::bad_alloc &) {
        return fail(ctx, FMM_ENOMEM, "host memory exhausted in precompute");
    } catch (...) {
        return fail(ctx, FMM_EINVAL, "precompute failed");
    }
    if (hs.size() != ku.size()) return fail(ctx, FMM_EINVAL, "precompute failed: " + err);
    for (int l = 0; l <= kMaxDepth; ++l)
        ctx->host_ops[l] = lap ? hs[0] : hs[std::min(std::max(l, lo), d) - lo];
    cudaError_t e;
    if (!ctx->dev_flag) {
        if (dev_malloc((void **)&ctx->dev_flag, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FMM_ENOMEM, "flag allocation failed");
        }
        if ((e = cudaMemset(ctx->dev_flag, 0, sizeof(int))) != cudaSuccess) return cuda_fail(ctx, e, "memset");
    }
    try {
        e = upload_operators(ctx);
    } catch (const std::bad_alloc &) {
        free_ops(ctx);
        return fail(ctx, FMM_ENOMEM, "host memory exhausted in operator upload");
    }
    if (e == cudaErrorNotSupported) {
        free_ops(ctx);
        return fail(ctx, FMM_EUNSUPPORTED, "tensor-core contractions are not available in this library");
    }
    if (e != cudaSuccess) {
        free_ops(ctx);
        return cuda_fail(ctx, e, "operator upload");
    }
    free_workspace(ctx);   // operator ranks size the workspaces
    ctx->have_ops = true;
    return FMM_OK;
}

fmm_status fmm_evaluate_parts(fmm_ctx *ctx, const void *q, void *phi, void *grad, int parts) {
    // phi == NULL with grad: the gradient-only ("force") evaluation
    fmm_status st = check_ready(ctx, q, phi ? phi : grad);
    if (st != FMM_OK) return st;
    if (grad && !ctx->opt.with_gradient) return fail(ctx, FMM_EINVAL, "gradients were not enabled (with_gradient = 0)");
    if (parts < 1 || parts > FMM_PART_ALL) return fail(ctx, FMM_EINVAL, "parts must be a nonempty subset of near|far");
    return ctx->fp64 ? run_evaluate<double>(ctx, q, phi, grad, parts, false)
                     : run_evaluate<float>(ctx, q, phi, grad, parts, false);
}

fmm_status fmm_adaptive_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad, int parts) {
    fmm_status st = check_ready(ctx, q, phi ? phi : grad);
    if (st != FMM_OK) return st;
    if (!ctx->adaptive) return fail(ctx, FMM_ESTATE, "fmm_adaptive_setup has not been called");
    if (ctx->tensor) return fail(ctx, FMM_EUNSUPPORTED, "the adaptive evaluation runs in FMM_FP32 or FMM_FP64");
    if (ctx->opt.kernel != FMM_LAPLACE) return fail(ctx, FMM_EUNSUPPORTED, "the adaptive evaluation is for the Laplace kernel");
    if (ctx->opt.mean_free) return fail(ctx, FMM_EUNSUPPORTED, "the adaptive evaluation does not take mean_free");
    if (grad && !ctx->opt.with_gradient) return fail(ctx, FMM_EINVAL, "gradients were not enabled (with_gradient = 0)");
    if (parts < 1 || parts > FMM_PART_ALL) return fail(ctx, FMM_EINVAL, "parts must be a nonempty subset of near|far");
    if ((st = adaptive_prepare(ctx)) != FMM_OK) return st;
    ctx->adaptive_eval = true;
    st = ctx->fp64 ? run_evaluate<double>(ctx, q, phi, grad, parts, false)
                   : run_evaluate<float>(ctx, q, phi, grad, parts, false);
    ctx->adaptive_eval = false;
    ctx->last_far = false;   // the check rows of an adaptive evaluation are not exported
    return st;
}

fmm_status fmm_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad) {
    return fmm_evaluate_parts(ctx, q, phi, grad, FMM_PART_ALL);
}

fmm_status fmm_adjoint(fmm_ctx *ctx, const void *g, void *psi, void *grad_psi) {
    fmm_status st = check_ready(ctx, g, psi);
    if (st != FMM_OK) return st;
    if (ctx->cplx) return fail(ctx, FMM_EUNSUPPORTED, "no adjoint for the Helmholtz kernel");
    if (ctx->fft) return fail(ctx, FMM_EUNSUPPORTED, "no adjoint with the FFT form of the M2L");
    if (grad_psi && !ctx->opt.with_gradient) return fail(ctx, FMM_EINVAL, "gradients were not enabled (with_gradient = 0)");
    st = ctx->fp64 ? run_evaluate<double>(ctx, g, psi, nullptr, FMM_PART_ALL, true)
                   : run_evaluate<float>(ctx, g, psi, nullptr, FMM_PART_ALL, true);
    if (st != FMM_OK || !grad_psi) return st;
    // grad phi_g: a forward pass with densities g, potentials into scratch
    void *scratch = ctx->far_phi;   // sorted-order buffer reused as the discarded potential
    const size_t es = elem_size(ctx);
    void *tmp = nullptr;
    if (pool_alloc(&tmp, (size_t)ctx->n * es, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FMM_ENOMEM, "scratch allocation failed");
    }
    (void)scratch;
    st = ctx->fp64 ? run_evaluate<double>(ctx, g, tmp, grad_psi, FMM_PART_ALL, false)
                   : run_evaluate<float>(ctx, g, tmp, grad_psi, FMM_PART_ALL, false);
    cudaFreeAsync(tmp, ctx->stream);
    if (st == FMM_OK) ctx->last_adjoint = true;
    return st;
}

fmm_status fmm_partition_setup(fmm_ctx *ctx, int d_global, int n_ranks) {
    if (!ctx) return FMM_EINVAL;
    if (ctx->cplx) return fail(ctx, FMM_EUNSUPPORTED, "no partitioned evaluation for the Helmholtz kernel");
    if (ctx->fft) return fail(ctx, FMM_EUNSUPPORTED, "no partitioned evaluation with the FFT form of the M2L");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    try {
        return split_setup(ctx, d_global, n_ranks);
    } catch (const std::bad_alloc &) {
        split_free(ctx);
        return fail(ctx, FMM_ENOMEM, "host memory exhausted in the partition setup");
    }
}

fmm_status fmm_partition_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad) {
    if (!ctx) return FMM_EINVAL;
    if (!ctx->split) return fail(ctx, FMM_ESTATE, "fmm_partition_setup has not been called");
    if (!q || (!phi && !grad)) return fail(ctx, FMM_EINVAL, "null density or output pointer");
    if (grad && !ctx->opt.with_gradient) return fail(ctx, FMM_EINVAL, "gradients were not enabled (with_gradient = 0)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    return ctx->fp64 ? run_partition<double>(ctx, q, phi, grad) : run_partition<float>(ctx, q, phi, grad);
}

fmm_status fmm_partition_info(fmm_ctx *ctx, int rank, fmm_rank_info *info) {
    if (!ctx || !info) return FMM_EINVAL;
    return split_info(ctx, rank, info);
}

fmm_status fmm_partition_export(fmm_ctx *ctx, int rank, int level, int kind, uint64_t *out, int64_t *count) {
    if (!ctx) return FMM_EINVAL;
    return split_export(ctx, rank, level, kind, out, count);
}

fmm_status fmm_partition_timings(fmm_ctx *ctx, double *ms, int n) {
    if (!ctx || !ms || n < 0) return FMM_EINVAL;
    return split_timings(ctx, ms, n);
}

fmm_status fmm_adaptive_setup(fmm_ctx *ctx, int capacity) {
    if (!ctx) return FMM_EINVAL;
    if (ctx->fft) return fail(ctx, FMM_EUNSUPPORTED, "no adaptive evaluation with the FFT form of the M2L");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    try {
        return adaptive_setup(ctx, capacity);
    } catch (const std::bad_alloc &) {
        adaptive_free(ctx);
        return fail(ctx, FMM_ENOMEM, "host memory exhausted in the adaptive setup");
    }
}

fmm_status fmm_adaptive_info(fmm_ctx *ctx, fmm_adaptive_tree_info *info) {
    if (!ctx || !info) return FMM_EINVAL;
    std::memset(info, 0, sizeof(*info));
    fmm_status st = adaptive_info(ctx, &info->capacity, info->n_leaves, info->n_refined, info->n_entries);
    if (st == FMM_OK) info->n_rows = ctx->total_rows;
    return st;
}

fmm_status fmm_adaptive_export(fmm_ctx *ctx, int kind, int64_t *offsets, int64_t *idx, int64_t *count) {
    if (!ctx) return FMM_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    try {
        return adaptive_export(ctx, kind, offsets, idx, count);
    } catch (const std::bad_alloc &) {
        return fail(ctx, FMM_ENOMEM, "host memory exhausted in the adaptive export");
    }
}

fmm_status fmm_get_tree_info(const fmm_ctx *ctx, fmm_tree_info *info) {
    if (!ctx || !info) return FMM_EINVAL;
    if (!ctx->have_tree) return FMM_ESTATE;
    std::memset(info, 0, sizeof(*info));
    info->n_points = ctx->n;
    info->depth = ctx->opt.depth;
    info->n_surface = ctx->npts;
    info->m2l_rank_in = ctx->have_ops ? ctx->fwd[ctx->opt.depth].kin : 0;
    info->m2l_rank_out = ctx->have_ops ? ctx->fwd[ctx->opt.depth].kout : 0;
    for (int l = 0; l <= ctx->opt.depth; ++l) info->n_boxes[l] = ctx->lev[l].n;
    info->n_u_entries = ctx->n_u;
    info->p2p_pairs = ctx->p2p_pairs;
    if (ctx->p2p_pairs < 0 && ctx->dev_pairs) {   // computed on the device by the last build
        unsigned long long h = 0;
        if (cudaMemcpyAsync(&h, ctx->dev_pairs, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return FMM_ECUDA;
        }
        info->p2p_pairs = (int64_t)h;
    }
    for (int a = 0; a < 3; ++a) info->origin[a] = ctx->origin[a];
    info->side = ctx->side;
    return FMM_OK;
}

fmm_status fmm_export_tree(fmm_ctx *ctx, int64_t *perm, uint64_t *leaf_keys, int64_t *leaf_offsets,
                           int64_t *u_offsets, int64_t *u_idx) {
    if (!ctx) return FMM_EINVAL;
    if (!ctx->have_tree) return fail(ctx, FMM_ESTATE, "fmm_build_tree has not been called");
    cudaStream_t s = ctx->stream;
    const int d = ctx->opt.depth;
    auto copy_i32 = [&](const int *src, int64_t count, int64_t *dst) -> cudaError_t {
        std::vector<int> h(count);
        cudaError_t e = cudaMemcpyAsync(h.data(), src, count * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int64_t i = 0; i < count; ++i) dst[i] = h[i];
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (perm && e == cudaSuccess) e = copy_i32(ctx->perm, ctx->n, perm);
    if (leaf_offsets && e == cudaSuccess) e = copy_i32(ctx->leaf_off, ctx->nleaf + 1, leaf_offsets);
    if (u_offsets && e == cudaSuccess) e = copy_i32(ctx->u_off, ctx->nleaf + 1, u_offsets);
    if (u_idx && e == cudaSuccess) e = copy_i32(ctx->u_idx, ctx->n_u, u_idx);
    if (leaf_keys && e == cudaSuccess) {
        std::vector<uint32_t> h(ctx->nleaf);
        e = cudaMemcpyAsync(h.data(), ctx->lev[d].keys, ctx->nleaf * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int i = 0; i < ctx->nleaf; ++i) leaf_keys[i] = h[i];
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "export");
    return FMM_OK;
}

fmm_status fmm_export_level(fmm_ctx *ctx, int level, uint64_t *keys, int64_t *v_offsets, int64_t *v_idx,
                            int32_t *v_tvec, int64_t *n_v_entries) {
    if (!ctx) return FMM_EINVAL;
    if (!ctx->have_tree) return fail(ctx, FMM_ESTATE, "fmm_build_tree has not been called");
    if (level < 0 || level > ctx->opt.depth) return fail(ctx, FMM_EINVAL, "level out of range");
    cudaStream_t s = ctx->stream;
    const LevelTables &L = ctx->lev[level];
    cudaError_t e = cudaSuccess;
    if (keys) {
        std::vector<uint32_t> h(L.n);
        e = cudaMemcpyAsync(h.data(), L.keys, L.n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int64_t i = 0; i < L.n; ++i) keys[i] = h[i];
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "export");
    if (level < 2) {
        if (v_offsets)
            for (int64_t i = 0; i <= L.n; ++i) v_offsets[i] = 0;
        if (n_v_entries) *n_v_entries = 0;
        return FMM_OK;
    }
    if (v_offsets || v_idx || v_tvec || n_v_entries) {
        try {
            e = export_v_lists(ctx, level, v_offsets, v_idx, v_tvec, n_v_entries);
        } catch (const std::bad_alloc &) {
            return fail(ctx, FMM_ENOMEM, "host memory exhausted in export");
        }
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(ctx, FMM_ENOMEM, "device memory exhausted in export");
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "V-list export");
    }
    return FMM_OK;
}

fmm_status fmm_export_check(fmm_ctx *ctx, int level, int kind, void *host_out) {
    if (!ctx || !host_out) return FMM_EINVAL;
    if (!ctx->have_ws || ctx->last_adjoint || !ctx->last_far)
        return fail(ctx, FMM_ESTATE, "no forward far-field evaluation to export");
    if (level < 2 || level > ctx->opt.depth) return fail(ctx, FMM_EINVAL, "level must be in [2, depth]");
    if (kind != 0 && kind != 1) return fail(ctx, FMM_EINVAL, "kind must be 0 (upward) or 1 (downward)");
    const size_t es = elem_size(ctx);
    const LevelTables &L = ctx->lev[level];
    const void *src = kind == 0 ? ctx->Uc : ctx->Dc;
    std::vector<unsigned char> h((size_t)L.n * ctx->nsp * es);
    cudaError_t e = cudaMemcpyAsync(h.data(), (const unsigned char *)src + (size_t)L.row_base * ctx->nsp * es,
                                    h.size(), cudaMemcpyDeviceToHost, ctx->stream);
    // downward rows are stored without their per-box mean (carried separately): add it back
    const bool add_mean = kind == 1 && ctx->opt.mean_free;
    std::vector<double> cm(add_mean ? L.n : 0);
    if (e == cudaSuccess && add_mean)
        e = cudaMemcpyAsync(cm.data(), (const double *)ctx->Cmean + L.row_base, L.n * sizeof(double),
                            cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "export");
    for (int64_t b = 0; b < L.n; ++b) {
        unsigned char *dst = (unsigned char *)host_out + (size_t)b * ctx->ns * es;
        std::memcpy(dst, h.data() + (size_t)b * ctx->nsp * es, ctx->ns * es);
        if (add_mean)
            for (int j = 0; j < ctx->ns; ++j) {
                if (ctx->fp64) ((double *)dst)[j] += cm[b];
                else ((float *)dst)[j] = (float)((double)((float *)dst)[j] + cm[b]);
            }
    }
    return FMM_OK;
}

fmm_status fmm_last_timings(fmm_ctx *ctx, double *ms, int n) {
    if (!ctx || !ms || n < 0) return FMM_EINVAL;
    if (cudaEventSynchronize(ctx->ev[6]) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "timings");
    float t[5] = {};
    cudaEventElapsedTime(&t[0], ctx->ev[7], ctx->ev[1]);
    cudaEventElapsedTime(&t[1], ctx->ev[7], ctx->ev[3]);
    cudaEventElapsedTime(&t[2], ctx->ev[3], ctx->ev[4]);
    cudaEventElapsedTime(&t[3], ctx->ev[4], ctx->ev[5]);
    cudaEventElapsedTime(&t[4], ctx->ev[0], ctx->ev[6]);
    cudaGetLastError();
    for (int i = 0; i < n && i < 5; ++i) ms[i] = t[i];
    return FMM_OK;
}

long long fmm_kernel_launches(void) { return launches(); }

fmm_status fmm_set_wait_limit(fmm_ctx *ctx, double seconds) {
    if (!ctx) return FMM_EINVAL;
    if (!(seconds >= 0) || !(seconds <= 60)) return fail(ctx, FMM_EINVAL, "wait limit must be in [0, 60] s");
    ctx->tc_wait_ns = (unsigned long long)(seconds * 1e9);
    return FMM_OK;
}

void fmm_set_alloc_limit(size_t bytes) { g_alloc_cap.store(bytes); }

fmm_status fmm_debug_check(fmm_ctx *ctx, uint32_t *flags, int32_t *in_kernel) {
    if (!ctx || !flags) return ctx ? fail(ctx, FMM_EINVAL, "null flags pointer") : FMM_EINVAL;
    if (!ctx->have_tree) return fail(ctx, FMM_ESTATE, "fmm_build_tree has not been called");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    uint32_t f = 0;
    if (e == cudaSuccess) e = validate_tree(ctx, &f);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tree validation");
    f |= debug_word_tree(true) | debug_word_p2p(true) | debug_word_output(true);
    *flags = f;
#ifdef FMM_DEBUG
    if (in_kernel) *in_kernel = 1;
#else
    if (in_kernel) *in_kernel = 0;
#endif
    return FMM_OK;
}

const char *fmm_last_error(const fmm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void fmm_destroy(fmm_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    split_free(ctx);
    adaptive_free(ctx);
    free_tree(ctx);
    free_workspace(ctx);
    free_ops(ctx);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->class_slots) cudaFree(ctx->class_slots);
    if (ctx->class_delta) cudaFree(ctx->class_delta);
    if (ctx->dev_counts) cudaFree(ctx->dev_counts);
    if (ctx->dev_pairs) cudaFree(ctx->dev_pairs);
    if (ctx->host_counts) cudaFreeHost(ctx->host_counts);
    if (ctx->host_tiles) cudaFreeHost(ctx->host_tiles);
    if (ctx->tiles_ev) cudaEventDestroy(ctx->tiles_ev);
    if (ctx->masks_fork_ev) cudaEventDestroy(ctx->masks_fork_ev);
    if (ctx->masks_ev) cudaEventDestroy(ctx->masks_ev);
    pool_trim();
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < kMaxDepth + 2; ++k) {
        if (ctx->aux[k]) cudaStreamSynchronize(ctx->aux[k]), cudaStreamDestroy(ctx->aux[k]);
        if (ctx->fork_ev[k]) cudaEventDestroy(ctx->fork_ev[k]);
        if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
    }
    if (ctx->dev_flag) cudaFree(ctx->dev_flag);
    cudaGetLastError();
    delete ctx;
}

fmm_status fmm_sync(fmm_ctx *ctx) {
    if (!ctx) return FMM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    if (!ctx->dev_flag) return FMM_OK;
    int flag = 0;
    if ((e = cudaMemcpy(&flag, ctx->dev_flag, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, e, "flag read");
    if (flag) {
        cudaMemset(ctx->dev_flag, 0, sizeof(int));
        return fail(ctx, (fmm_status)flag, "a kernel gave up waiting on the device (bounded wait expired); "
                                           "results of the calls since the last fmm_sync are invalid");
    }
    return FMM_OK;
}

}  // extern "C"
