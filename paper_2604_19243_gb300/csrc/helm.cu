// Point kernels of the Helmholtz kernel exp(i k r) / (4 pi r) with complex densities (Eq. 1 with
// F = C): the ULI near field, the S2U check values of the leaves and the D2T evaluation.  The
// surface contractions between them are the real kernels' (the operators act on the real form
// [Re v; Im v] of a box vector), so only these kernels see complex arithmetic.
//
// Per (target x, source y) pair, r = |x - y| and d = x - y:
//   w = s exp(i k r) / r,  phi += w / (4 pi),  grad phi += w (i k r - 1) d / (4 pi r^2).
// Pairs at distance zero are skipped.  The densities' imaginary parts live beside the points
// (pts holds (x, y, z, Re s)); potentials and gradients are interleaved (re, im).  In shallow
// trees k r exceeds pi, so the FP32 sine and cosine reduce the argument first.
#include <algorithm>
#include <type_traits>

#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

template <typename T> __host__ __device__ constexpr T k_inv4pi() { return (T)0.079577471545947667884441881686257181; }

__device__ __forceinline__ float rsqrt_c(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_c(double x) { return rsqrt(x); }
// FP32: Cody-Waite reduction of x by multiples of 2 pi (2 pi split into its FP32 rounding and the
// remainder), then the hardware sin/cos approximation, whose absolute error is about 2^-21 on
// [-pi, pi]; the reduction keeps that error for |k r| up to about 10^5.
__device__ __forceinline__ void sincos_c(float x, float *s, float *c) {
    const float t = rintf(x * 0.15915494309189535f);     // x / (2 pi), rounded
    float r = fmaf(-t, 6.2831854820251465f, x);          // 2 pi rounded to FP32
    r = fmaf(-t, -1.7484555314695172e-07f, r);           // 2 pi minus its FP32 rounding
    __sincosf(r, s, c);
}
__device__ __forceinline__ void sincos_c(double x, double *s, double *c) { sincos(x, s, c); }

// one pair: accumulate the potential (pr, pi) and, with GRAD, the gradient g[6]
template <typename T, bool GRAD>
__device__ __forceinline__ void helm_pair(T dx, T dy, T dz, T qr, T qi, T k, T &pr, T &pim, T *g) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T ri = r2 > (T)0 ? rsqrt_c(r2) : (T)0;
    const T r = r2 * ri;
    T s, c;
    sincos_c(k * r, &s, &c);
    const T wr = (qr * c - qi * s) * ri, wi = (qr * s + qi * c) * ri;
    pr += wr;
    pim += wi;
    if (GRAD) {
        const T ri2 = ri * ri;
        const T zr = (-wr - k * r * wi) * ri2, zi = (-wi + k * r * wr) * ri2;
        g[0] += zr * dx, g[1] += zi * dx;
        g[2] += zr * dy, g[3] += zi * dy;
        g[4] += zr * dz, g[5] += zi * dz;
    }
}

constexpr int kThreads = 128;
constexpr int kChunk = 1024;

// ULI: one CTA per target leaf; every thread holds one target at a time, the sources of the
// leaf's U list (itself included) pass through shared memory in chunks.
template <typename T, bool POT, bool GRAD>
__global__ void __launch_bounds__(kThreads)
helm_p2p_kernel(const typename V4<T>::type *__restrict__ pts, const T *__restrict__ qi, const int *__restrict__ leaf_off,
                const int *__restrict__ u_off, const int *__restrict__ u_idx, const int *__restrict__ order, T k,
                T *__restrict__ phi, T *__restrict__ grad) {
    using P = typename V4<T>::type;
    __shared__ P sp[kChunk];
    __shared__ T sq[kChunk];
    const int b = order[blockIdx.x];
    const int t0 = leaf_off[b], t1 = leaf_off[b + 1];
    for (int tb = t0; tb < t1; tb += kThreads) {
        const int i = tb + threadIdx.x;
        const P x = pts[min(i, t1 - 1)];
        T pr = 0, pim = 0, g[6] = {0, 0, 0, 0, 0, 0};
        for (int e = u_off[b]; e < u_off[b + 1]; ++e) {
            const int a = u_idx[e];
            const int s0 = leaf_off[a], s1 = leaf_off[a + 1];
            for (int c0 = s0; c0 < s1; c0 += kChunk) {
                const int n = min(kChunk, s1 - c0);
                __syncthreads();
                for (int j = threadIdx.x; j < n; j += kThreads) sp[j] = pts[c0 + j], sq[j] = qi[c0 + j];
                __syncthreads();
                for (int j = 0; j < n; ++j) {
                    const P y = sp[j];
                    helm_pair<T, GRAD>(x.x - y.x, x.y - y.y, x.z - y.z, y.w, sq[j], k, pr, pim, g);
                }
            }
        }
        if (i < t1) {
            if (POT) phi[2 * (int64_t)i] = pr * k_inv4pi<T>(), phi[2 * (int64_t)i + 1] = pim * k_inv4pi<T>();
            if (GRAD)
                for (int a = 0; a < 6; ++a) grad[6 * (int64_t)i + a] = g[a] * k_inv4pi<T>();
        }
    }
}

// S2U: the complex check values on the 2.95 surface of every leaf, row = [Re (npts) | Im (npts) | 0]
template <typename T>
__global__ void __launch_bounds__(kThreads)
helm_check_kernel(const typename V4<T>::type *__restrict__ pts, const T *__restrict__ qi, const int *__restrict__ leaf_off,
                  const uint32_t *__restrict__ keys, const T *__restrict__ grid, int npts, int nsp, double ox, double oy,
                  double oz, double width, double radius, T k, T *__restrict__ out) {
    using P = typename V4<T>::type;
    __shared__ P sp[kChunk];
    __shared__ T sq[kChunk];
    __shared__ double cen[3];
    const int b = blockIdx.x;
    const int s0 = leaf_off[b], s1 = leaf_off[b + 1];
    if (threadIdx.x == 0) {
        int ax, ay, az;
        demorton3(keys[b], ax, ay, az);
        cen[0] = ox + (ax + 0.5) * width, cen[1] = oy + (ay + 0.5) * width, cen[2] = oz + (az + 0.5) * width;
    }
    __syncthreads();
    T *row = out + (int64_t)b * nsp;
    for (int j = 2 * npts + threadIdx.x; j < nsp; j += kThreads) row[j] = (T)0;
    for (int j0 = 0; j0 < npts; j0 += kThreads) {
        const int j = j0 + threadIdx.x;
        T px = 0, py = 0, pz = 0;
        if (j < npts) {
            px = (T)(cen[0] + radius * (double)grid[3 * j]);
            py = (T)(cen[1] + radius * (double)grid[3 * j + 1]);
            pz = (T)(cen[2] + radius * (double)grid[3 * j + 2]);
        }
        T pr = 0, pim = 0;
        for (int c0 = s0; c0 < s1; c0 += kChunk) {
            const int n = min(kChunk, s1 - c0);
            __syncthreads();
            for (int e = threadIdx.x; e < n; e += kThreads) sp[e] = pts[c0 + e], sq[e] = qi[c0 + e];
            __syncthreads();
            if (j < npts)
                for (int e = 0; e < n; ++e) {
                    const P y = sp[e];
                    helm_pair<T, false>(px - y.x, py - y.y, pz - y.z, y.w, sq[e], k, pr, pim, nullptr);
                }
        }
        if (j < npts) row[j] = pr * k_inv4pi<T>(), row[npts + j] = pim * k_inv4pi<T>();
    }
}

// D2T: potentials and gradients at the points of every leaf from the complex densities
// [Re (npts) | Im (npts)] on its 2.95 surface
template <typename T, bool POT, bool GRAD>
__global__ void __launch_bounds__(kThreads)
helm_eval_kernel(const typename V4<T>::type *__restrict__ pts, const int *__restrict__ leaf_off,
                 const uint32_t *__restrict__ keys, const T *__restrict__ grid, int npts, const T *__restrict__ dens,
                 int ldd, double ox, double oy, double oz, double width, double radius, T k, T *__restrict__ phi,
                 T *__restrict__ grad) {
    using P = typename V4<T>::type;
    extern __shared__ unsigned char smem_raw[];
    P *sp = reinterpret_cast<P *>(smem_raw);                    // [npts] (x, y, z, Re density)
    T *sq = reinterpret_cast<T *>(sp + npts);                   // [npts] Im density
    __shared__ double cen[3];
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        int ax, ay, az;
        demorton3(keys[b], ax, ay, az);
        cen[0] = ox + (ax + 0.5) * width, cen[1] = oy + (ay + 0.5) * width, cen[2] = oz + (az + 0.5) * width;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < npts; j += kThreads) {
        P p;
        p.x = (T)(cen[0] + radius * (double)grid[3 * j]);
        p.y = (T)(cen[1] + radius * (double)grid[3 * j + 1]);
        p.z = (T)(cen[2] + radius * (double)grid[3 * j + 2]);
        p.w = dens[(int64_t)b * ldd + j];
        sp[j] = p;
        sq[j] = dens[(int64_t)b * ldd + npts + j];
    }
    __syncthreads();
    for (int i = leaf_off[b] + threadIdx.x; i < leaf_off[b + 1]; i += kThreads) {
        const P x = pts[i];
        T pr = 0, pim = 0, g[6] = {0, 0, 0, 0, 0, 0};
        for (int e = 0; e < npts; ++e) {
            const P y = sp[e];
            helm_pair<T, GRAD>(x.x - y.x, x.y - y.y, x.z - y.z, y.w, sq[e], k, pr, pim, g);
        }
        if (POT) phi[2 * (int64_t)i] = pr * k_inv4pi<T>(), phi[2 * (int64_t)i + 1] = pim * k_inv4pi<T>();
        if (GRAD)
            for (int a = 0; a < 6; ++a) grad[6 * (int64_t)i + a] = g[a] * k_inv4pi<T>();
    }
}

template <typename T>
__global__ void gather_qc_kernel(const T *__restrict__ q, const int *__restrict__ perm,
                                 typename V4<T>::type *__restrict__ pts, T *__restrict__ qi, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = perm[i];
    pts[i].w = q[2 * (int64_t)o];
    qi[i] = q[2 * (int64_t)o + 1];
}

template <typename T>
__global__ void scatter_c_kernel(const T *__restrict__ np, const T *__restrict__ ng, const T *__restrict__ fp,
                                 const T *__restrict__ fg, const int *__restrict__ perm, T *__restrict__ phi,
                                 T *__restrict__ grad, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    if (phi)
        for (int c = 0; c < 2; ++c) phi[2 * o + c] = (np ? np[2 * i + c] : (T)0) + (fp ? fp[2 * i + c] : (T)0);
    if (grad)
        for (int c = 0; c < 6; ++c) grad[6 * o + c] = (ng ? ng[6 * i + c] : (T)0) + (fg ? fg[6 * i + c] : (T)0);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t launch_gather_points_c(const T *q, const int *perm, void *pts, T *qi, int64_t n, cudaStream_t s) {
    gather_qc_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(q, perm, (typename V4<T>::type *)pts, qi, n);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_c(const T *np, const T *ng, const T *fp, const T *fg, const int *perm, T *phi, T *grad,
                             int64_t n, cudaStream_t s) {
    scatter_c_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(np, ng, fp, fg, perm, phi, grad, n);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t helm_p2p(const fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s) {
    if (ctx->nleaf == 0) return cudaSuccess;
    using P = typename V4<T>::type;
    const T k = (T)ctx->opt.kappa;
    auto go = [&](auto kern) {
        kern<<<ctx->nleaf, kThreads, 0, s>>>((const P *)ctx->pts, (const T *)ctx->pts_qi, ctx->leaf_off, ctx->u_off,
                                              ctx->u_idx, ctx->p2p_order, k, phi, grad);
    };
    if (phi && grad) go(helm_p2p_kernel<T, true, true>);
    else if (grad) go(helm_p2p_kernel<T, false, true>);
    else go(helm_p2p_kernel<T, true, false>);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t helm_leaf_check(const fmm_ctx *ctx, const T *grid, T *out, cudaStream_t s) {
    if (ctx->nleaf == 0) return cudaSuccess;
    const int d = ctx->opt.depth;
    const double width = ctx->side / (double)(1 << d);
    helm_check_kernel<T><<<ctx->nleaf, kThreads, 0, s>>>(
        (const typename V4<T>::type *)ctx->pts, (const T *)ctx->pts_qi, ctx->leaf_off, ctx->lev[d].keys, grid,
        ctx->npts, ctx->nsp, ctx->origin[0], ctx->origin[1], ctx->origin[2], width, 2.95 * 0.5 * width,
        (T)ctx->opt.kappa, out);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t helm_leaf_eval(const fmm_ctx *ctx, const T *grid, const T *dens, int ldd, T *phi, T *grad,
                           cudaStream_t s) {
    if (ctx->nleaf == 0) return cudaSuccess;
    const int d = ctx->opt.depth;
    const double width = ctx->side / (double)(1 << d);
    using P = typename V4<T>::type;
    const size_t smem = (sizeof(P) + sizeof(T)) * ctx->npts;
    auto go = [&](auto kern) {
        kern<<<ctx->nleaf, kThreads, smem, s>>>((const P *)ctx->pts, ctx->leaf_off, ctx->lev[d].keys, grid, ctx->npts,
                                                dens, ldd, ctx->origin[0], ctx->origin[1], ctx->origin[2], width,
                                                2.95 * 0.5 * width, (T)ctx->opt.kappa, phi, grad);
    };
    if (phi && grad) go(helm_eval_kernel<T, true, true>);
    else if (grad) go(helm_eval_kernel<T, false, true>);
    else go(helm_eval_kernel<T, true, false>);
    count_launch();
    return cudaGetLastError();
}

#define HELM_INST(T)                                                                                         \
    template cudaError_t launch_gather_points_c<T>(const T *, const int *, void *, T *, int64_t, cudaStream_t); \
    template cudaError_t launch_scatter_c<T>(const T *, const T *, const T *, const T *, const int *, T *, T *,  \
                                             int64_t, cudaStream_t);                                          \
    template cudaError_t helm_p2p<T>(const fmm_ctx *, T *, T *, cudaStream_t);                                \
    template cudaError_t helm_leaf_check<T>(const fmm_ctx *, const T *, T *, cudaStream_t);                   \
    template cudaError_t helm_leaf_eval<T>(const fmm_ctx *, const T *, const T *, int, T *, T *, cudaStream_t);
HELM_INST(float)
HELM_INST(double)
#undef HELM_INST

}  // namespace fmm
