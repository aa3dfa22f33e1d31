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

// FP32 ULI on pairs of sources: the two-wide FP32 instructions (add, mul, fma on float2) do the
// arithmetic of two (target, source) pairs per issue slot.  The U list's leaves form one sequence of
// sources, staged kChunk at a time across leaf boundaries (fewer barriers than one leaf per stage),
// and a chunk's sources are staged as pairs
// (j, k): A = [-x_j -x_k -y_j -y_k], B = [-z_j -z_k Re s_j Re s_k], C = [Im s_j Im s_k], padded with
// a zero density to an even count, so that one add forms x - y.  The reciprocal square root, the
// argument reduction and the hardware sine and cosine stay per lane.
template <bool POT, bool GRAD>
__global__ void __launch_bounds__(kThreads)
helm_p2p_f32_kernel(const float4 *__restrict__ pts, const float *__restrict__ qi, const int *__restrict__ leaf_off,
                    const int *__restrict__ u_off, const int *__restrict__ u_idx, const int *__restrict__ order, float k,
                    float *__restrict__ phi, float *__restrict__ grad) {
    constexpr int kPairs = kChunk / 2;
    __shared__ __align__(16) float4 sa[kPairs], sb[kPairs];
    __shared__ __align__(16) float2 sc[kPairs];
    __shared__ int rbeg[27], rlen[27];
    __shared__ int nr, total;
    const int b = order[blockIdx.x];
    const int t0 = leaf_off[b], t1 = leaf_off[b + 1];
    if (threadIdx.x == 0) {   // the U list's point ranges, one sequence of sources (at most 27 leaves)
        int n = 0, tot = 0;
        for (int e = u_off[b]; e < u_off[b + 1] && n < 27; ++e) {
            const int a = u_idx[e];
            rbeg[n] = leaf_off[a];
            rlen[n] = leaf_off[a + 1] - leaf_off[a];
            tot += rlen[n++];
        }
        nr = n, total = tot;
    }
    __syncthreads();
    const float2 k2 = make_float2(k, k);
    for (int tb = t0; tb < t1; tb += kThreads) {
        const int i = tb + threadIdx.x;
        // a warp without targets in this pass only helps stage the sources
        const bool busy = tb + (int)(threadIdx.x & ~31u) < t1;
        const float4 x = pts[min(i, t1 - 1)];
        const float2 x2 = make_float2(x.x, x.x), y2 = make_float2(x.y, x.y), z2 = make_float2(x.z, x.z);
        float2 pr = make_float2(0.f, 0.f), pim = pr, gxr = pr, gxi = pr, gyr = pr, gyi = pr, gzr = pr, gzi = pr;
        // the sources in chunks of kChunk across leaf boundaries: two barriers per chunk
        for (int c0 = 0; c0 < total; c0 += kChunk) {
            const int n = min(kChunk, total - c0), L = (n + 1) >> 1;
            __syncthreads();
            for (int j = threadIdx.x; j < 2 * L; j += kThreads) {
                const bool real = j < n;
                int g = c0 + min(j, n - 1), r = 0;   // source j of the chunk: range r, point g
                while (g >= rlen[r]) g -= rlen[r++];
                const int src = rbeg[r] + g;
                const float4 v = pts[src];
                const float q_i = real ? qi[src] : 0.f;
                float *A = reinterpret_cast<float *>(sa + (j >> 1)), *B = reinterpret_cast<float *>(sb + (j >> 1));
                float *C = reinterpret_cast<float *>(sc + (j >> 1));
                const int h = j & 1;
                A[h] = -v.x, A[2 + h] = -v.y, B[h] = -v.z, B[2 + h] = real ? v.w : 0.f, C[h] = q_i;
            }
            __syncthreads();
            for (int e2 = 0; e2 < (busy ? L : 0); ++e2) {
                const float4 A = sa[e2], B = sb[e2];
                const float2 qim = sc[e2], qre = make_float2(B.z, B.w);
                const float2 dx = __fadd2_rn(make_float2(A.x, A.y), x2);    // x - y
                const float2 dy = __fadd2_rn(make_float2(A.z, A.w), y2);
                const float2 dz = __fadd2_rn(make_float2(B.x, B.y), z2);
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                const float2 ri = make_float2(r2.x > 0.f ? rsqrtf(r2.x) : 0.f, r2.y > 0.f ? rsqrtf(r2.y) : 0.f);
                const float2 kr = __fmul2_rn(k2, __fmul2_rn(r2, ri));
                float2 sn, cs;
                sincos_c(kr.x, &sn.x, &cs.x);
                sincos_c(kr.y, &sn.y, &cs.y);
                // w = s e^{ikr} / r
                const float2 nqi = __fmul2_rn(qim, make_float2(-1.f, -1.f));
                const float2 wr = __fmul2_rn(__ffma2_rn(qre, cs, __fmul2_rn(nqi, sn)), ri);
                const float2 wi = __fmul2_rn(__ffma2_rn(qre, sn, __fmul2_rn(qim, cs)), ri);
                if (POT) {
                    pr = __fadd2_rn(pr, wr);
                    pim = __fadd2_rn(pim, wi);
                }
                if (GRAD) {
                    // z = w (i k r - 1) / r^2: zr = -(wr + kr wi) / r^2, zi = -(wi - kr wr) / r^2
                    const float2 nri2 = __fmul2_rn(ri, __fmul2_rn(ri, make_float2(-1.f, -1.f)));
                    const float2 nkr = __fmul2_rn(kr, make_float2(-1.f, -1.f));
                    const float2 zr = __fmul2_rn(__ffma2_rn(kr, wi, wr), nri2);
                    const float2 zi = __fmul2_rn(__ffma2_rn(nkr, wr, wi), nri2);
                    gxr = __ffma2_rn(zr, dx, gxr), gxi = __ffma2_rn(zi, dx, gxi);
                    gyr = __ffma2_rn(zr, dy, gyr), gyi = __ffma2_rn(zi, dy, gyi);
                    gzr = __ffma2_rn(zr, dz, gzr), gzi = __ffma2_rn(zi, dz, gzi);
                }
            }
        }
        if (i < t1) {
            const float f = k_inv4pi<float>();
            if (POT) phi[2 * (int64_t)i] = (pr.x + pr.y) * f, phi[2 * (int64_t)i + 1] = (pim.x + pim.y) * f;
            if (GRAD) {
                float *g = grad + 6 * (int64_t)i;
                g[0] = (gxr.x + gxr.y) * f, g[1] = (gxi.x + gxi.y) * f;
                g[2] = (gyr.x + gyr.y) * f, g[3] = (gyi.x + gyi.y) * f;
                g[4] = (gzr.x + gzr.y) * f, g[5] = (gzi.x + gzi.y) * f;
            }
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
    if constexpr (std::is_same<T, float>::value) {
        if (phi && grad) go(helm_p2p_f32_kernel<true, true>);
        else if (grad) go(helm_p2p_f32_kernel<false, true>);
        else go(helm_p2p_f32_kernel<true, false>);
    } else {
        if (phi && grad) go(helm_p2p_kernel<T, true, true>);
        else if (grad) go(helm_p2p_kernel<T, false, true>);
        else go(helm_p2p_kernel<T, true, false>);
    }
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
