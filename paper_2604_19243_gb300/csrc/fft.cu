// FFT form of the M2L (VLI, Algorithm 1 step 2a; Section 2.2 names it beside the BLAS form), in
// FP32 or FP64 SIMT arithmetic, Laplace kernel.
//
// The upward-equivalent and downward-check surfaces lie on the radius (p - 1)/(p - 2) lattice
// (precompute.cpp), whose spacing divides the box width, so the M2L of a transfer vector t is a
// convolution on the p^3 grid.  Per level l:
//   u'_b  = UC2E U_b                     equivalent densities of every box (two SIMT GEMMs with
//                                        the factored pseudo-inverse of the unit box; the map of
//                                        check potentials is level-invariant for Laplace)
//   û_b   = DFT_n(u'_b on the p^3 grid, zero-padded to n = 2p)       (fwd kernel)
//   ĉ_β   = sum_{α in V(β)} Ĝ_{t(β,α)} ⊙ û_α                          (hadamard kernel)
//   D_β  += IDFT_n(ĉ_β) at the surface points                         (inv kernel)
// with Ĝ_t the transform of the kernel sampled on the lattice differences of t (precomputed on
// the host for the unit box).  The frequencies (ka, kb, kc), kc in [0, n/2] (real signals), are
// processed in chunks of consecutive ka, so that the transformed vectors of one chunk of a whole
// level fit a bounded workspace and stay in L2 while the products are summed.  Every transform
// is separable: three passes of small DFTs along the axes, the zero padding skipped.
#include <algorithm>
#include <cmath>
#include <vector>

#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

constexpr int kFftMaxN = 20;       // n = 2p, p <= 10
constexpr int kFftThreads = 128;

struct FftShape {
    int p, n, nh, ns;              // order, transform size, half spectrum n/2 + 1, surface points
    double wr[kFftMaxN], wi[kFftMaxN];   // e^{-2 pi i k / n}
};

template <typename T>
__device__ __forceinline__ typename C2<T>::type cmul(typename C2<T>::type a, typename C2<T>::type b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Forward: û[b][(ka - ka0) n nh + kb nh + kc] for ka in [ka0, ka0 + nka).  One CTA per box.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
fft_fwd_kernel(FftShape sh, const T *__restrict__ u, int ldu, const int *__restrict__ surf, int nbox, int ka0,
               int nka, typename C2<T>::type *__restrict__ out) {
    using V = typename C2<T>::type;
    extern __shared__ unsigned char fft_smem[];
    const int p = sh.p, n = sh.n, nh = sh.nh;
    T *g = reinterpret_cast<T *>(fft_smem);                            // [p][p][p]
    V *x1 = reinterpret_cast<V *>(fft_smem + ((p * p * p * sizeof(T) + 15) / 16) * 16);   // [p][p][nh]
    V *x2 = x1 + p * p * nh;                                           // [p][n][nh]
    __shared__ T wr[kFftMaxN], wi[kFftMaxN];
    const int b = blockIdx.x, tid = threadIdx.x;
    if (b >= nbox) return;
    if (tid < n) wr[tid] = (T)sh.wr[tid], wi[tid] = (T)sh.wi[tid];
    for (int i = tid; i < p * p * p; i += blockDim.x) g[i] = (T)0;
    __syncthreads();
    for (int i = tid; i < sh.ns; i += blockDim.x) g[surf[i]] = u[(size_t)b * ldu + i];
    __syncthreads();
    // along c (real input, half spectrum)
    for (int e = tid; e < p * p * nh; e += blockDim.x) {
        const int kc = e % nh, ab = e / nh;
        V s = {(T)0, (T)0};
        for (int c = 0, w = 0; c < p; ++c, w = w + kc < n ? w + kc : w + kc - n) {   // w = c kc mod n
            const T v = g[ab * p + c];
            s.x += v * wr[w], s.y += v * wi[w];
        }
        x1[e] = s;
    }
    __syncthreads();
    // along b
    for (int e = tid; e < p * n * nh; e += blockDim.x) {
        const int kc = e % nh, kb = (e / nh) % n, a = e / (nh * n);
        V s = {(T)0, (T)0};
        for (int bb = 0, w = 0; bb < p; ++bb, w = w + kb < n ? w + kb : w + kb - n) {
            const V v = x1[(a * p + bb) * nh + kc];
            s.x += v.x * wr[w] - v.y * wi[w], s.y += v.x * wi[w] + v.y * wr[w];
        }
        x2[e] = s;
    }
    __syncthreads();
    // along a, for this chunk's ka only
    const int per = n * nh;
    V *o = out + (size_t)b * nka * per;
    for (int e = tid; e < nka * per; e += blockDim.x) {
        const int ka = ka0 + e / per, r = e % per;
        V s = {(T)0, (T)0};
        for (int a = 0, w = 0; a < p; ++a, w = w + ka < n ? w + ka : w + ka - n) {
            const V v = x2[a * per + r];
            s.x += v.x * wr[w] - v.y * wi[w], s.y += v.x * wi[w] + v.y * wr[w];
        }
        o[e] = s;
    }
}

// ĉ[β] = sum over the V list of β of Ĝ_t ⊙ û[α], for this chunk's frequencies.  The V list of a
// child of parent P is the children of P's 26 neighbours that are not adjacent to it, and the
// transfer vector of (target octant c, neighbour offset o, source octant c') is 2o + c' - c in
// child units, the same for every parent (table `pairs`: index t of Ĝ_t, or -1 when adjacent).
// A CTA takes kHadG consecutive parents and one slice of 32 consecutive frequencies: Ĝ of the
// slice for all 316 transfer vectors is staged in shared memory; warp g owns parent g, lane j
// frequency j of the slice, and the thread keeps the 8 children's sums in registers.  Each
// source value is then read from memory once per parent and applied to all 8 targets.
constexpr int kHadG = 16;          // parents (warps) per CTA
constexpr int kHadF = 32;          // frequencies per CTA

template <typename T>
__global__ void __launch_bounds__(kHadG * 32)
fft_hadamard_kernel(const typename C2<T>::type *__restrict__ uh, long long row, int nfreq,
                    const typename C2<T>::type *__restrict__ ghat, long long ghat_stride,
                    const uint32_t *__restrict__ pkeys, const int *__restrict__ pdense, const int *__restrict__ pchild,
                    int plevel, int nparent, const int *__restrict__ pairs, typename C2<T>::type *__restrict__ ch) {
    using V = typename C2<T>::type;
    extern __shared__ unsigned char fft_smem[];
    V *gs = reinterpret_cast<V *>(fft_smem);   // [316][32]: Ĝ_t of this slice
    __shared__ int src[kHadG][26][8];          // children of each parent's neighbours (-1: none)
    __shared__ int tgt[kHadG][8];              // children of each parent
    __shared__ int tt[26 * 8 * 8];             // transfer index of (o, c', c), -1 when adjacent
    const int tid = threadIdx.x, g = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * kHadG, f0 = blockIdx.y * kHadF, f = f0 + lane;
    const bool fl = f < nfreq;
    for (int i = tid; i < 26 * 64; i += blockDim.x) tt[i] = pairs[i];
    constexpr int kU = 8;   // staging loads in flight per thread
    for (int i0 = tid; i0 < kNumTransfer * kHadF; i0 += kU * kHadG * 32) {
        V v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = i0 + u * kHadG * 32, t = i / kHadF, j = i % kHadF;
            v[u] = (i < kNumTransfer * kHadF && f0 + j < nfreq) ? ghat[(long long)t * ghat_stride + f0 + j]
                                                                : V{(T)0, (T)0};
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * kHadG * 32 < kNumTransfer * kHadF) gs[i0 + u * kHadG * 32] = v[u];
    }
    for (int e = tid; e < kHadG * 8; e += blockDim.x) {
        const int gg = e / 8, c = e % 8, P = p0 + gg;
        tgt[gg][c] = P < nparent ? pchild[(size_t)P * 8 + c] : -1;
    }
    for (int e = tid; e < kHadG * 26; e += blockDim.x) {
        const int gg = e / 26, oi = e % 26, P = p0 + gg;
        const int o = oi < 13 ? oi : oi + 1;   // offsets of [-1,1]^3 without the centre
        int nb = -1;
        if (P < nparent) {
            int ax, ay, az;
            demorton3(pkeys[P], ax, ay, az);
            nb = dense_find(pdense, plevel, ax + o / 9 - 1, ay + (o / 3) % 3 - 1, az + o % 3 - 1);
        }
        for (int c = 0; c < 8; ++c) src[gg][oi][c] = nb >= 0 ? pchild[(size_t)nb * 8 + c] : -1;
    }
    __syncthreads();
    if (p0 + g >= nparent) return;
    V acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = {(T)0, (T)0};
    for (int oi = 0; oi < 26; ++oi) {
        V u[8];
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2) {
            const int sb = src[g][oi][c2];
            u[c2] = (sb >= 0 && fl) ? uh[(long long)sb * row + f] : V{(T)0, (T)0};
        }
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2) {
            if (src[g][oi][c2] < 0) continue;
            const int *tp = tt + (oi * 8 + c2) * 8;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int t = tp[c];
                if (t < 0) continue;   // adjacent to the target: near field, not V
                const V gv = gs[t * kHadF + lane];
                acc[c].x += gv.x * u[c2].x - gv.y * u[c2].y;
                acc[c].y += gv.x * u[c2].y + gv.y * u[c2].x;
            }
        }
    }
    if (!fl) return;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int tb = tgt[g][c];
        if (tb >= 0) ch[(long long)tb * row + f] = acc[c];
    }
}

// D[β] += the inverse transform of this chunk's part of ĉ[β], at the surface points.  One CTA
// per target.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
fft_inv_kernel(FftShape sh, const typename C2<T>::type *__restrict__ ch, int ka0, int nka,
               const int *__restrict__ surf, int nbox, T *__restrict__ D, int ldd) {
    using V = typename C2<T>::type;
    extern __shared__ unsigned char fft_smem[];
    const int p = sh.p, n = sh.n, nh = sh.nh;
    V *z1 = reinterpret_cast<V *>(fft_smem);   // [p][n][nh]
    V *z2 = z1 + p * n * nh;                   // [p][p][nh]
    __shared__ T wr[kFftMaxN], wi[kFftMaxN];
    const int b = blockIdx.x, tid = threadIdx.x;
    if (b >= nbox) return;
    if (tid < n) wr[tid] = (T)sh.wr[tid], wi[tid] = (T)sh.wi[tid];
    __syncthreads();
    const int per = n * nh;
    const V *c = ch + (size_t)b * nka * per;
    // along ka (this chunk's ka only) to a < p; the inverse uses the conjugate roots
    for (int e = tid; e < p * per; e += blockDim.x) {
        const int a = e / per, r = e % per;
        V s = {(T)0, (T)0};
        for (int k = 0, w = (a * ka0) % n; k < nka; ++k, w = w + a < n ? w + a : w + a - n) {
            const V v = c[k * per + r];
            s.x += v.x * wr[w] + v.y * wi[w], s.y += v.y * wr[w] - v.x * wi[w];
        }
        z1[e] = s;
    }
    __syncthreads();
    // along kb to b < p
    for (int e = tid; e < p * p * nh; e += blockDim.x) {
        const int kc = e % nh, bb = (e / nh) % p, a = e / (nh * p);
        V s = {(T)0, (T)0};
        for (int kb = 0, w = 0; kb < n; ++kb, w = w + bb < n ? w + bb : w + bb - n) {
            const V v = z1[(a * n + kb) * nh + kc];
            s.x += v.x * wr[w] + v.y * wi[w], s.y += v.y * wr[w] - v.x * wi[w];
        }
        z2[e] = s;
    }
    __syncthreads();
    // along kc, complex to real (the half spectrum: kc = 0 and n/2 once, the others twice), at
    // the surface points, scaled by 1/n^3
    const T scale = (T)1 / ((T)n * (T)n * (T)n);
    for (int i = tid; i < sh.ns; i += blockDim.x) {
        const int q = surf[i], cc = q % p, ab = q / p;
        T y = (T)0;
        for (int kc = 0, w = 0; kc < nh; ++kc, w = w + cc < n ? w + cc : w + cc - n) {
            const V v = z2[ab * nh + kc];
            const T re = v.x * wr[w] + v.y * wi[w];   // Re(v e^{+2 pi i cc kc / n})
            y += (kc == 0 || 2 * kc == n) ? re : (T)2 * re;
        }
        D[(size_t)b * ldd + i] += y * scale;
    }
}

FftShape make_shape(int p) {
    FftShape s{};
    s.p = p, s.n = 2 * p, s.nh = p + 1, s.ns = 6 * (p - 1) * (p - 1) + 2;
    for (int k = 0; k < s.n; ++k) {
        s.wr[k] = std::cos(2.0 * M_PI * k / s.n);
        s.wi[k] = -std::sin(2.0 * M_PI * k / s.n);
    }
    return s;
}

template <typename T> size_t fwd_smem(const FftShape &s) {
    using V = typename C2<T>::type;
    return ((s.p * s.p * s.p * sizeof(T) + 15) / 16) * 16 + (size_t)(s.p * s.p * s.nh + s.p * s.n * s.nh) * sizeof(V);
}
template <typename T> size_t inv_smem(const FftShape &s) {
    using V = typename C2<T>::type;
    return (size_t)(s.p * s.n * s.nh + s.p * s.p * s.nh) * sizeof(V);
}

}  // namespace

// Kernel transforms (FP32 or FP64 complex, [316][nf]) and the surface point -> grid index table.
cudaError_t fft_upload(fmm_ctx *ctx) {
    const HostOps &h = *ctx->host_ops[ctx->opt.depth];
    const int p = ctx->opt.order_p, n = h.fft_n, nf = n * n * (n / 2 + 1);
    const size_t count = (size_t)kNumTransfer * nf;
    void *d = nullptr;
    if (ctx->fp64) {
        FMM_CUDA_TRY(dev_malloc(&d, count * sizeof(double2)));
        FMM_CUDA_TRY(cudaMemcpy(d, h.fft_ghat.data(), count * sizeof(double2), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(h.fft_ghat.begin(), h.fft_ghat.end());
        FMM_CUDA_TRY(dev_malloc(&d, count * sizeof(float2)));
        FMM_CUDA_TRY(cudaMemcpy(d, f.data(), count * sizeof(float2), cudaMemcpyHostToDevice));
    }
    ctx->op_allocs.push_back(d);
    ctx->fft_ghat = d;
    std::vector<int> surf;
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b)
            for (int c = 0; c < p; ++c)
                if (a == 0 || b == 0 || c == 0 || a == p - 1 || b == p - 1 || c == p - 1)
                    surf.push_back((a * p + b) * p + c);
    FMM_CUDA_TRY(dev_malloc((void **)&ctx->fft_surf, surf.size() * sizeof(int)));
    ctx->op_allocs.push_back(ctx->fft_surf);
    FMM_CUDA_TRY(cudaMemcpy(ctx->fft_surf, surf.data(), surf.size() * sizeof(int), cudaMemcpyHostToDevice));
    // transfer index of every (dx, dy, dz) in [-3, 3]^3 (the order of the kernel transforms:
    // lexicographic, the near range |d| <= 1 left out), -1 in the near range; then the index of
    // (neighbour offset o, source octant c', target octant c) with d = 2o + c' - c
    std::vector<int> tix(343, -1);
    int t = 0;
    for (int i = -3; i <= 3; ++i)
        for (int j = -3; j <= 3; ++j)
            for (int k = -3; k <= 3; ++k)
                if (std::max(std::abs(i), std::max(std::abs(j), std::abs(k))) > 1) tix[((i + 3) * 7 + j + 3) * 7 + k + 3] = t++;
    if (t != kNumTransfer) return cudaErrorInvalidValue;
    std::vector<int> pairs(26 * 64);
    for (int oi = 0; oi < 26; ++oi) {
        const int o = oi < 13 ? oi : oi + 1, ox = o / 9 - 1, oy = (o / 3) % 3 - 1, oz = o % 3 - 1;
        for (int c2 = 0; c2 < 8; ++c2)
            for (int c = 0; c < 8; ++c) {
                const int dx = 2 * ox + ((c2 >> 2) & 1) - ((c >> 2) & 1), dy = 2 * oy + ((c2 >> 1) & 1) - ((c >> 1) & 1),
                          dz = 2 * oz + (c2 & 1) - (c & 1);
                pairs[(oi * 8 + c2) * 8 + c] = tix[((dx + 3) * 7 + dy + 3) * 7 + dz + 3];
            }
    }
    FMM_CUDA_TRY(dev_malloc((void **)&ctx->fft_tindex, pairs.size() * sizeof(int)));
    ctx->op_allocs.push_back(ctx->fft_tindex);
    FMM_CUDA_TRY(cudaMemcpy(ctx->fft_tindex, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice));
    return cudaSuccess;
}

// The FFT M2L of level l added into D (the level's downward check rows), the rows U being the
// level's upward check potentials.  Workspaces come from the stream-ordered pool.
template <typename T>
cudaError_t fft_vli(fmm_ctx *ctx, int l, const T *U, T *D, cudaStream_t s) {
    using V = typename C2<T>::type;
    const LevelTables &L = ctx->lev[l];
    const int64_t nb = L.n;
    if (nb == 0) return cudaSuccess;
    const OpSet &o = ctx->fwd[l];
    const int nsp = ctx->nsp, p = ctx->opt.order_p;
    const FftShape sh = make_shape(p);
    const int per = sh.n * sh.nh;
    // ka values per chunk: every frequency at once when the level's transformed vectors fit the
    // workspace budget (the forward transform is then computed once per box), else fewer
    const size_t budget = (size_t)4 << 30;
    const int nka = (int)std::max<int64_t>(1, std::min<int64_t>(sh.n, (int64_t)(budget / ((size_t)nb * per * sizeof(V)))));
    const int chunk = nka * per;
    Scratch<T> t1, up;
    Scratch<V> uh, ch;
    FMM_CUDA_TRY(t1.alloc((size_t)nb * o.rclup, s));
    FMM_CUDA_TRY(up.alloc((size_t)nb * nsp, s));
    FMM_CUDA_TRY(uh.alloc((size_t)nb * chunk, s));
    FMM_CUDA_TRY(ch.alloc((size_t)nb * chunk, s));
    // u' = UC2E U through the factored pseudo-inverse
    GemmCall c1;
    c1.mode = GM_IDENTITY, c1.level = l, c1.n_out = o.rclup;
    c1.X0 = U, c1.ldx0 = nsp, c1.k0 = nsp, c1.W0 = o.uclose1;
    c1.Y = t1.p, c1.ldy = o.rclup;
    FMM_CUDA_TRY(gemm_simt<T>(ctx, c1, s));
    GemmCall c2;
    c2.mode = GM_IDENTITY, c2.level = l, c2.n_out = nsp;
    c2.X0 = t1.p, c2.ldx0 = o.rclup, c2.k0 = o.rclup, c2.W0 = o.uclose2;
    c2.Y = up.p, c2.ldy = nsp;
    FMM_CUDA_TRY(gemm_simt<T>(ctx, c2, s));
    const V *ghat = (const V *)ctx->fft_ghat;
    const size_t fs = fwd_smem<T>(sh), is = inv_smem<T>(sh);
    if (fs > 48 * 1024) FMM_CUDA_TRY(cudaFuncSetAttribute(fft_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs));
    if (is > 48 * 1024) FMM_CUDA_TRY(cudaFuncSetAttribute(fft_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)is));
    const size_t hs = (size_t)kNumTransfer * kHadF * sizeof(V);
    FMM_CUDA_TRY(cudaFuncSetAttribute(fft_hadamard_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs));
    for (int ka0 = 0; ka0 < sh.n; ka0 += nka) {
        const int k = std::min(nka, sh.n - ka0);
        fft_fwd_kernel<T><<<(unsigned)nb, kFftThreads, fs, s>>>(sh, up.p, nsp, ctx->fft_surf, (int)nb, ka0, k, uh.p);
        count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        const LevelTables &P = ctx->lev[l - 1];
        const dim3 hg((unsigned)((P.n + kHadG - 1) / kHadG), (unsigned)((k * per + kHadF - 1) / kHadF));
        fft_hadamard_kernel<T><<<hg, kHadG * 32, hs, s>>>(uh.p, (long long)k * per, k * per, ghat + (size_t)ka0 * per,
                                                          (long long)sh.n * per, P.keys, P.dense, P.child, l - 1,
                                                          (int)P.n, ctx->fft_tindex, ch.p);
        count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        fft_inv_kernel<T><<<(unsigned)nb, kFftThreads, is, s>>>(sh, ch.p, ka0, k, ctx->fft_surf, (int)nb, D, nsp);
        count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

template cudaError_t fft_vli<float>(fmm_ctx *, int, const float *, float *, cudaStream_t);
template cudaError_t fft_vli<double>(fmm_ctx *, int, const double *, double *, cudaStream_t);

}  // namespace fmm
