// Outputs written straight into pinned (mapped) host memory: the near- and far-field sums of
// every point, in the caller's order, cross the host link once, with no staging buffer and no
// separate copy.
#include <algorithm>

#include "debugcheck.cuh"
#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

constexpr int kOutThreads = 256;

// Store m values of shared memory to dst with 16-byte vectors where dst is 16-byte aligned (the
// host link carries whole lines better than scattered words), the rest one by one.
template <typename T>
__device__ __forceinline__ void store_run(T *__restrict__ dst, const T *src, int m) {
    constexpr int v = 16 / sizeof(T);
    const bool aligned = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
    const int mv = aligned ? m / v : 0;
    for (int j = threadIdx.x; j < mv; j += blockDim.x)
        reinterpret_cast<float4 *>(dst)[j] = reinterpret_cast<const float4 *>(src)[j];
    for (int j = mv * v + threadIdx.x; j < m; j += blockDim.x) dst[j] = src[j];
}

// Block b: outputs [256 b, 256 b + 256).  Thread t reads the sorted position inv[o] of input o
// and sums the near and far parts into shared memory; the block then writes its potentials and
// gradients as contiguous runs.
template <typename T>
__global__ void __launch_bounds__(kOutThreads)
gather_out_kernel(const T *__restrict__ near_phi, const T *__restrict__ near_grad, const T *__restrict__ far_phi,
                  const T *__restrict__ far_grad, const int *__restrict__ inv, T *__restrict__ phi,
                  T *__restrict__ grad, int64_t n) {
    __shared__ __align__(16) T sp[kOutThreads];
    __shared__ __align__(16) T sg[3 * kOutThreads];
    const int64_t o0 = (int64_t)blockIdx.x * kOutThreads;
    const int m = n - o0 < kOutThreads ? (int)(n - o0) : kOutThreads, t = threadIdx.x;
    if (t < m) {
        int i = inv[o0 + t];
        if (!dbg_ok(i >= 0 && i < n, kDbgScatter)) i = 0;
        T v = 0;
        if (near_phi) v += near_phi[i];
        if (far_phi) v += far_phi[i];
        sp[t] = v;
        for (int a = 0; a < 3; ++a) {
            T g = 0;
            if (near_grad) g += near_grad[3 * (int64_t)i + a];
            if (far_grad) g += far_grad[3 * (int64_t)i + a];
            sg[3 * t + a] = g;
        }
    }
    __syncthreads();
    if (phi) store_run(phi + o0, sp, m);
    if (grad) store_run(grad + 3 * o0, sg, 3 * m);
}

__global__ void invert_perm_kernel(const int *__restrict__ perm, int64_t n, int *__restrict__ inv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = perm[i];
    if (dbg_ok(o >= 0 && o < n, kDbgScatter)) inv[o] = (int)i;
}

unsigned blocks(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t launch_gather_out(const T *near_phi, const T *near_grad, const T *far_phi, const T *far_grad,
                              const int *inv, T *phi, T *grad, int64_t n, cudaStream_t s) {
    gather_out_kernel<T><<<blocks(n, kOutThreads), kOutThreads, 0, s>>>(near_phi, near_grad, far_phi, far_grad, inv,
                                                                       phi, grad, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_invert_perm(const int *perm, int64_t n, int *inv, cudaStream_t s) {
    invert_perm_kernel<<<blocks(n, 256), 256, 0, s>>>(perm, n, inv);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_gather_out<float>(const float *, const float *, const float *, const float *, const int *,
                                              float *, float *, int64_t, cudaStream_t);
template cudaError_t launch_gather_out<double>(const double *, const double *, const double *, const double *,
                                               const int *, double *, double *, int64_t, cudaStream_t);

FMM_DEBUG_UNIT(output)

}  // namespace fmm
