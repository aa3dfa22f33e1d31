// SIMT (CUDA-core) form of the gathered GEMM of gemm_common.cuh, in FP32 or FP64.
// This is the plain-precision path (FMM_FP32 / FMM_FP64): a BM x BN output tile per CTA,
// source rows gathered into shared memory BK columns at a time, 4 x 4 register blocking.
#include <algorithm>

#include "gemm_common.cuh"

namespace fmm {
namespace {

constexpr int BM = 64, BN = 32, BK = 16, THREADS = 128;   // 4 x 4 outputs per thread

// A tile of the level's row list may be taller than BM (the tensor-core tiles are 128 rows):
// blockIdx.x enumerates (tile, BM-row slice) pairs, `subs` slices per tile.
template <typename T>
__global__ void __launch_bounds__(THREADS) gemm_simt_kernel(GemmDev g, int subs) {
    __shared__ T As[BK][BM + 4];
    __shared__ T Ws[BK][BN + 4];
    __shared__ int src[BM];
    __shared__ int box[BM];
    const Tile t = g.tiles[blockIdx.x / subs];
    const int r_off = (blockIdx.x % subs) * BM;     // first tile row of this slice
    const int nrows = min(BM, t.nrows - r_off);     // may be <= 0 for a short tile
    const int n0 = blockIdx.y * BN;
    const int tid = threadIdx.x;
    const int tr = tid / 8, tc = tid % 8;          // 16 x 8 thread grid -> rows tr*4.., cols tc*4..
    if (nrows <= 0) return;
    if (tid < BM) box[tid] = tid < nrows ? gemm_row_box(g, t, r_off + tid) : -1;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    const int nseg = gemm_nseg(g);
    for (int seg = 0; seg < nseg; ++seg) {
        if (!gemm_seg_active(g, t, seg)) continue;
        __syncthreads();
        if (tid < BM) src[tid] = box[tid] >= 0 ? gemm_src_row(g, t, box[tid], seg) : -1;
        const bool second = g.mode == GM_PARENT2 && seg == 1;
        const T *X = (const T *)(second ? g.X1 : g.X0);
        const int ldx = second ? g.ldx1 : g.ldx0;
        const int K = gemm_seg_k(g, seg);
        const T *W = second ? (const T *)g.W1[t.cls] : (const T *)g.W0 + gemm_w_index(g, t, seg) * g.w_stride;
        for (int k0 = 0; k0 < K; k0 += BK) {
            __syncthreads();
            // A tile: BM rows x BK columns, stored transposed
            for (int e = tid; e < BM * BK; e += THREADS) {
                int r = e / BK, k = e % BK;
                int sr = src[r];
                As[k][r] = (sr >= 0 && k0 + k < K) ? X[(size_t)sr * ldx + k0 + k] : (T)0;
            }
            // W tile: BN output rows x BK columns, stored transposed
            for (int e = tid; e < BN * BK; e += THREADS) {
                int n = e / BK, k = e % BK;
                Ws[k][n] = (n0 + n < g.n_out && k0 + k < K) ? W[(size_t)(n0 + n) * K + k0 + k] : (T)0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < BK; ++k) {
                T a[4], w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[k][tr * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = Ws[k][tc * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * w[j];
            }
        }
    }
    T *Y = (T *)g.Y;
    const T alpha = sizeof(T) == 8 ? (T)g.alpha_d : (T)g.alpha;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int r = tr * 4 + i;
        if (r >= nrows) continue;
        int b = box[r];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tc * 4 + j;
            if (n >= g.n_out) continue;
            T v = alpha * acc[i][j];
            T *y = Y + (size_t)b * g.ldy + n;
            *y = g.accumulate ? *y + v : v;
        }
    }
}

}  // namespace

GemmDev make_gemm_dev(const fmm_ctx *ctx, const GemmCall &c);

template <typename T>
cudaError_t gemm_simt(const fmm_ctx *ctx, const GemmCall &c, cudaStream_t s) {
    GemmDev g = make_gemm_dev(ctx, c);
    const TileSet &ts = c.tiles ? *c.tiles
                        : (c.mode == GM_STENCIL || c.mode == GM_PARENT2) ? ctx->tiles_cls[c.level]
                                                                         : ctx->tiles_plain[c.level];
    if (ts.ntiles == 0) return cudaSuccess;
    g.tiles = ts.tiles;
    g.masks = ts.masks;
    if (c.mode == GM_STENCIL && ctx->masks_ev) {   // the masks are computed on a side stream
        cudaError_t e = cudaStreamWaitEvent(s, ctx->masks_ev, 0);
        if (e != cudaSuccess) return e;
    }
    const int tm = ts.tile_m ? ts.tile_m : ctx->tile_m;
    const int subs = (tm + BM - 1) / BM;
    dim3 grid(ts.ntiles * subs, (c.n_out + BN - 1) / BN);
    gemm_simt_kernel<T><<<grid, THREADS, 0, s>>>(g, subs); count_launch();
    return cudaGetLastError();
}

template cudaError_t gemm_simt<float>(const fmm_ctx *, const GemmCall &, cudaStream_t);
template cudaError_t gemm_simt<double>(const fmm_ctx *, const GemmCall &, cudaStream_t);

}  // namespace fmm
