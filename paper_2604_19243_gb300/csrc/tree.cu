// Octree construction on the GPU (Section 2.1 of the paper, uniform refinement):
//   1. bounding cube (given, or from the points' extent),
//   2. Morton key of every point at depth d,
//   3. stable LSD radix sort of (key, input index),
//   4. leaf run-lengths, the non-empty boxes of every level, parent/child tables,
//   5. dense key -> box tables (the GPU stand-in for the hashing of non-empty keys: with a
//      uniform tree a direct-address table of 8^l entries is cheaper than a hash),
//   6. U lists of the leaves (colleagues plus self, Table 1), and for the VLI the boxes of each
//      level ordered by child octant with per-tile masks of the transfer vectors that occur
//      (the stencil existence checks of Section 2.2).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "debugcheck.cuh"
#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------------------
// exclusive scan (three-phase: block scans, scan of block sums, add-back)
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

template <typename T>
__global__ void scan_blocks(T *d, int64_t n, T *block_sums) {
    __shared__ T warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T run = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        T x = k < n ? d[k] : (T)0;
        v[i] = run;
        run += x;
    }
    // inclusive scan of per-thread totals within the warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? warp_tot[lane] : (T)0;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    T excl = inc - run + (warp > 0 ? warp_tot[warp - 1] : (T)0);
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        if (k < n) d[k] = v[i] + excl;
    }
    if (threadIdx.x == kScanThreads - 1 && block_sums) block_sums[blockIdx.x] = excl + run;
}

template <typename T>
__global__ void scan_add(T *d, int64_t n, const T *offsets) {
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    const T add = offsets[blockIdx.x];
    for (int i = threadIdx.x; i < kScanBlock; i += kScanThreads) {
        int64_t k = base + i;
        if (k < n) d[k] += add;
    }
}

template <typename T>
__global__ void scan_total(const T *d_scanned, const T *d_orig_last, int64_t n, T *total) {
    // total = scanned[n-1] + original last value (saved before the scan)
    *total = n > 0 ? d_scanned[n - 1] + *d_orig_last : (T)0;
}

}  // namespace

template <typename T>
cudaError_t exclusive_scan(T *d, int64_t n, T *d_total, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) FMM_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(T), s));
        return cudaSuccess;
    }
    Scratch<T> last;
    if (d_total) {
        FMM_CUDA_TRY(last.alloc(1, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(last.p, d + n - 1, sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        scan_blocks<T><<<1, kScanThreads, 0, s>>>(d, n, nullptr); count_launch();
    } else {
        Scratch<T> sums;
        FMM_CUDA_TRY(sums.alloc(nb, s));
        scan_blocks<T><<<(unsigned)nb, kScanThreads, 0, s>>>(d, n, sums.p); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        FMM_CUDA_TRY(exclusive_scan<T>(sums.p, nb, nullptr, s));
        scan_add<T><<<(unsigned)nb, kScanThreads, 0, s>>>(d, n, sums.p); count_launch();
    }
    FMM_CUDA_TRY(cudaGetLastError());
    if (d_total) {
        scan_total<T><<<1, 1, 0, s>>>(d, last.p, n, d_total); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}
template cudaError_t exclusive_scan<int>(int *, int64_t, int *, cudaStream_t);
template cudaError_t exclusive_scan<long long>(long long *, int64_t, long long *, cudaStream_t);

namespace {

// ---------------------------------------------------------------------------------------
// domain and Morton keys
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void extent_kernel(const T *xyz, int64_t n, double *minmax /*[6]*/, int *bad) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            double v = (double)xyz[3 * i + a];
            if (!isfinite(v)) nonfinite = 1;
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    }
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    if ((threadIdx.x & 31) == 0) {
        // doubles have no native atomicMin; order-preserving map to signed 64-bit integers
        for (int a = 0; a < 3; ++a) {
            long long l = __double_as_longlong(lo[a]), h = __double_as_longlong(hi[a]);
            l = l >= 0 ? l : (l ^ 0x7fffffffffffffffLL);
            h = h >= 0 ? h : (h ^ 0x7fffffffffffffffLL);
            atomicMin((long long *)&minmax[a], l);
            atomicMax((long long *)&minmax[3 + a], h);
        }
        if (nonfinite) atomicOr(bad, 1);
    }
}

long long ordered_bits(double v) {
    long long l;
    memcpy(&l, &v, sizeof(l));
    return l >= 0 ? l : (l ^ 0x7fffffffffffffffLL);
}
double from_ordered_bits(long long l) {
    l = l >= 0 ? l : (l ^ 0x7fffffffffffffffLL);
    double v;
    memcpy(&v, &l, sizeof(v));
    return v;
}

// anchor a = min(max(floor((x - o) * scale), 0), 2^d - 1), every FP64 operation rounded
// separately (no fused multiply-add) so that the host oracle reproduces it bit for bit.
template <typename T>
__device__ __forceinline__ uint32_t anchor_fp64(T x, double o, double scale, double amax) {
    double t = __dmul_rn(__dsub_rn((double)x, o), scale);
    t = floor(t);
    t = fmin(fmax(t, 0.0), amax);
    return (uint32_t)t;
}

// The same anchor from FP32 arithmetic where that is provably the same integer: t32 =
// (x - o32) * s32 is within 2^-24 (s (|o| + 2 |x - o32|) + |t32|) of the exact (x - o) * s
// (one rounding each for o32, s32, the difference and the product), and the FP64 value is
// within 2^-50 of it.  When the fractional part of t32 is farther than four times that bound
// from 0 and from 1, all three floor to the same integer; otherwise (a point within rounding
// distance of a box face) the FP64 form decides.  FP64 arithmetic is slow on this part, and
// this leaves it to a vanishing fraction of the points.
__device__ __forceinline__ uint32_t anchor_fast(float x, double o, double scale, float o32, float s32, float amax32,
                                                double amax) {
    const float d = __fsub_rn(x, o32);
    const float t = __fmul_rn(d, s32);
    const float bound = 2.4e-7f * (s32 * (fabsf(o32) + 2.f * fabsf(d)) + fabsf(t)) + 1e-6f;   // 4 x 2^-24 x (...)
    const float fl = floorf(t);
    const float fr = t - fl;
    if (fr > bound && 1.f - fr > bound && fabsf(t) < 8388608.f) return (uint32_t)fminf(fmaxf(fl, 0.f), amax32);
    return anchor_fp64<float>(x, o, scale, amax);
}

// A non-finite coordinate sets *bad (when given).
// (The FP32 copies of the origin and scale come from the host: conversions from FP64 would
// run on the FP64 pipe for every point.)
template <typename T>
__global__ void morton_kernel(const T *xyz, int64_t n, double ox, double oy, double oz,
                              double scale, int depth, uint32_t *keys, int *idx, int *bad,
                              float ox32, float oy32, float oz32, float s32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double o[3] = {ox, oy, oz};
    const float o32[3] = {ox32, oy32, oz32};
    const double amax = (double)((1 << depth) - 1);
    const float amax32 = (float)((1 << depth) - 1);
    uint32_t a[3];
    for (int k = 0; k < 3; ++k) {
        const T x = xyz[3 * i + k];
        if (bad && !isfinite(x)) *bad = 1;
        if constexpr (std::is_same<T, float>::value)
            a[k] = isfinite(x) ? anchor_fast(x, o[k], scale, o32[k], s32, amax32, amax)
                               : anchor_fp64<float>(x, o[k], scale, amax);
        else
            a[k] = anchor_fp64<T>(x, o[k], scale, amax);
    }
    keys[i] = morton3(a[0], a[1], a[2]);
    idx[i] = (int)i;
}

// ---------------------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, int value), 8-bit digits
// ---------------------------------------------------------------------------------------
constexpr int kSortWarps = 8;
constexpr int kSortThreads = kSortWarps * 32;
constexpr int kSortRounds = 16;                         // 32-key rounds per warp
constexpr int kSortWarpItems = 32 * kSortRounds;        // 512 keys per warp
constexpr int kSortTile = kSortWarps * kSortWarpItems;  // 4096 keys per tile

__global__ void radix_hist(const uint32_t *keys, int64_t n, int shift, int ntiles, int *hist) {
    __shared__ int cnt[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        int64_t k = base + i;
        if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = cnt[d];
}

// Scatter of one 4096-key tile: the tile is first ordered by digit in shared memory (stable:
// warp, then round, then lane order), then every digit run is written out by consecutive
// threads to consecutive addresses, so that the global writes are coalesced.
__global__ void radix_scatter(const uint32_t *keys, const int *vals, int64_t n, int shift,
                              int ntiles, const int *offs, uint32_t *keys_out, int *vals_out) {
    __shared__ int wcnt[kSortWarps][256];   // per-warp digit counts, then tile positions
    __shared__ int dstart[256];             // tile-local start of each digit's run
    __shared__ int gbase[256];              // global start of this tile's run of each digit
    __shared__ int wsum[kSortThreads / 32];
    __shared__ uint32_t sk[kSortTile];
    __shared__ int sv[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    const int64_t wbase = tbase + (int64_t)warp * kSortWarpItems;
    const int count = n - tbase < (int64_t)kSortTile ? (int)(n - tbase) : kSortTile;
    // per-warp digit counts
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t k = wbase + r * 32 + lane;
        if (k < n) atomicAdd(&wcnt[warp][(keys[k] >> shift) & 255u], 1);
    }
    __syncthreads();
    // digit totals of the tile and their exclusive scan (one digit per thread: 256 threads)
    {
        const int d = threadIdx.x;
        int tot = 0;
        for (int w = 0; w < kSortWarps; ++w) tot += wcnt[w][d];
        int x = tot;   // inclusive scan within the warp, then across warps
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const int start = before + x - tot;
        dstart[d] = start;
        gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
        int run = start;
        for (int w = 0; w < kSortWarps; ++w) {
            const int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // tile order in shared memory
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t k = wbase + r * 32 + lane;
        bool valid = k < n;
        uint32_t key = valid ? keys[k] : 0u;
        int digit = valid ? (int)((key >> shift) & 255u) : 256 + lane;   // invalid lanes unique
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & lt);
        int pos = valid ? wcnt[warp][digit] + rank : 0;
        __syncwarp();
        if (valid && rank == 0) wcnt[warp][digit] += __popc(peers);
        __syncwarp();
        if (valid) {
            sk[pos] = key;
            sv[pos] = vals[k];
        }
    }
    __syncthreads();
    // coalesced write-out: element i of the tile order goes to its digit's global run
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const uint32_t key = sk[i];
        const int d = (int)((key >> shift) & 255u);
        const int pos = gbase[d] + (i - dstart[d]);
        if (!dbg_ok(pos >= 0 && pos < n, kDbgSort)) continue;
        keys_out[pos] = key;
        vals_out[pos] = sv[i];
    }
}

// Stable sort of (keys, vals) by the low `bits` bits of the keys.  Results end in (keys, vals).
cudaError_t radix_sort(uint32_t *keys, int *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    Scratch<uint32_t> k2;
    Scratch<int> v2, hist;
    FMM_CUDA_TRY(k2.alloc(n, s));
    FMM_CUDA_TRY(v2.alloc(n, s));
    FMM_CUDA_TRY(hist.alloc((size_t)256 * ntiles, s));
    uint32_t *ka = keys, *kb = k2.p;
    int *va = vals, *vb = v2.p;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        radix_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, hist.p); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        FMM_CUDA_TRY(exclusive_scan<int>(hist.p, (int64_t)256 * ntiles, nullptr, s));
        radix_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, ntiles, hist.p, kb, vb); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        FMM_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// leaves, levels and tables
// ---------------------------------------------------------------------------------------

template <typename T, typename P>
__global__ void gather_sorted_points(const T *xyz, const int *perm, int64_t n, P *pts) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = perm[i];
    P p;
    p.x = xyz[3 * j];
    p.y = xyz[3 * j + 1];
    p.z = xyz[3 * j + 2];
    p.w = 0;
    pts[i] = p;
}

// Kernels below take the element count either from the host (`cnt` null) or from device
// memory (`cnt`), with `n` then an upper bound that sizes the grid: the tree build runs from
// the keys to the U lists without reading a count back.
__device__ __forceinline__ int64_t count_of(const int *cnt, int64_t n) { return cnt ? (int64_t)*cnt : n; }

// flag[i] = 1 where a new run of (keys >> shift) starts; 0 past the count (up to n)
__global__ void run_flags(const uint32_t *keys, int64_t n, const int *cnt, int shift, int *flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i < count_of(cnt, n) && (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift))) ? 1 : 0;
}

// After an exclusive scan of the flags: runs get contiguous ids.  For every run start record
// its position (offsets) and key; for every element record its run id (optional).  The
// exclusive scan counts the starts strictly before i, so an element that does not start a run
// sees its own run's start too and its id is the scanned value minus one.
__global__ void run_compact(const uint32_t *keys, const int *flags_scanned, int64_t n, const int *cnt,
                            int shift, int *run_start, uint32_t *run_key, int *elem_run) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count_of(cnt, n)) return;
    const bool start = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift));
    const int id = flags_scanned[i] - (start ? 0 : 1);
    if (start) {
        if (run_start) run_start[id] = (int)i;
        run_key[id] = keys[i] >> shift;
    }
    if (elem_run) elem_run[i] = id;
}

// arr[pos] = value, pos from the device when given there
__global__ void set_last(int *arr, const int *pos_dev, int64_t pos, const int *value_dev, int value) {
    arr[pos_dev ? *pos_dev : pos] = value_dev ? *value_dev : value;
}

__global__ void fill_child(const uint32_t *keys, const int *parent, int64_t n, const int *cnt, int *child) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count_of(cnt, n)) return;
    child[(int64_t)parent[i] * 8 + (keys[i] & 7u)] = (int)i;
}

__global__ void fill_dense(const uint32_t *keys, int64_t n, const int *cnt, int *dense) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count_of(cnt, n)) return;
    dense[keys[i]] = (int)i;
}

// boxes per child octant (key & 7) of one level
__global__ void octant_hist(const uint32_t *keys, int64_t n, const int *cnt, int *hist8) {
    __shared__ int h[8];
    if (threadIdx.x < 8) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t c = count_of(cnt, n);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[keys[i] & 7u], 1);
    __syncthreads();
    if (threadIdx.x < 8 && h[threadIdx.x]) atomicAdd(&hist8[threadIdx.x], h[threadIdx.x]);
}

// U list of every leaf: its non-empty colleagues and itself, ascending box index (= Morton).
__global__ void u_count(const uint32_t *keys, int nbound, const int *nleaf, const int *dense, int depth, int *cnt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbound) return;
    if (b >= *nleaf) {
        cnt[b] = 0;
        return;
    }
    int ax, ay, az;
    demorton3(keys[b], ax, ay, az);
    int c = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz)
                c += dense_find(dense, depth, ax + dx, ay + dy, az + dz) >= 0;
    cnt[b] = c;
}

__global__ void u_fill(const uint32_t *keys, int nleaf, const int *dense, int depth,
                       const int *off, int *idx) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int ax, ay, az;
    demorton3(keys[b], ax, ay, az);
    int list[27];
    int c = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int j = dense_find(dense, depth, ax + dx, ay + dy, az + dz);
                if (j >= 0) {
                    int k = c++;   // insertion sort, ascending
                    while (k > 0 && list[k - 1] > j) {
                        list[k] = list[k - 1];
                        --k;
                    }
                    list[k] = j;
                }
            }
    for (int k = 0; k < c; ++k) idx[off[b] + k] = list[k];
}

// work of each leaf for the P2P: |leaf| * sum_{a in U(leaf)} |a|
__global__ void p2p_work(const int *leaf_off, const int *u_off, const int *u_idx, int nleaf,
                         uint32_t *work_key, int *order, unsigned long long *total) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    long long src = 0;
    for (int k = u_off[b]; k < u_off[b + 1]; ++k) {
        int a = u_idx[k];
        src += leaf_off[a + 1] - leaf_off[a];
    }
    long long w = src * (long long)(leaf_off[b + 1] - leaf_off[b]);
    atomicAdd(total, (unsigned long long)w);
    // descending work order through an ascending sort of a 16-bit complement: the top 16 bits
    // of the work as a float (exponent and 7 mantissa bits, monotone in w), so two radix passes
    // order the leaves by work to within 1 part in 128 (equal codes keep Morton order)
    const uint32_t code = __float_as_uint((float)w) >> 16;
    work_key[b] = 0xffffu - code;
    order[b] = b;
}

// Class keys of the boxes of every level, concatenated level after level: (level, child
// octant) as key, the index within the level as value, so that one stable sort gives every
// level's boxes in class order.
struct ClassKeyArgs {
    const uint32_t *keys[kMaxDepth + 1];
    long long base[kMaxDepth + 2];   // first row of each level; base[depth + 1] = all rows
    int depth;
};

__global__ void class_keys(ClassKeyArgs a, uint32_t *cls_key, int *idx) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= a.base[a.depth + 1]) return;
    int l = 0;
    while (r >= a.base[l + 1]) ++l;
    const long long i = r - a.base[l];
    cls_key[r] = ((uint32_t)l << 3) | (a.keys[l][i] & 7u);
    idx[r] = (int)i;
}

}  // namespace

cudaError_t stable_sort_by_key(uint32_t *keys, int *vals, int64_t n, int bits, cudaStream_t s) {
    return radix_sort(keys, vals, n, bits, s);
}

// Class slot table: for child octant c, the 189 transfer indices t (ascending) whose source
// box has a parent adjacent to (or equal to) the target's parent.
void class_slot_table(std::vector<int> &slots, std::vector<int> &deltas) {
    slots.assign(8 * kClassSlots, -1);
    deltas.assign(8 * kClassSlots, 0);
    for (int c = 0; c < 8; ++c) {
        int b[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
        int k = 0, t = 0;
        for (int i = -3; i <= 3; ++i)
            for (int j = -3; j <= 3; ++j)
                for (int l = -3; l <= 3; ++l) {
                    if (std::max(std::abs(i), std::max(std::abs(j), std::abs(l))) <= 1) continue;
                    int d[3] = {i, j, l};
                    bool ok = true;
                    for (int a = 0; a < 3; ++a) {
                        int q = b[a] + d[a];   // (2P + b + d) >> 1 - P = (b + d) >> 1
                        int pd = q >= 0 ? q / 2 : -((-q + 1) / 2);
                        if (pd < -1 || pd > 1) ok = false;
                    }
                    if (ok) {
                        deltas[c * kClassSlots + k] = pack_delta(i, j, l);
                        slots[c * kClassSlots + k++] = t;
                    }
                    ++t;
                }
    }
}

namespace {

// Per tile: bit s of masks[tile*6 + s/32] is set when some row of the tile has a non-empty
// source box for class slot s.
__global__ void tile_masks(const Tile *tiles, int ntiles, const int *cls_rows, const uint32_t *keys,
                           const int *dense, int level, const int *class_delta, uint32_t *masks) {
    __shared__ uint32_t m[6];
    __shared__ int dlt[kClassSlots][3];
    const int tid = blockIdx.x;
    if (tid >= ntiles) return;
    Tile tl = tiles[tid];
    if (threadIdx.x < 6) m[threadIdx.x] = 0;
    for (int s = threadIdx.x; s < kClassSlots; s += blockDim.x) {
        int dx, dy, dz;
        unpack_delta(class_delta[tl.cls * kClassSlots + s], dx, dy, dz);
        dlt[s][0] = dx, dlt[s][1] = dy, dlt[s][2] = dz;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < tl.nrows * kClassSlots; w += blockDim.x) {
        int r = w / kClassSlots, s = w % kClassSlots;
        int box = cls_rows[tl.row0 + r];
        int ax, ay, az;
        demorton3(keys[box], ax, ay, az);
        if (dense_find(dense, level, ax + dlt[s][0], ay + dlt[s][1], az + dlt[s][2]) >= 0)
            atomicOr(&m[s >> 5], 1u << (s & 31));
    }
    __syncthreads();
    if (threadIdx.x < 6) masks[tid * 6 + threadIdx.x] = m[threadIdx.x];
}

// V lists for export: count, then fill sorted ascending by source index.
__global__ void v_count(const uint32_t *keys, int64_t n, const int *dense, int level,
                        const int *class_delta, long long *cnt) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    uint32_t k = keys[b];
    int ax, ay, az;
    demorton3(k, ax, ay, az);
    int c = k & 7u;
    long long total = 0;
    for (int s = 0; s < kClassSlots; ++s) {
        int dx, dy, dz;
        unpack_delta(class_delta[c * kClassSlots + s], dx, dy, dz);
        total += dense_find(dense, level, ax + dx, ay + dy, az + dz) >= 0;
    }
    cnt[b] = total;
}

__global__ void v_fill(const uint32_t *keys, int64_t n, const int *dense, int level,
                       const int *class_slots, const int *class_delta, const long long *off,
                       int *idx, int *tv) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    uint32_t k = keys[b];
    int ax, ay, az;
    demorton3(k, ax, ay, az);
    int c = k & 7u;
    long long o = off[b], m = 0;
    for (int s = 0; s < kClassSlots; ++s) {
        int t = class_slots[c * kClassSlots + s];
        int dx, dy, dz;
        unpack_delta(class_delta[c * kClassSlots + s], dx, dy, dz);
        int j = dense_find(dense, level, ax + dx, ay + dy, az + dz);
        if (j < 0) continue;
        // insertion into the sorted output segment
        long long q = o + m++;
        while (q > o && idx[q - 1] > j) {
            idx[q] = idx[q - 1];
            tv[q] = tv[q - 1];
            --q;
        }
        idx[q] = j;
        tv[q] = t;
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t launch_tile_masks(const Tile *tiles, int ntiles, const int *rows, const uint32_t *keys, const int *dense,
                              int level, const int *class_delta, uint32_t *masks, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    tile_masks<<<ntiles, 256, 0, s>>>(tiles, ntiles, rows, keys, dense, level, class_delta, masks); count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// build
// ---------------------------------------------------------------------------------------

// Per-context constant tables and count buffers (allocated on the first build).
static cudaError_t ensure_build_buffers(fmm_ctx *ctx) {
    if (!ctx->dev_counts) FMM_CUDA_TRY(dev_malloc((void **)&ctx->dev_counts, kCntSize * sizeof(int)));
    if (!ctx->host_counts) FMM_CUDA_TRY(cudaMallocHost((void **)&ctx->host_counts, kCntSize * sizeof(int)));
    if (!ctx->dev_pairs) FMM_CUDA_TRY(dev_malloc((void **)&ctx->dev_pairs, sizeof(unsigned long long)));
    if (!ctx->class_slots) {
        std::vector<int> slots, deltas;
        class_slot_table(slots, deltas);
        FMM_CUDA_TRY(dev_malloc((void **)&ctx->class_slots, slots.size() * sizeof(int)));
        FMM_CUDA_TRY(dev_malloc((void **)&ctx->class_delta, deltas.size() * sizeof(int)));
        FMM_CUDA_TRY(cudaMemcpy(ctx->class_slots, slots.data(), slots.size() * sizeof(int), cudaMemcpyHostToDevice));
        FMM_CUDA_TRY(cudaMemcpy(ctx->class_delta, deltas.data(), deltas.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    return cudaSuccess;
}

// The build runs on the device from the coordinates to the U-list offsets with every box
// count kept in device memory (arrays sized by the bound min(n, 8^l) of level l), then reads
// all counts back in one copy; the remaining steps are sized on the host and stay
// stream-ordered, so that a build waits on the device once (twice without a given domain).
template <typename T>
static cudaError_t build_tree_t(fmm_ctx *ctx, const T *xyz) {
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n;
    const int depth = ctx->opt.depth;
    FMM_CUDA_TRY(ensure_build_buffers(ctx));
    int *cnt = ctx->dev_counts;
    FMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, kCntSize * sizeof(int), s));
    FMM_CUDA_TRY(cudaMemsetAsync(ctx->dev_pairs, 0, sizeof(unsigned long long), s));
    // 1. bounding cube
    if (ctx->opt.has_domain) {
        for (int a = 0; a < 3; ++a) ctx->origin[a] = ctx->opt.origin[a];
        ctx->side = ctx->opt.side;
    } else {
        Scratch<double> mm;
        FMM_CUDA_TRY(mm.alloc(6, s));
        long long init[6];
        for (int a = 0; a < 3; ++a) {
            init[a] = ordered_bits(INFINITY);
            init[3 + a] = ordered_bits(-INFINITY);
        }
        FMM_CUDA_TRY(cudaMemcpyAsync(mm.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
        extent_kernel<T><<<std::min<unsigned>(blocks_for(n, 256), 1024), 256, 0, s>>>(xyz, n, mm.p, cnt + kCntBad); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        long long res[6];
        FMM_CUDA_TRY(cudaMemcpyAsync(res, mm.p, sizeof(res), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        double ext = 0;
        for (int a = 0; a < 3; ++a) {
            double lo = from_ordered_bits(res[a]), hi = from_ordered_bits(res[3 + a]);
            ctx->origin[a] = std::isfinite(lo) ? lo : 0.0;
            if (std::isfinite(hi - lo)) ext = std::max(ext, hi - lo);
        }
        ctx->side = ext > 0 ? ext * (1.0 + std::ldexp(1.0, -20)) : 1.0;
    }
    const double scale = std::ldexp(1.0, depth) / ctx->side;
    auto bound = [&](int l) { return std::min<int64_t>(n, (int64_t)1 << (3 * l)); };
    // 2-3. keys and stable sort
    Scratch<uint32_t> keys;
    FMM_CUDA_TRY(keys.alloc(n, s));
    FMM_CUDA_TRY(pool_alloc((void **)&ctx->perm, n * sizeof(int), s));
    morton_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, ctx->origin[0], ctx->origin[1], ctx->origin[2],
                                                          scale, depth, keys.p, ctx->perm, cnt + kCntBad,
                                                          (float)ctx->origin[0], (float)ctx->origin[1],
                                                          (float)ctx->origin[2], (float)scale); count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    FMM_CUDA_TRY(radix_sort(keys.p, ctx->perm, n, 3 * depth, s));
    // sorted points (x, y, z, q=0)
    const size_t psz = ctx->fp64 ? sizeof(double4) : sizeof(float4);
    FMM_CUDA_TRY(pool_alloc(&ctx->pts, n * psz, s));
    if (ctx->fp64)
        gather_sorted_points<T, double4><<<blocks_for(n, 256), 256, 0, s>>>(xyz, ctx->perm, n, (double4 *)ctx->pts);
    else
        gather_sorted_points<T, float4><<<blocks_for(n, 256), 256, 0, s>>>(xyz, ctx->perm, n, (float4 *)ctx->pts);
    count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    // 4. leaves (runs of equal keys) and the boxes of every level (runs of equal parent keys)
    {
        Scratch<int> flags;
        FMM_CUDA_TRY(flags.alloc(n, s));
        run_flags<<<blocks_for(n, 256), 256, 0, s>>>(keys.p, n, nullptr, 0, flags.p); count_launch();
        FMM_CUDA_TRY(exclusive_scan<int>(flags.p, n, cnt + kCntLevel + depth, s));
        const int64_t bd = bound(depth);
        FMM_CUDA_TRY(pool_alloc((void **)&ctx->leaf_off, (bd + 1) * sizeof(int), s));
        FMM_CUDA_TRY(pool_alloc((void **)&ctx->lev[depth].keys, bd * sizeof(uint32_t), s));
        run_compact<<<blocks_for(n, 256), 256, 0, s>>>(keys.p, flags.p, n, nullptr, 0, ctx->leaf_off,
                                                         ctx->lev[depth].keys, nullptr); count_launch();
        set_last<<<1, 1, 0, s>>>(ctx->leaf_off, cnt + kCntLevel + depth, 0, nullptr, (int)n); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    for (int l = depth; l >= 1; --l) {
        LevelTables &C = ctx->lev[l], &P = ctx->lev[l - 1];
        const int64_t bc = bound(l), bp = bound(l - 1);
        const int *nc = cnt + kCntLevel + l;
        Scratch<int> f;
        FMM_CUDA_TRY(f.alloc(bc, s));
        run_flags<<<blocks_for(bc, 256), 256, 0, s>>>(C.keys, bc, nc, 3, f.p); count_launch();
        FMM_CUDA_TRY(exclusive_scan<int>(f.p, bc, cnt + kCntLevel + l - 1, s));
        FMM_CUDA_TRY(pool_alloc((void **)&P.keys, bp * sizeof(uint32_t), s));
        FMM_CUDA_TRY(pool_alloc((void **)&C.parent, bc * sizeof(int), s));
        run_compact<<<blocks_for(bc, 256), 256, 0, s>>>(C.keys, f.p, bc, nc, 3, nullptr, P.keys, C.parent); count_launch();
        FMM_CUDA_TRY(pool_alloc((void **)&P.child, (size_t)bp * 8 * sizeof(int), s));
        FMM_CUDA_TRY(cudaMemsetAsync(P.child, 0xff, (size_t)bp * 8 * sizeof(int), s));
        fill_child<<<blocks_for(bc, 256), 256, 0, s>>>(C.keys, C.parent, bc, nc, P.child); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    // 5. dense tables and the octant histograms
    for (int l = 0; l <= depth; ++l) {
        LevelTables &T_ = ctx->lev[l];
        const int64_t bl = bound(l);
        size_t sz = (size_t)1 << (3 * l);
        FMM_CUDA_TRY(pool_alloc((void **)&T_.dense, sz * sizeof(int), s));
        FMM_CUDA_TRY(cudaMemsetAsync(T_.dense, 0xff, sz * sizeof(int), s));
        fill_dense<<<blocks_for(bl, 256), 256, 0, s>>>(T_.keys, bl, cnt + kCntLevel + l, T_.dense); count_launch();
        if (l >= 1) {
            octant_hist<<<std::min<unsigned>(blocks_for(bl, 256), 256), 256, 0, s>>>(T_.keys, bl, cnt + kCntLevel + l,
                                                                                       cnt + kCntOct + 8 * l); count_launch();
        }
        FMM_CUDA_TRY(cudaGetLastError());
    }
    // 6. U-list sizes and offsets
    const int64_t bd = bound(depth);
    FMM_CUDA_TRY(pool_alloc((void **)&ctx->u_off, (bd + 1) * sizeof(int), s));
    u_count<<<blocks_for(bd, 128), 128, 0, s>>>(ctx->lev[depth].keys, (int)bd, cnt + kCntLevel + depth,
                                                 ctx->lev[depth].dense, depth, ctx->u_off); count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    FMM_CUDA_TRY(exclusive_scan<int>(ctx->u_off, bd, cnt + kCntU, s));
    set_last<<<1, 1, 0, s>>>(ctx->u_off, cnt + kCntLevel + depth, 0, cnt + kCntU, 0); count_launch();
    // the one read-back of the build
    int *hc = ctx->host_counts;
    FMM_CUDA_TRY(cudaMemcpyAsync(hc, cnt, kCntSize * sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hc[kCntBad]) return cudaErrorInvalidValue;   // mapped to FMM_EINVAL by the caller
    int64_t rows = 0;
    for (int l = 0; l <= depth; ++l) {
        LevelTables &T_ = ctx->lev[l];
        T_.n = hc[kCntLevel + l];
        T_.row_base = rows;
        rows += T_.n;
        T_.cls_off[0] = 0;
        for (int c = 0; c < 8; ++c) T_.cls_off[c + 1] = T_.cls_off[c] + (l >= 1 ? hc[kCntOct + 8 * l + c] : 0);
    }
    ctx->total_rows = rows;
    const int nleaf = (int)ctx->lev[depth].n;
    ctx->nleaf = nleaf;
    ctx->n_u = hc[kCntU];
    // U lists
    FMM_CUDA_TRY(pool_alloc((void **)&ctx->u_idx, std::max<int64_t>(ctx->n_u, 1) * sizeof(int), s));
    u_fill<<<blocks_for(nleaf, 128), 128, 0, s>>>(ctx->lev[depth].keys, nleaf, ctx->lev[depth].dense, depth,
                                                   ctx->u_off, ctx->u_idx); count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    // P2P schedule (decreasing work) and the total pair count (read when asked for)
    {
        Scratch<uint32_t> wk;
        FMM_CUDA_TRY(wk.alloc(nleaf, s));
        FMM_CUDA_TRY(pool_alloc((void **)&ctx->p2p_order, std::max(nleaf, 1) * sizeof(int), s));
        p2p_work<<<blocks_for(nleaf, 256), 256, 0, s>>>(ctx->leaf_off, ctx->u_off, ctx->u_idx, nleaf,
                                                          wk.p, ctx->p2p_order, ctx->dev_pairs); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        FMM_CUDA_TRY(radix_sort(wk.p, ctx->p2p_order, nleaf, 16, s));
        ctx->p2p_pairs = -1;
    }
    // class (octant) order of every level at once: one stable sort of all boxes by (level,
    // octant); level l's part starts at its row base, class offsets come from the counts
    {
        ClassKeyArgs a{};
        for (int l = 0; l <= depth; ++l) a.keys[l] = ctx->lev[l].keys, a.base[l] = ctx->lev[l].row_base;
        a.base[depth + 1] = ctx->total_rows;
        a.depth = depth;
        Scratch<uint32_t> ck;
        FMM_CUDA_TRY(ck.alloc(ctx->total_rows, s));
        FMM_CUDA_TRY(pool_alloc((void **)&ctx->cls_all, std::max<int64_t>(ctx->total_rows, 1) * sizeof(int), s));
        class_keys<<<blocks_for(ctx->total_rows, 256), 256, 0, s>>>(a, ck.p, ctx->cls_all); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        int bits = 3;
        while ((1 << (bits - 3)) <= depth) ++bits;   // level in the bits above the octant
        FMM_CUDA_TRY(radix_sort(ck.p, ctx->cls_all, ctx->total_rows, bits, s));
        for (int l = 1; l <= depth; ++l) ctx->lev[l].cls_rows = ctx->cls_all + ctx->lev[l].row_base;
    }
    return cudaSuccess;
}

cudaError_t build_tree(fmm_ctx *ctx, const void *d_xyz) {
    if (ctx->fp64) return build_tree_t<double>(ctx, (const double *)d_xyz);
    return build_tree_t<float>(ctx, (const float *)d_xyz);
}

// Tile lists of every level, copied to the device from one pinned staging buffer (reused once
// the copies out of it have completed).
cudaError_t build_tiles(fmm_ctx *ctx, int tile_m) {
    cudaStream_t s = ctx->stream;
    const int depth = ctx->opt.depth;
    std::vector<Tile> staged;
    struct Copy {
        Tile *dst;
        int count;
    };
    std::vector<Copy> copies;
    for (int l = 0; l <= depth; ++l) {
        for (TileSet *ts : {&ctx->tiles_plain[l], &ctx->tiles_cls[l]}) {
            if (ts->tiles) cudaFreeAsync(ts->tiles, s);
            if (ts->masks) cudaFreeAsync(ts->masks, s);
            ts->tiles = nullptr;
            ts->masks = nullptr;
            ts->host.clear();
            ts->ntiles = 0;
        }
        LevelTables &T_ = ctx->lev[l];
        // plain order
        TileSet &pl = ctx->tiles_plain[l];
        for (int64_t r = 0; r < T_.n; r += tile_m)
            pl.host.push_back(Tile{(int)r, (int)std::min<int64_t>(tile_m, T_.n - r), -1, 0});
        // class order
        TileSet &cl = ctx->tiles_cls[l];
        if (l >= 1)
            for (int c = 0; c < 8; ++c)
                for (int r = T_.cls_off[c]; r < T_.cls_off[c + 1]; r += tile_m)
                    cl.host.push_back(Tile{r, std::min(tile_m, T_.cls_off[c + 1] - r), c, (int)cl.host.size()});
        for (TileSet *ts : {&pl, &cl}) {
            ts->ntiles = (int)ts->host.size();
            if (!ts->ntiles) continue;
            FMM_CUDA_TRY(pool_alloc((void **)&ts->tiles, ts->ntiles * sizeof(Tile), s));
            staged.insert(staged.end(), ts->host.begin(), ts->host.end());
            copies.push_back({ts->tiles, ts->ntiles});
        }
    }
    if (!ctx->tiles_ev) FMM_CUDA_TRY(cudaEventCreateWithFlags(&ctx->tiles_ev, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventSynchronize(ctx->tiles_ev));   // earlier copies out of the staging buffer
    if (staged.size() > ctx->host_tiles_cap) {
        if (ctx->host_tiles) cudaFreeHost(ctx->host_tiles);
        ctx->host_tiles = nullptr;
        ctx->host_tiles_cap = 0;
        FMM_CUDA_TRY(cudaMallocHost((void **)&ctx->host_tiles, staged.size() * 2 * sizeof(Tile)));
        ctx->host_tiles_cap = staged.size() * 2;
    }
    std::copy(staged.begin(), staged.end(), ctx->host_tiles);
    size_t off = 0;
    for (const Copy &c : copies) {
        FMM_CUDA_TRY(cudaMemcpyAsync(c.dst, ctx->host_tiles + off, c.count * sizeof(Tile), cudaMemcpyHostToDevice, s));
        off += c.count;
    }
    FMM_CUDA_TRY(cudaEventRecord(ctx->tiles_ev, s));
    // The stencil masks are needed only by the VLI, after the upward pass: they are computed on a
    // side stream (aux[1]) while the evaluation starts, and every stencil contraction waits for
    // masks_ev first.
    for (int l = 2; l <= depth; ++l) {
        TileSet &cl = ctx->tiles_cls[l];
        if (cl.ntiles) FMM_CUDA_TRY(pool_alloc((void **)&cl.masks, (size_t)cl.ntiles * 6 * sizeof(uint32_t), s));
    }
    // (a context without the side stream, a virtual rank's, computes them in stream order)
    const bool side = ctx->aux[1] && ctx->masks_fork_ev && ctx->masks_ev;
    cudaStream_t ms = side ? ctx->aux[1] : s;
    if (side) {
        FMM_CUDA_TRY(cudaEventRecord(ctx->masks_fork_ev, s));
        FMM_CUDA_TRY(cudaStreamWaitEvent(ms, ctx->masks_fork_ev, 0));
    }
    for (int l = depth; l >= 2; --l) {
        LevelTables &T_ = ctx->lev[l];
        TileSet &cl = ctx->tiles_cls[l];
        if (!cl.ntiles) continue;
        tile_masks<<<cl.ntiles, 256, 0, ms>>>(cl.tiles, cl.ntiles, T_.cls_rows, T_.keys, T_.dense, l,
                                              ctx->class_delta, cl.masks); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    if (side) FMM_CUDA_TRY(cudaEventRecord(ctx->masks_ev, ms));
    ctx->tile_m = tile_m;
    return cudaSuccess;
}

cudaError_t export_v_lists(fmm_ctx *ctx, int level, int64_t *off, int64_t *idx, int32_t *tv,
                           int64_t *count) {
    cudaStream_t s = ctx->stream;
    LevelTables &T_ = ctx->lev[level];
    const int64_t n = T_.n;
    Scratch<long long> o;
    Scratch<long long> tot;
    FMM_CUDA_TRY(o.alloc(n + 1, s));
    FMM_CUDA_TRY(tot.alloc(1, s));
    v_count<<<blocks_for(n, 128), 128, 0, s>>>(T_.keys, n, T_.dense, level, ctx->class_delta, o.p); count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    FMM_CUDA_TRY(exclusive_scan<long long>(o.p, n, tot.p, s));
    long long total = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&total, tot.p, sizeof(total), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    if (count) *count = total;
    std::vector<long long> ho(n + 1);
    FMM_CUDA_TRY(cudaMemcpyAsync(ho.data(), o.p, n * sizeof(long long), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    ho[n] = total;
    if (off)
        for (int64_t i = 0; i <= n; ++i) off[i] = ho[i];
    if (idx || tv) {
        Scratch<int> di, dt;
        FMM_CUDA_TRY(di.alloc(total, s));
        FMM_CUDA_TRY(dt.alloc(total, s));
        v_fill<<<blocks_for(n, 128), 128, 0, s>>>(T_.keys, n, T_.dense, level, ctx->class_slots,
                                                   ctx->class_delta, o.p, di.p, dt.p); count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        std::vector<int> hi(total), ht(total);
        FMM_CUDA_TRY(cudaMemcpyAsync(hi.data(), di.p, total * sizeof(int), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(ht.data(), dt.p, total * sizeof(int), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        for (long long i = 0; i < total; ++i) {
            if (idx) idx[i] = hi[i];
            if (tv) tv[i] = ht[i];
        }
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// Table validation (fmm_debug_check): every index table of the built tree against its bounds
// and its definition, one thread per entry; a violation ORs its bit (debugcheck.cuh) into *flag.
// ---------------------------------------------------------------------------------------
namespace {

__global__ void val_count(const int *v, int64_t n, int64_t range, int *cnt, uint32_t bit, uint32_t *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = v[i];
    if (x < 0 || x >= range) atomicOr(flag, bit);
    else atomicAdd(&cnt[x], 1);
}

__global__ void val_once(const int *cnt, int64_t n, uint32_t bit, uint32_t *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && cnt[i] != 1) atomicOr(flag, bit);
}

__global__ void val_leaf(const int *leaf_off, int nleaf, int64_t n, uint32_t *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaf) return;
    if (leaf_off[i] >= leaf_off[i + 1] || (i == 0 && leaf_off[0] != 0) || (i == nleaf - 1 && leaf_off[nleaf] != n))
        atomicOr(flag, kDbgLeaf);
}

__global__ void val_ulist(const uint32_t *keys, const int *u_off, const int *u_idx, int nleaf, int64_t n_u,
                          uint32_t *flag) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const int o0 = u_off[b], o1 = u_off[b + 1];
    if (o0 < 0 || o1 < o0 || o1 > n_u || o1 - o0 > 27) {
        atomicOr(flag, kDbgUList);
        return;
    }
    int bx, by, bz;
    demorton3(keys[b], bx, by, bz);
    bool self = false;
    for (int m = o0, prev = -1; m < o1; ++m) {
        const int a = u_idx[m];
        if (a < 0 || a >= nleaf || a <= prev) {
            atomicOr(flag, kDbgUList);
            return;
        }
        prev = a, self = self || a == b;
        int ax, ay, az;
        demorton3(keys[a], ax, ay, az);
        if (abs(ax - bx) > 1 || abs(ay - by) > 1 || abs(az - bz) > 1) atomicOr(flag, kDbgUList);
    }
    if (!self) atomicOr(flag, kDbgUList);
}

// level l: keys strictly increasing and inside the level, the dense table, the parent
__global__ void val_level(const uint32_t *keys, int n, int level, const int *dense, const int *parent,
                          const uint32_t *pkeys, int np, uint32_t *flag) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const uint32_t k = keys[b];
    if ((b > 0 && keys[b - 1] >= k) || k >= (1u << (3 * level)) || dense[k] != b) atomicOr(flag, kDbgKeys);
    if (level > 0) {
        const int pp = parent[b];
        if (pp < 0 || pp >= np || pkeys[pp] != (k >> 3)) atomicOr(flag, kDbgTree);
    }
}

// every slot of the dense table: -1 or the box of that key
__global__ void val_dense(const int *dense, int64_t slots, const uint32_t *keys, int n, uint32_t *flag) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= slots) return;
    const int d = dense[j];
    if (d != -1 && (d < 0 || d >= n || keys[d] != (uint32_t)j)) atomicOr(flag, kDbgKeys);
}

__global__ void val_child(const uint32_t *keys, int n, const int *child, const uint32_t *ckeys, const int *cparent,
                          int nc, uint32_t *flag) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * 8) return;
    const int b = (int)(e >> 3), c = (int)(e & 7), ch = child[e];
    if (ch == -1) return;
    if (ch < 0 || ch >= nc || cparent[ch] != b || ckeys[ch] != ((keys[b] << 3) | (uint32_t)c)) atomicOr(flag, kDbgTree);
}

struct ClassOff {
    int off[9];
};

// the class order of a level: rows [off[c], off[c + 1]) hold the boxes of octant c
__global__ void val_class(const int *cls_rows, int n, const uint32_t *keys, ClassOff co, uint32_t *flag) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int c = 0;
    while (c < 8 && r >= co.off[c + 1]) ++c;
    const int b = cls_rows[r];
    if (c == 8 || b < 0 || b >= n || (int)(keys[b] & 7u) != c) atomicOr(flag, kDbgClass);
}

unsigned vblocks(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace

cudaError_t validate_tree(const fmm_ctx *ctx, uint32_t *flags) {
    cudaStream_t s = ctx->stream;
    const int depth = ctx->opt.depth;
    const int64_t n = ctx->n;
    const int nleaf = ctx->nleaf;
    uint32_t hflags = 0;
    Scratch<uint32_t> flag;
    Scratch<int> cnt;
    FMM_CUDA_TRY(flag.alloc(1, s));
    FMM_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(uint32_t), s));
    FMM_CUDA_TRY(cnt.alloc(std::max<int64_t>(n, ctx->total_rows), s));
    auto permutation = [&](const int *v, int64_t m, uint32_t bit) -> cudaError_t {
        FMM_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, std::max<int64_t>(m, 1) * sizeof(int), s));
        val_count<<<vblocks(m), 256, 0, s>>>(v, m, m, cnt.p, bit, flag.p); count_launch();
        val_once<<<vblocks(m), 256, 0, s>>>(cnt.p, m, bit, flag.p); count_launch();
        return cudaGetLastError();
    };
    FMM_CUDA_TRY(permutation(ctx->perm, n, kDbgPerm));
    val_leaf<<<vblocks(nleaf), 256, 0, s>>>(ctx->leaf_off, nleaf, n, flag.p); count_launch();
    val_ulist<<<vblocks(nleaf), 256, 0, s>>>(ctx->lev[depth].keys, ctx->u_off, ctx->u_idx, nleaf, ctx->n_u, flag.p);
    count_launch();
    FMM_CUDA_TRY(permutation(ctx->p2p_order, nleaf, kDbgOrder));
    for (int l = 0; l <= depth; ++l) {
        const LevelTables &T = ctx->lev[l];
        const int nl = (int)T.n;
        if (!nl) continue;
        const LevelTables *P = l > 0 ? &ctx->lev[l - 1] : nullptr;
        val_level<<<vblocks(nl), 256, 0, s>>>(T.keys, nl, l, T.dense, T.parent, P ? P->keys : nullptr,
                                             P ? (int)P->n : 0, flag.p);
        count_launch();
        val_dense<<<vblocks((int64_t)1 << (3 * l)), 256, 0, s>>>(T.dense, (int64_t)1 << (3 * l), T.keys, nl, flag.p);
        count_launch();
        if (l < depth) {
            const LevelTables &C = ctx->lev[l + 1];
            val_child<<<vblocks((int64_t)nl * 8), 256, 0, s>>>(T.keys, nl, T.child, C.keys, C.parent, (int)C.n, flag.p);
            count_launch();
        }
        if (l >= 1 && T.cls_rows) {
            ClassOff co;
            for (int c = 0; c < 9; ++c) co.off[c] = T.cls_off[c];
            if (co.off[0] != 0 || co.off[8] != nl) hflags |= kDbgClass;
            val_class<<<vblocks(nl), 256, 0, s>>>(T.cls_rows, nl, T.keys, co, flag.p); count_launch();
            FMM_CUDA_TRY(permutation(T.cls_rows, nl, kDbgClass));
        }
    }
    FMM_CUDA_TRY(cudaGetLastError());
    uint32_t h = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&h, flag.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    *flags = h | hflags;
    return cudaSuccess;
}

FMM_DEBUG_UNIT(tree)

}  // namespace fmm

// ---------------------------------------------------------------------------------------
// Allocation-free point sort (fmm_sort_points_noalloc).  The paper has no counterpart: this is
// for callers that cannot let a library allocate device memory (their device memory is owned
// by one allocator or reserved in full at start-up).  Its scratch lives in one file-scope
// device array shared by every call, sized for kNoAllocMaxPoints points.
// ---------------------------------------------------------------------------------------
namespace fmm {
namespace {

constexpr int64_t kNoAllocMaxPoints = 1 << 20;
constexpr int64_t kNoAllocTiles = (kNoAllocMaxPoints + kSortTile - 1) / kSortTile;   // radix tiles
constexpr int64_t kNoAllocHist = 256 * kNoAllocTiles;                                // digit counts
constexpr int64_t kNoAllocSums = (kNoAllocHist + kScanBlock - 1) / kScanBlock;      // scan blocks
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxPoints * (sizeof(uint32_t) + sizeof(int)) +
                                 (size_t)(kNoAllocHist + kNoAllocSums + 1) * sizeof(int);

// keys copy | values copy | digit counts | scan block sums | non-finite flag.  Every pass
// overwrites the part it reads; only the flag is cleared at the start of every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
struct NoAllocAddr {
    void *ctx;               // the context the address was taken in
    unsigned char *addr;
};
NoAllocAddr g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// The calling thread's current context (driver handle), or null.
void *current_context() {
    using GetCurrent = int (*)(void **);
    static GetCurrent fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (GetCurrent)f;
    }();
    void *c = nullptr;
    if (!fn || fn(&c) != 0) return nullptr;
    return c;
}

// Device address of the scratch array on the current device.  It is looked up once per device
// and context: after a device reset the runtime makes a new primary context, in which the array
// has a new address, so a cached address is used only while the context it was taken in is
// still the current one.
cudaError_t noalloc_scratch(unsigned char **out) {
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocAddr &e = g_noalloc_addr[dev];
    void *cur = current_context();
    if (!e.addr || !cur || e.ctx != cur) {
        void *p = nullptr;
        FMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));   // makes the primary context current
        e.addr = (unsigned char *)p;
        e.ctx = current_context();
    }
    *out = e.addr;
    return cudaSuccess;
}

// Exclusive scan of n <= kScanBlock * kScanBlock ints with the given block-sum buffer.
cudaError_t scan_fixed(int *d, int64_t n, int *sums, cudaStream_t s) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        scan_blocks<int><<<1, kScanThreads, 0, s>>>(d, n, nullptr); count_launch();
        return cudaGetLastError();
    }
    scan_blocks<int><<<(unsigned)nb, kScanThreads, 0, s>>>(d, n, sums); count_launch();
    scan_blocks<int><<<1, kScanThreads, 0, s>>>(sums, nb, nullptr); count_launch();
    scan_add<int><<<(unsigned)nb, kScanThreads, 0, s>>>(d, n, sums); count_launch();
    return cudaGetLastError();
}

}  // namespace

}  // namespace fmm

extern "C" fmm_status fmm_sort_points_noalloc(const float *xyz, int64_t n, int depth, const double origin[3],
                                              double side, int32_t *perm, uint32_t *keys, void *cuda_stream) {
    using namespace fmm;
    if (!xyz || !perm || !keys || !origin) return FMM_EINVAL;
    if (n <= 0 || n > kNoAllocMaxPoints) return FMM_EINVAL;   // beyond the scratch array's size
    if (depth < 0 || depth > kMaxDepth) return FMM_EINVAL;
    if (!(side > 0) || !std::isfinite(side)) return FMM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(origin[a])) return FMM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    uint32_t *k2 = (uint32_t *)base;
    int *v2 = (int *)(base + (size_t)kNoAllocMaxPoints * sizeof(uint32_t));
    int *hist = v2 + kNoAllocMaxPoints;
    int *sums = hist + kNoAllocHist;
    int *bad = sums + kNoAllocSums;   // set by the key kernel on a non-finite coordinate
    const double scale = std::ldexp(1.0, depth) / side;
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    morton_kernel<float><<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, origin[0], origin[1], origin[2], scale, depth,
                                                           keys, perm, bad, (float)origin[0], (float)origin[1],
                                                           (float)origin[2], (float)scale);
    count_launch();
    // stable LSD radix sort of (keys, perm), 8-bit digits, ping-ponging with the scratch copies
    const int bits = 3 * depth;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    uint32_t *ka = keys, *kb = k2;
    int *va = perm, *vb = v2;
    for (int pass = 0; pass < (bits + 7) / 8 && n > 1; ++pass) {
        radix_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, 8 * pass, ntiles, hist); count_launch();
        if (scan_fixed(hist, (int64_t)256 * ntiles, sums, s) != cudaSuccess) return FMM_ECUDA;
        radix_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, n, 8 * pass, ntiles, hist, kb, vb); count_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        if (cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(perm, va, n * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return FMM_ECUDA;
        }
    }
    // the non-finite flag, read back as fmm_build_tree reads its counts (one wait on the stream)
    int h_bad = 0;
    if (cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return FMM_ECUDA;
    return h_bad ? FMM_EINVAL : FMM_OK;
}
