// Small device utilities shared by the CUDA sources of libfmm: error checks, a stream-ordered
// scratch allocation helper, Morton bit interleaving and an exclusive scan.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#define FMM_CUDA_TRY(expr)                      \
    do {                                        \
        cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return _e;       \
    } while (0)

namespace fmm {

// Stream-ordered allocation from a per-device memory pool that keeps freed memory cached
// (release threshold at its maximum): repeated tree builds and evaluations then reuse device
// memory instead of mapping it again after every synchronisation.  Freed with cudaFreeAsync.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
// Return the cached, unused memory of the current device's pool to the driver.
void pool_trim();

// Stream-ordered temporary buffer (pool_alloc / cudaFreeAsync).
template <typename T>
struct Scratch {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t alloc(size_t n, cudaStream_t st) {
        s = st;
        if (n == 0) n = 1;
        return pool_alloc((void **)&p, n * sizeof(T), st);
    }
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

// Spread the low 10 bits of v to every third bit (bit i -> bit 3i).
__host__ __device__ inline uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Inverse of spread3: gather every third bit back into the low 10 bits.
__host__ __device__ inline uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x3ffu;
    return v;
}

// Morton key of box coordinates (x bit most significant in every triple).
__host__ __device__ inline uint32_t morton3(uint32_t ax, uint32_t ay, uint32_t az) {
    return (spread3(ax) << 2) | (spread3(ay) << 1) | spread3(az);
}

__host__ __device__ inline void demorton3(uint32_t k, int &ax, int &ay, int &az) {
    ax = (int)compact3(k >> 2);
    ay = (int)compact3(k >> 1);
    az = (int)compact3(k);
}

// Transfer vector components in [-3, 3] packed into one int (4 bits each, offset by 3).
__host__ __device__ inline int pack_delta(int dx, int dy, int dz) {
    return (dx + 3) | ((dy + 3) << 4) | ((dz + 3) << 8);
}
__host__ __device__ inline void unpack_delta(int p, int &dx, int &dy, int &dz) {
    dx = (p & 15) - 3;
    dy = ((p >> 4) & 15) - 3;
    dz = ((p >> 8) & 15) - 3;
}

// Non-empty box at integer coordinates (ax, ay, az) of `level` through its dense table, or -1.
__device__ inline int dense_find(const int *dense, int level, int ax, int ay, int az) {
    const int m = 1 << level;
    if (ax < 0 || ay < 0 || az < 0 || ax >= m || ay >= m || az >= m) return -1;
    return dense[morton3((uint32_t)ax, (uint32_t)ay, (uint32_t)az)];
}

// Exclusive scan in place of n values; the total is written to *d_total (device) if non-null.
template <typename T>
cudaError_t exclusive_scan(T *d, int64_t n, T *d_total, cudaStream_t s);

// Stable LSD radix sort of (keys, vals) by the low `bits` bits of the keys, results in place
// (scratch from the stream-ordered pool).
cudaError_t stable_sort_by_key(uint32_t *keys, int *vals, int64_t n, int bits, cudaStream_t s);

// Stencil slot masks of class-ordered tiles (Tile.row0 + r indexes `rows`, the level's box indices;
// Tile.mask is the tile's index): bit s of masks[tile * 6 + s / 32] is set when a row of the tile
// has a source box in `dense` for class slot s.
struct Tile;
cudaError_t launch_tile_masks(const Tile *tiles, int ntiles, const int *rows, const uint32_t *keys, const int *dense,
                              int level, const int *class_delta, uint32_t *masks, cudaStream_t s);

}  // namespace fmm
