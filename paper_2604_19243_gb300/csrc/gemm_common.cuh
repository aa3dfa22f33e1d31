// Row gathering shared by the SIMT and tensor-core GEMM kernels.
//
// Every surface contraction of the FMM has the form
//     Y[b] (+)= alpha * sum_seg W_seg X_seg[src(b, seg)]
// over the boxes b of one level, with the source row chosen by one of four rules:
//   GM_IDENTITY  one segment, src = b                       (M2L compress/decompress, closing)
//   GM_CHILDREN  8 segments (child octant c), src = child_c(b), W_c   (U2U, and D2D^T)
//   GM_PARENT2   segment 0: src = b in X0 with W0; segment 1: src = parent(b) in X1 with the
//                operator of b's octant (M2L decompress fused with D2D, and U2U^T)
//   GM_STENCIL   189 segments (class slots), src = the box at b + t, W = C_t (VLI core)
// Missing source boxes (empty children, empty or out-of-domain V-list boxes) contribute zero.
#pragma once

#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {

struct GemmDev {
    int mode, accumulate, n_out, level;
    float alpha;
    double alpha_d;
    const void *X0; int ldx0; int k0;
    const void *W0; long long w_stride;
    const void *X1; int ldx1; int k1;
    const void *W1[8];
    void *Y; int ldy;
    const Tile *tiles;
    const uint32_t *masks;
    const int *rows;             // class-ordered row list (nullptr: plain order)
    const int *child;            // [n x 8] (GM_CHILDREN)
    const int *parent;           // (GM_PARENT2)
    const uint32_t *keys;        // level keys (GM_STENCIL)
    const int *dense;            // dense table of the level (GM_STENCIL)
    const int *class_slots;      // [8][189]
    const int *class_delta;      // [8][189]
};

// number of segments of a tile for the mode
__device__ inline int gemm_nseg(const GemmDev &g) {
    switch (g.mode) {
        case GM_CHILDREN: return 8;
        case GM_PARENT2: return g.X1 ? 2 : 1;
        case GM_STENCIL: return kClassSlots;
        default: return 1;
    }
}

__device__ inline bool gemm_seg_active(const GemmDev &g, const Tile &t, int seg) {
    if (g.mode != GM_STENCIL) return true;
    return (g.masks[(size_t)t.mask * 6 + (seg >> 5)] >> (seg & 31)) & 1u;
}

__device__ inline int gemm_seg_k(const GemmDev &g, int seg) {
    return (g.mode == GM_PARENT2 && seg == 1) ? g.k1 : g.k0;
}

// box index of tile row r
__device__ inline int gemm_row_box(const GemmDev &g, const Tile &t, int r) {
    return g.rows ? g.rows[t.row0 + r] : t.row0 + r;
}

// source row for (box, seg); -1 = zero row
__device__ inline int gemm_src_row(const GemmDev &g, const Tile &t, int box, int seg) {
    switch (g.mode) {
        case GM_CHILDREN: return g.child[(size_t)box * 8 + seg];
        case GM_PARENT2: return seg == 0 ? box : g.parent[box];
        case GM_STENCIL: {
            int ax, ay, az, dx, dy, dz;
            demorton3(g.keys[box], ax, ay, az);
            unpack_delta(g.class_delta[t.cls * kClassSlots + seg], dx, dy, dz);
            return dense_find(g.dense, g.level, ax + dx, ay + dy, az + dz);
        }
        default: return box;
    }
}

// operator index of (tile, seg): the W matrix is W0 + index * w_stride, except PARENT2 seg 1
__device__ inline long long gemm_w_index(const GemmDev &g, const Tile &t, int seg) {
    switch (g.mode) {
        case GM_CHILDREN: return seg;
        case GM_STENCIL: return g.class_slots[t.cls * kClassSlots + seg];
        default: return 0;
    }
}

}  // namespace fmm
