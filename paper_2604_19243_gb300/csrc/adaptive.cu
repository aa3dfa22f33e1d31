// Adaptive refinement (Section 2.1) of the uniform octree that fmm_build_tree makes, and the
// interaction lists of the adaptive tree (U, V, W and X; Table 1 and Algorithm 1's adaptive
// branches), built on the device.
//
// The uniform tree of depth D holds every non-empty box of every level with its children and,
// through the leaf ranges, its point count.  The adaptive tree keeps the root and the children of
// every kept box of level < D that holds more than q points; a kept box that is not refined is a
// leaf.  Lists of the adaptive tree:
//   U(b), leaf b:        the kept leaves adjacent to b (sharing a vertex, edge or face), b itself
//                        included, at any level;
//   V(b), level >= 2:    kept boxes of b's level whose parents are adjacent to b's parent and
//                        that are not adjacent to b;
//   W(b), leaf b:        kept boxes below b's colleagues that are not adjacent to b while their
//                        parents are (the largest such boxes, as in the kiFMM of Ying, Biros and
//                        Zorin that Section 2.1 follows);
//   X(b):                the leaves whose W list holds b.
// Boxes are named by their row in the all-level tables (level-major, ascending Morton key within
// a level), and every list is sorted by row.  One thread builds the U, V and W lists of one box:
// the same-level positions through the dense tables, coarser leaves by walking up from an empty
// position, and finer boxes by a depth-first walk below each refined colleague.
//
// The evaluation over the adaptive tree (adaptive_far, FP32/FP64) runs the steps of Algorithm 1
// over the kept boxes only, through the SIMT GEMMs restricted to per-level box lists: S2U at every
// leaf at its own level and U2U at the refined boxes (levels D .. 2); at every kept box of level
// >= 2 the VLI (sources from a dense table of the kept boxes), the decompress with D2D from the
// parent, and XLI, which adds the X lists' sources to the downward check potentials (step 2b);
// then the closing and D2T at every leaf of level >= 2 at its own level, and WLI, which evaluates
// the upward equivalent densities of the W lists at the leaves' points (step 3a).  The ULI runs the
// packed FP32 near-field kernel of the uniform tree over the adaptive U lists (FP64: uli_kernel).
#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {

// The boxes of one level that the adaptive tree keeps, as index lists (the level's box indices)
// and the tiles of the SIMT GEMMs over them.
struct AdaptiveLevel {
    int *kept = nullptr;        // kept boxes, grouped by octant (class), ascending within a class
    int *refined = nullptr;     // refined boxes, ascending
    int *leaves = nullptr;      // leaves, ascending
    int n_kept = 0, n_refined = 0, n_leaves = 0;
    int *xlist = nullptr;       // boxes with a non-empty X list, ascending
    int n_x = 0;
    TileSet kept_tiles;         // class tiles over `kept` (with the stencil slot masks, levels >= 2)
    TileSet refined_tiles, leaf_tiles;
};

struct AdaptiveState {
    int capacity = 0;
    int64_t rows = 0;
    int *count = nullptr;                  // [rows] points per box
    int *state = nullptr;                  // [rows] 0 not kept, 1 leaf, 2 refined
    int *off[4] = {};                      // U, V, W, X offsets [rows + 1]
    int *idx[4] = {};                      // U, V, W, X members (rows)
    int64_t entries[4] = {};
    std::vector<int> host_state;           // copy of state, for the summary counts
    int *uli_order = nullptr;              // [rows] the leaves in decreasing ULI work, then the other rows
    int uli_leaves = 0;                    // leaves at the head of uli_order
    AdaptiveLevel lv[kMaxDepth + 1];       // per level: the far pass's box lists and tiles
    int *wlist = nullptr;                  // rows with a non-empty W list, ascending
    int n_w = 0;
    int *begin = nullptr;                  // [rows] first sorted point of each box
    int *dense_kept[kMaxDepth + 1] = {};   // levels >= 2: the level's dense table without unkept boxes
    // evaluation workspaces (allocated by the first evaluation)
    void *ue = nullptr;                    // [rows x nsp] upward equivalent densities
    void *y1 = nullptr;                    // [max level size x rclup] closing intermediate
    size_t ue_bytes = 0, y1_bytes = 0;
};

namespace {

constexpr int kStack = 80;   // depth-first walk: at most 8 + 7 (D - 1) <= 71 pending boxes for D <= 10

struct Levels {
    const uint32_t *keys[kMaxDepth + 1];
    const int *child[kMaxDepth + 1];
    const int *dense[kMaxDepth + 1];
    int base[kMaxDepth + 2];   // first row of each level; base[depth + 1] = rows
    int depth;
};

__device__ inline int row_level(const Levels &L, int r) {
    int l = 0;
    while (l < L.depth && r >= L.base[l + 1]) ++l;
    return l;
}

// Closed cubes of box e (level l + k, coordinates ex..ez) and box a (level l) intersect.
__device__ inline bool touches(int ex, int ey, int ez, int k, int ax, int ay, int az) {
    const int w = 1 << k, lx = ax << k, ly = ay << k, lz = az << k;
    return ex >= lx - 1 && ex <= lx + w && ey >= ly - 1 && ey <= ly + w && ez >= lz - 1 && ez <= lz + w;
}

// The smallest offset o in {-1, 0, 1} for which coordinate a + o (level l) lies in the coarser
// box coordinate c (level l - k); 2 if none does.
__device__ inline int first_offset(int a, int c, int k) {
    for (int o = -1; o <= 1; ++o) {
        const int v = a + o;
        if (v >= 0 && (v >> k) == c) return o;
    }
    return 2;
}

template <bool FILL>
struct Sink {
    int *out;
    int n = 0;
    __device__ void add(int v) {
        if (FILL) out[n] = v;
        ++n;
    }
};

__device__ inline void sort_segment(int *a, int n) {
    for (int i = 1; i < n; ++i) {
        const int v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

__global__ void leaf_count_kernel(const int *leaf_off, int n, int *count, int *begin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    count[i] = leaf_off[i + 1] - leaf_off[i];
    begin[i] = leaf_off[i];
}

__global__ void parent_count_kernel(const int *child, int n, const int *count_child, const int *begin_child,
                                    int *count, int *begin) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int s = 0, first = -1;
    for (int c = 0; c < 8; ++c) {
        const int ch = child[(size_t)b * 8 + c];
        if (ch >= 0) {
            s += count_child[ch];
            if (first < 0) first = begin_child[ch];
        }
    }
    count[b] = s;
    begin[b] = first;
}

// the dense table of a level without the boxes the adaptive tree does not keep
__global__ void mask_dense_kernel(const uint32_t *keys, int n, const int *state, int *dense) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && state[b] == 0) dense[keys[b]] = -1;
}

__global__ void state_kernel(int level, int depth, const int *parent, int n, const int *state_parent,
                             const int *count, int capacity, int *state) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const bool kept = level == 0 || state_parent[parent[b]] == 2;
    state[b] = !kept ? 0 : (level < depth && count[b] > capacity) ? 2 : 1;
}

// U, V and W lists of every row: sizes (FILL = false, into the offset arrays) or members.
template <bool FILL>
__global__ void lists_kernel(Levels L, int rows, const int *__restrict__ state, int *u_off, int *u_idx,
                             int *v_off, int *v_idx, int *w_off, int *w_idx, int *flag) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int st = state[r];
    Sink<FILL> U{FILL ? u_idx + u_off[r] : nullptr}, V{FILL ? v_idx + v_off[r] : nullptr},
        W{FILL ? w_idx + w_off[r] : nullptr};
    if (st != 0) {
        const int l = row_level(L, r), b = r - L.base[l], m = 1 << l;
        int ax, ay, az;
        demorton3(L.keys[l][b], ax, ay, az);
        if (l >= 2) {   // V: children of the parent's neighbours (and of the parent), not adjacent
            const int px = ax >> 1, py = ay >> 1, pz = az >> 1;
            for (int i = -1; i <= 1; ++i)
                for (int j = -1; j <= 1; ++j)
                    for (int k = -1; k <= 1; ++k)
                        for (int c = 0; c < 8; ++c) {
                            const int sx = 2 * (px + i) + ((c >> 2) & 1), sy = 2 * (py + j) + ((c >> 1) & 1),
                                      sz = 2 * (pz + k) + (c & 1);
                            if (max(abs(sx - ax), max(abs(sy - ay), abs(sz - az))) <= 1) continue;
                            const int e = dense_find(L.dense[l], l, sx, sy, sz);
                            if (e >= 0 && state[L.base[l] + e] != 0) V.add(L.base[l] + e);
                        }
        }
        if (st == 1) {
            for (int ox = -1; ox <= 1; ++ox)
                for (int oy = -1; oy <= 1; ++oy)
                    for (int oz = -1; oz <= 1; ++oz) {
                        const int sx = ax + ox, sy = ay + oy, sz = az + oz;
                        if (sx < 0 || sy < 0 || sz < 0 || sx >= m || sy >= m || sz >= m) continue;
                        const int e = dense_find(L.dense[l], l, sx, sy, sz);
                        const int se = e >= 0 ? state[L.base[l] + e] : 0;
                        if (se == 1) {          // a leaf of the same level (b itself for o = 0)
                            U.add(L.base[l] + e);
                            continue;
                        }
                        if (se == 2) {          // a refined colleague: finer U members and W
                            int2 stack[kStack];
                            int top = 0;
                            for (int c = 0; c < 8; ++c) {
                                const int ch = L.child[l][(size_t)e * 8 + c];
                                if (ch >= 0) stack[top++] = make_int2(l + 1, ch);
                            }
                            while (top > 0) {
                                const int2 t = stack[--top];
                                const int lv = t.x, ix = t.y, row = L.base[lv] + ix;
                                int ex, ey, ez;
                                demorton3(L.keys[lv][ix], ex, ey, ez);
                                if (!touches(ex, ey, ez, lv - l, ax, ay, az)) {
                                    W.add(row);
                                } else if (state[row] == 1) {
                                    U.add(row);
                                } else {
                                    if (top + 8 > kStack) {   // cannot happen for depth <= 10
                                        atomicExch(flag, 1);
                                        top = 0;
                                        break;
                                    }
                                    for (int c = 0; c < 8; ++c) {
                                        const int ch = L.child[lv][(size_t)ix * 8 + c];
                                        if (ch >= 0) stack[top++] = make_int2(lv + 1, ch);
                                    }
                                }
                            }
                            continue;
                        }
                        // empty at this level: the first kept box above the position, if a leaf,
                        // is a coarser adjacent leaf, counted from the first offset reaching it
                        for (int lc = l - 1; lc >= 0; --lc) {
                            const int k = l - lc, cx = sx >> k, cy = sy >> k, cz = sz >> k;
                            const int ce = dense_find(L.dense[lc], lc, cx, cy, cz);
                            const int cs = ce >= 0 ? state[L.base[lc] + ce] : 0;
                            if (cs == 0) continue;
                            if (cs == 1 && first_offset(ax, cx, k) == ox && first_offset(ay, cy, k) == oy &&
                                first_offset(az, cz, k) == oz)
                                U.add(L.base[lc] + ce);
                            break;
                        }
                    }
        }
    }
    if (!FILL) {
        u_off[r] = U.n, v_off[r] = V.n, w_off[r] = W.n;
    } else {
        sort_segment(U.out, U.n);
        sort_segment(V.out, V.n);
        sort_segment(W.out, W.n);
    }
}

// X lists: the transpose of the W lists
__global__ void x_count_kernel(int rows, const int *w_off, const int *w_idx, int *x_cnt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int i = w_off[r]; i < w_off[r + 1]; ++i) atomicAdd(&x_cnt[w_idx[i]], 1);
}

__global__ void x_fill_kernel(int rows, const int *w_off, const int *w_idx, int *cursor, int *x_idx) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int i = w_off[r]; i < w_off[r + 1]; ++i) x_idx[atomicAdd(&cursor[w_idx[i]], 1)] = r;
}

__global__ void sort_segments_kernel(int rows, const int *off, int *idx) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) sort_segment(idx + off[r], off[r + 1] - off[r]);
}

// ---------------------------------------------------------------------------------------
// Evaluation over the adaptive tree: the parts that the uniform pipeline does not have.
// ---------------------------------------------------------------------------------------
template <typename T> struct Pt4;
template <> struct Pt4<float> { using type = float4; };
template <> struct Pt4<double> { using type = double4; };
template <typename T> __device__ inline T inv_sqrt(T x);
template <> __device__ inline float inv_sqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ inline double inv_sqrt<double>(double x) { return 1.0 / sqrt(x); }
template <typename T> __host__ __device__ constexpr T one_over_4pi() { return (T)0.079577471545947667884441881686257181; }

constexpr int kEvalThreads = 128;
constexpr int kEvalChunk = 512;     // sources staged per round
constexpr int kMaxSurface = 488;    // 6 (p - 1)^2 + 2 for p <= 10

// centre of box `key` of a level whose boxes are `width` wide
__device__ inline void box_centre(uint32_t key, double ox, double oy, double oz, double width, double c[3]) {
    int ax, ay, az;
    demorton3(key, ax, ay, az);
    c[0] = ox + (ax + 0.5) * width, c[1] = oy + (ay + 0.5) * width, c[2] = oz + (az + 0.5) * width;
}

// XLI (Algorithm 1, step 2b): the sources of every leaf in X(b) on the downward check surface
// (1.05) of b, added to b's downward check potentials.  One block per box of the level with a
// non-empty X list (`list`, the level's box indices).
template <typename T>
__global__ void __launch_bounds__(kEvalThreads)
xli_kernel(const typename Pt4<T>::type *__restrict__ pts, const uint32_t *__restrict__ keys, int base,
           const int *__restrict__ x_off, const int *__restrict__ x_idx, const int *__restrict__ begin,
           const int *__restrict__ count, const T *__restrict__ grid, int ns, double ox, double oy, double oz,
           double width, double radius, T *__restrict__ D, int ld, const int *__restrict__ list) {
    using P = typename Pt4<T>::type;
    __shared__ P src[kEvalChunk];
    const int b = list[blockIdx.x], r = base + b;
    const int m0 = x_off[r], m1 = x_off[r + 1];
    if (m0 == m1) return;
    double c[3];
    box_centre(keys[b], ox, oy, oz, width, c);
    for (int i0 = 0; i0 < ns; i0 += kEvalThreads) {
        const int i = i0 + threadIdx.x;
        T px = 0, py = 0, pz = 0, acc = 0;
        if (i < ns) {
            px = (T)(c[0] + radius * (double)grid[3 * i]);
            py = (T)(c[1] + radius * (double)grid[3 * i + 1]);
            pz = (T)(c[2] + radius * (double)grid[3 * i + 2]);
        }
        for (int m = m0; m < m1; ++m) {
            const int a = x_idx[m], s0 = begin[a], s1 = s0 + count[a];
            for (int c0 = s0; c0 < s1; c0 += kEvalChunk) {
                const int c1 = min(s1, c0 + kEvalChunk);
                __syncthreads();
                for (int e = c0 + threadIdx.x; e < c1; e += kEvalThreads) src[e - c0] = pts[e];
                __syncthreads();
                if (i < ns)
                    for (int e = 0; e < c1 - c0; ++e) {
                        const P y = src[e];
                        const T dx = px - y.x, dy = py - y.y, dz = pz - y.z;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > (T)0) acc += y.w * inv_sqrt<T>(r2);
                    }
            }
        }
        if (i < ns) D[(size_t)b * ld + i] += acc * one_over_4pi<T>();
    }
}

// WLI (Algorithm 1, step 3a): the upward equivalent densities (1.05 surface) of every box in
// W(b) evaluated at the points of leaf b, added to the far-field outputs.  One block per row with
// a non-empty W list (`list`).
template <typename T, bool GRAD>
__global__ void __launch_bounds__(kEvalThreads)
wli_kernel(const typename Pt4<T>::type *__restrict__ pts, Levels L, const int *__restrict__ w_off,
           const int *__restrict__ w_idx, const int *__restrict__ begin, const int *__restrict__ count,
           const T *__restrict__ grid, int ns, double ox, double oy, double oz, double side,
           const T *__restrict__ ue, int ldu, T *__restrict__ phi, T *__restrict__ grad, const int *__restrict__ list) {
    using P = typename Pt4<T>::type;
    __shared__ P src[kMaxSurface];
    const int r = list[blockIdx.x];
    const int m0 = w_off[r], m1 = w_off[r + 1];
    if (m0 == m1) return;
    const int t0 = begin[r], t1 = t0 + count[r];
    for (int i0 = t0; i0 < t1; i0 += kEvalThreads) {
        const int i = i0 + threadIdx.x;
        const P x = pts[min(i, t1 - 1)];
        T pot = 0, gx = 0, gy = 0, gz = 0;
        for (int m = m0; m < m1; ++m) {
            const int a = w_idx[m], la = row_level(L, a);
            const double width = side / (double)(1 << la), radius = 1.05 * 0.5 * width;
            double c[3];
            box_centre(L.keys[la][a - L.base[la]], ox, oy, oz, width, c);
            __syncthreads();
            for (int j = threadIdx.x; j < ns; j += kEvalThreads) {
                P y;
                y.x = (T)(c[0] + radius * (double)grid[3 * j]);
                y.y = (T)(c[1] + radius * (double)grid[3 * j + 1]);
                y.z = (T)(c[2] + radius * (double)grid[3 * j + 2]);
                y.w = ue[(size_t)a * ldu + j];
                src[j] = y;
            }
            __syncthreads();
            for (int j = 0; j < ns; ++j) {
                const P y = src[j];
                const T dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                const T ri = inv_sqrt<T>(dx * dx + dy * dy + dz * dz), w = y.w * ri;
                pot += w;
                if (GRAD) {
                    const T w3 = w * ri * ri;
                    gx -= w3 * dx, gy -= w3 * dy, gz -= w3 * dz;
                }
            }
        }
        if (i < t1) {
            if (phi) phi[i] += pot * one_over_4pi<T>();
            if (GRAD) {
                grad[3 * (size_t)i] += gx * one_over_4pi<T>();
                grad[3 * (size_t)i + 1] += gy * one_over_4pi<T>();
                grad[3 * (size_t)i + 2] += gz * one_over_4pi<T>();
            }
        }
    }
}

// ULI over the adaptive U lists: every point of leaf b against the points of every leaf in
// U(b) (pairs at distance zero skipped).  One block per leaf, row order[blockIdx.x] (the FP64 form).
template <typename T, bool POT, bool GRAD>
__global__ void __launch_bounds__(kEvalThreads)
uli_kernel(const typename Pt4<T>::type *__restrict__ pts, const int *__restrict__ state,
           const int *__restrict__ u_off, const int *__restrict__ u_idx, const int *__restrict__ begin,
           const int *__restrict__ count, T *__restrict__ phi, T *__restrict__ grad, const int *__restrict__ order) {
    using P = typename Pt4<T>::type;
    __shared__ P src[kEvalChunk];
    const int r = order[blockIdx.x];
    if (state[r] != 1) return;
    const int t0 = begin[r], t1 = t0 + count[r];
    for (int i0 = t0; i0 < t1; i0 += kEvalThreads) {
        const int i = i0 + threadIdx.x;
        const P x = pts[min(i, t1 - 1)];
        T pot = 0, gx = 0, gy = 0, gz = 0;
        for (int m = u_off[r]; m < u_off[r + 1]; ++m) {
            const int a = u_idx[m], s0 = begin[a], s1 = s0 + count[a];
            for (int c0 = s0; c0 < s1; c0 += kEvalChunk) {
                const int c1 = min(s1, c0 + kEvalChunk);
                __syncthreads();
                for (int e = c0 + threadIdx.x; e < c1; e += kEvalThreads) src[e - c0] = pts[e];
                __syncthreads();
                for (int e = 0; e < c1 - c0; ++e) {
                    const P y = src[e];
                    const T dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 > (T)0) {
                        const T ri = inv_sqrt<T>(r2), w = y.w * ri;
                        if (POT) pot += w;
                        if (GRAD) {
                            const T w3 = w * ri * ri;
                            gx -= w3 * dx, gy -= w3 * dy, gz -= w3 * dz;
                        }
                    }
                }
            }
        }
        if (i < t1) {
            if (POT) phi[i] = pot * one_over_4pi<T>();
            if (GRAD) {
                grad[3 * (size_t)i] = gx * one_over_4pi<T>();
                grad[3 * (size_t)i + 1] = gy * one_over_4pi<T>();
                grad[3 * (size_t)i + 2] = gz * one_over_4pi<T>();
            }
        }
    }
}

// ULI schedule key of every row: a leaf gets the complement of the top 16 bits of its work
// |b| * sum_{a in U(b)} |a| as a float (monotone in the work, so an ascending stable sort puts
// the leaves first in decreasing work), every other row 0xffff, above any leaf's key
__global__ void uli_work_kernel(int rows, const int *state, const int *count, const int *u_off, const int *u_idx,
                                uint32_t *key, int *order) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    uint32_t k = 0xffffu;
    if (state[r] == 1) {
        long long src = 0;
        for (int m = u_off[r]; m < u_off[r + 1]; ++m) src += count[u_idx[m]];
        const long long w = src * (long long)count[r];
        k = 0xffffu - (__float_as_uint((float)(w > 1 ? w : 1)) >> 16);
    }
    key[r] = k;
    order[r] = r;
}

Levels make_levels(const fmm_ctx *ctx) {
    Levels L{};
    const int D = ctx->opt.depth;
    for (int l = 0; l <= D; ++l) {
        L.keys[l] = ctx->lev[l].keys;
        L.child[l] = ctx->lev[l].child;
        L.dense[l] = ctx->lev[l].dense;
        L.base[l] = (int)ctx->lev[l].row_base;
    }
    L.base[D + 1] = (int)ctx->total_rows;
    L.depth = D;
    return L;
}

unsigned grid_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

fmm_status afail(fmm_ctx *ctx, fmm_status st, const std::string &m) {
    ctx->err = m;
    return st;
}

constexpr int kAdaptTile = 64;   // rows per tile of the far pass's GEMMs (the SIMT form's)

template <typename V>
cudaError_t upload_vec(const std::vector<V> &h, V **d) {
    if (h.empty()) return cudaSuccess;
    FMM_CUDA_TRY(dev_malloc(d, h.size() * sizeof(V)));
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
}

// Per level, from the host copy of the states: the kept boxes in class order, the refined boxes
// and the leaves, with their tiles; the stencil slot masks of the kept tiles against the kept
// boxes' dense table.
cudaError_t build_levels(fmm_ctx *ctx, AdaptiveState *A) {
    cudaStream_t s = ctx->stream;
    const int D = ctx->opt.depth;
    std::vector<int> w_off(A->rows + 1), x_off(A->rows + 1), wl;
    FMM_CUDA_TRY(cudaMemcpy(w_off.data(), A->off[2], (A->rows + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    FMM_CUDA_TRY(cudaMemcpy(x_off.data(), A->off[3], (A->rows + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t r = 0; r < A->rows; ++r)
        if (w_off[r + 1] > w_off[r]) wl.push_back((int)r);
    A->n_w = (int)wl.size();
    FMM_CUDA_TRY(upload_vec(wl, &A->wlist));
    for (int l = 0; l <= D; ++l) {
        const LevelTables &T = ctx->lev[l];
        AdaptiveLevel &L = A->lv[l];
        const int n = (int)T.n;
        std::vector<uint32_t> keys(std::max(n, 1));
        if (n) FMM_CUDA_TRY(cudaMemcpy(keys.data(), T.keys, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        const int *st = A->host_state.data() + T.row_base;
        std::vector<int> kept, refined, leaves, xl;
        std::vector<Tile> kt, rt, lt;
        for (int b = 0; b < n; ++b)
            if (x_off[T.row_base + b + 1] > x_off[T.row_base + b]) xl.push_back(b);
        L.n_x = (int)xl.size();
        FMM_CUDA_TRY(upload_vec(xl, &L.xlist));
        for (int c = 0; c < 8; ++c) {
            const size_t c0 = kept.size();
            for (int b = 0; b < n; ++b)
                if (st[b] != 0 && (l == 0 ? c == 0 : (int)(keys[b] & 7u) == c)) kept.push_back(b);
            for (size_t r = c0; r < kept.size(); r += kAdaptTile)
                kt.push_back(Tile{(int)r, (int)std::min<size_t>(kAdaptTile, kept.size() - r), c, (int)kt.size()});
        }
        for (int b = 0; b < n; ++b) {
            if (st[b] == 2) refined.push_back(b);
            if (st[b] == 1) leaves.push_back(b);
        }
        auto plain = [](const std::vector<int> &v, std::vector<Tile> &t) {
            for (size_t r = 0; r < v.size(); r += kAdaptTile)
                t.push_back(Tile{(int)r, (int)std::min<size_t>(kAdaptTile, v.size() - r), -1, 0});
        };
        plain(refined, rt);
        plain(leaves, lt);
        L.n_kept = (int)kept.size(), L.n_refined = (int)refined.size(), L.n_leaves = (int)leaves.size();
        FMM_CUDA_TRY(upload_vec(kept, &L.kept));
        FMM_CUDA_TRY(upload_vec(refined, &L.refined));
        FMM_CUDA_TRY(upload_vec(leaves, &L.leaves));
        for (auto [ts, h] : {std::pair<TileSet *, std::vector<Tile> *>{&L.kept_tiles, &kt}, {&L.refined_tiles, &rt},
                             {&L.leaf_tiles, &lt}}) {
            ts->ntiles = (int)h->size();
            ts->tile_m = kAdaptTile;
            FMM_CUDA_TRY(upload_vec(*h, &ts->tiles));
        }
        if (l >= 2 && L.kept_tiles.ntiles) {
            FMM_CUDA_TRY(dev_malloc(&L.kept_tiles.masks, (size_t)L.kept_tiles.ntiles * 6 * sizeof(uint32_t)));
            FMM_CUDA_TRY(launch_tile_masks(L.kept_tiles.tiles, L.kept_tiles.ntiles, L.kept, T.keys, A->dense_kept[l], l,
                                           ctx->class_delta, L.kept_tiles.masks, s));
        }
    }
    return cudaStreamSynchronize(s);
}

cudaError_t build(fmm_ctx *ctx, AdaptiveState *A) {
    cudaStream_t s = ctx->stream;
    const int D = ctx->opt.depth;
    const int64_t rows = A->rows;
    FMM_CUDA_TRY(dev_malloc(&A->count, rows * sizeof(int)));
    FMM_CUDA_TRY(dev_malloc(&A->begin, rows * sizeof(int)));
    FMM_CUDA_TRY(dev_malloc(&A->state, rows * sizeof(int)));
    for (int k = 0; k < 4; ++k) FMM_CUDA_TRY(dev_malloc(&A->off[k], (rows + 1) * sizeof(int)));
    Scratch<int> flag;
    FMM_CUDA_TRY(flag.alloc(1, s));
    FMM_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    // point counts, leaves up
    const LevelTables &LD = ctx->lev[D];
    leaf_count_kernel<<<grid_for(LD.n, 256), 256, 0, s>>>(ctx->leaf_off, (int)LD.n, A->count + LD.row_base,
                                                          A->begin + LD.row_base);
    count_launch();
    for (int l = D - 1; l >= 0; --l) {
        const LevelTables &T = ctx->lev[l];
        const int64_t cb = ctx->lev[l + 1].row_base;
        parent_count_kernel<<<grid_for(T.n, 256), 256, 0, s>>>(T.child, (int)T.n, A->count + cb, A->begin + cb,
                                                                A->count + T.row_base, A->begin + T.row_base);
        count_launch();
    }
    // kept / leaf / refined, root down
    for (int l = 0; l <= D; ++l) {
        const LevelTables &T = ctx->lev[l];
        state_kernel<<<grid_for(T.n, 256), 256, 0, s>>>(l, D, T.parent, (int)T.n,
                                                         l > 0 ? A->state + ctx->lev[l - 1].row_base : nullptr,
                                                         A->count + T.row_base, A->capacity, A->state + T.row_base);
        count_launch();
    }
    FMM_CUDA_TRY(cudaGetLastError());
    const Levels L = make_levels(ctx);
    const unsigned g = grid_for(rows, 128);
    lists_kernel<false><<<g, 128, 0, s>>>(L, (int)rows, A->state, A->off[0], nullptr, A->off[1], nullptr, A->off[2],
                                          nullptr, flag.p);
    count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    for (int k = 0; k < 3; ++k) FMM_CUDA_TRY(exclusive_scan<int>(A->off[k], rows, A->off[k] + rows, s));
    int tot[3];
    for (int k = 0; k < 3; ++k)
        FMM_CUDA_TRY(cudaMemcpyAsync(&tot[k], A->off[k] + rows, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; ++k) {
        A->entries[k] = tot[k];
        FMM_CUDA_TRY(dev_malloc(&A->idx[k], std::max(tot[k], 1) * sizeof(int)));
    }
    lists_kernel<true><<<g, 128, 0, s>>>(L, (int)rows, A->state, A->off[0], A->idx[0], A->off[1], A->idx[1],
                                         A->off[2], A->idx[2], flag.p);
    count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    // X = transpose of W
    FMM_CUDA_TRY(cudaMemsetAsync(A->off[3], 0, (rows + 1) * sizeof(int), s));
    x_count_kernel<<<grid_for(rows, 256), 256, 0, s>>>((int)rows, A->off[2], A->idx[2], A->off[3]);
    count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    FMM_CUDA_TRY(exclusive_scan<int>(A->off[3], rows, A->off[3] + rows, s));
    A->entries[3] = A->entries[2];
    FMM_CUDA_TRY(dev_malloc(&A->idx[3], std::max<int64_t>(A->entries[3], 1) * sizeof(int)));
    Scratch<int> cursor;
    FMM_CUDA_TRY(cursor.alloc(rows, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(cursor.p, A->off[3], rows * sizeof(int), cudaMemcpyDeviceToDevice, s));
    x_fill_kernel<<<grid_for(rows, 256), 256, 0, s>>>((int)rows, A->off[2], A->idx[2], cursor.p, A->idx[3]);
    count_launch();
    sort_segments_kernel<<<grid_for(rows, 256), 256, 0, s>>>((int)rows, A->off[3], A->idx[3]);
    count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    // the stencil's source tables: unkept boxes removed
    for (int l = 2; l <= D; ++l) {
        const LevelTables &T = ctx->lev[l];
        const size_t sz = (size_t)1 << (3 * l);
        FMM_CUDA_TRY(dev_malloc(&A->dense_kept[l], sz * sizeof(int)));
        FMM_CUDA_TRY(cudaMemcpyAsync(A->dense_kept[l], T.dense, sz * sizeof(int), cudaMemcpyDeviceToDevice, s));
        mask_dense_kernel<<<grid_for(T.n, 256), 256, 0, s>>>(T.keys, (int)T.n, A->state + T.row_base, A->dense_kept[l]);
        count_launch();
    }
    FMM_CUDA_TRY(cudaGetLastError());
    // ULI schedule
    {
        Scratch<uint32_t> key;
        FMM_CUDA_TRY(key.alloc(rows, s));
        FMM_CUDA_TRY(dev_malloc(&A->uli_order, rows * sizeof(int)));
        uli_work_kernel<<<grid_for(rows, 256), 256, 0, s>>>((int)rows, A->state, A->count, A->off[0], A->idx[0], key.p,
                                                            A->uli_order);
        count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
        FMM_CUDA_TRY(stable_sort_by_key(key.p, A->uli_order, rows, 16, s));
    }
    int hflag = 0;
    A->host_state.resize(rows);
    FMM_CUDA_TRY(cudaMemcpyAsync(A->host_state.data(), A->state, rows * sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    A->uli_leaves = (int)std::count(A->host_state.begin(), A->host_state.end(), 1);
    if (hflag) return cudaErrorInvalidValue;
    return build_levels(ctx, A);
}

}  // namespace

void adaptive_free(fmm_ctx *ctx) {
    AdaptiveState *A = ctx->adaptive;
    if (!A) return;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(A->count);
    cudaFree(A->begin);
    cudaFree(A->state);
    for (int k = 0; k < 4; ++k) {
        cudaFree(A->off[k]);
        cudaFree(A->idx[k]);
    }
    for (int l = 0; l <= kMaxDepth; ++l) cudaFree(A->dense_kept[l]);
    cudaFree(A->ue);
    cudaFree(A->y1);
    cudaFree(A->uli_order);
    cudaFree(A->wlist);
    for (int l = 0; l <= kMaxDepth; ++l) {
        AdaptiveLevel &L = A->lv[l];
        cudaFree(L.kept), cudaFree(L.refined), cudaFree(L.leaves), cudaFree(L.xlist);
        for (TileSet *ts : {&L.kept_tiles, &L.refined_tiles, &L.leaf_tiles}) cudaFree(ts->tiles), cudaFree(ts->masks);
    }
    delete A;
    ctx->adaptive = nullptr;
}

fmm_status adaptive_setup(fmm_ctx *ctx, int capacity) {
    if (!ctx->have_tree) return afail(ctx, FMM_ESTATE, "fmm_build_tree has not been called");
    if (capacity < 0) return afail(ctx, FMM_EINVAL, "capacity must be >= 0");
    if (ctx->total_rows >= (int64_t)1 << 30) return afail(ctx, FMM_EINVAL, "too many boxes for the adaptive lists");
    adaptive_free(ctx);
    AdaptiveState *A = new AdaptiveState;
    ctx->adaptive = A;
    A->capacity = capacity;
    A->rows = ctx->total_rows;
    cudaError_t e = build(ctx, A);
    if (e != cudaSuccess) {
        const bool walk = e == cudaErrorInvalidValue;
        cudaGetLastError();
        adaptive_free(ctx);
        return walk ? afail(ctx, FMM_EINVAL, "adaptive lists: depth-first walk exceeded its stack")
                    : afail(ctx, FMM_ECUDA, std::string("adaptive tree: ") + cudaGetErrorName(e));
    }
    return FMM_OK;
}

fmm_status adaptive_export(fmm_ctx *ctx, int kind, int64_t *offsets, int64_t *idx, int64_t *count) {
    AdaptiveState *A = ctx->adaptive;
    if (!A) return afail(ctx, FMM_ESTATE, "fmm_adaptive_setup has not been called");
    if (kind < FMM_ADAPTIVE_STATE || kind > FMM_ADAPTIVE_X) return afail(ctx, FMM_EINVAL, "unknown export kind");
    const int64_t rows = A->rows;
    const bool list = kind >= FMM_ADAPTIVE_U;
    const int k = kind - FMM_ADAPTIVE_U;
    const int64_t entries = list ? A->entries[k] : rows;
    if (count) count[0] = rows, count[1] = entries;
    cudaStream_t s = ctx->stream;
    auto copy = [&](const int *src, int64_t n, int64_t *dst) -> cudaError_t {
        std::vector<int> h((size_t)std::max<int64_t>(n, 1));
        cudaError_t e = cudaMemcpyAsync(h.data(), src, n * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) std::copy(h.begin(), h.begin() + n, dst);
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (idx) {
        const int *src = kind == FMM_ADAPTIVE_STATE ? A->state : kind == FMM_ADAPTIVE_COUNT ? A->count : A->idx[k];
        e = copy(src, entries, idx);
    }
    if (e == cudaSuccess && offsets && list) e = copy(A->off[k], rows + 1, offsets);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return afail(ctx, FMM_ECUDA, std::string("adaptive export: ") + cudaGetErrorName(e));
    }
    return FMM_OK;
}

fmm_status adaptive_info(fmm_ctx *ctx, int32_t *capacity, int64_t *leaves, int64_t *refined, int64_t *entries) {
    AdaptiveState *A = ctx->adaptive;
    if (!A) return afail(ctx, FMM_ESTATE, "fmm_adaptive_setup has not been called");
    if (capacity) *capacity = A->capacity;
    const int D = ctx->opt.depth;
    for (int l = 0; l <= kMaxDepth; ++l) {
        int64_t nl = 0, nr = 0;
        if (l <= D) {
            const LevelTables &T = ctx->lev[l];
            for (int64_t b = 0; b < T.n; ++b) {
                const int st = A->host_state[T.row_base + b];
                nl += st == 1, nr += st == 2;
            }
        }
        if (leaves) leaves[l] = nl;
        if (refined) refined[l] = nr;
    }
    if (entries)
        for (int k = 0; k < 4; ++k) entries[k] = A->entries[k];
    return FMM_OK;
}

// ---- evaluation hooks (called by run_far and run_evaluate while an adaptive evaluation runs) ----

template <typename T>
cudaError_t adaptive_xli(const fmm_ctx *ctx, int level, T *D, int ld, cudaStream_t s) {
    const AdaptiveState *A = ctx->adaptive;
    const LevelTables &T_ = ctx->lev[level];
    const AdaptiveLevel &L = A->lv[level];
    if (L.n_x == 0) return cudaSuccess;
    const double width = ctx->side / (double)(1 << level);
    xli_kernel<T><<<(unsigned)L.n_x, kEvalThreads, 0, s>>>(
        (const typename Pt4<T>::type *)ctx->pts, T_.keys, (int)T_.row_base, A->off[3], A->idx[3], A->begin, A->count,
        (const T *)ctx->grid_dev, ctx->npts, ctx->origin[0], ctx->origin[1], ctx->origin[2], width, 1.05 * 0.5 * width,
        D, ld, L.xlist);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t adaptive_wli(fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s) {
    AdaptiveState *A = ctx->adaptive;
    const int D = ctx->opt.depth;
    if (A->n_w == 0 || D < 2) return cudaSuccess;
    if (ctx->npts > kMaxSurface) return cudaErrorInvalidValue;   // p <= 10 is checked at fmm_create
    const int nsp = ctx->nsp;
    // upward equivalent densities of the kept boxes of levels 2..D: r_l (V S^-1)(U^T U_l)
    for (int l = 2; l <= D; ++l) {
        const AdaptiveLevel &L = A->lv[l];
        if (!L.n_kept) continue;
        const OpSet &o = ctx->fwd[l];
        GemmCall c1;
        c1.mode = GM_IDENTITY, c1.level = l, c1.n_out = o.rclup;
        c1.X0 = (T *)ctx->Uc + (size_t)ctx->lev[l].row_base * nsp, c1.ldx0 = nsp, c1.k0 = nsp, c1.W0 = o.uclose1;
        c1.Y = A->y1, c1.ldy = o.rclup;
        c1.tiles = &L.kept_tiles, c1.rows = L.kept;
        FMM_CUDA_TRY(gemm_simt<T>(ctx, c1, s));
        GemmCall c2;
        c2.mode = GM_IDENTITY, c2.level = l, c2.n_out = nsp, c2.alpha = ctx->side / (double)(1 << l) * 0.5;
        c2.X0 = A->y1, c2.ldx0 = o.rclup, c2.k0 = o.rclup, c2.W0 = o.uclose2;
        c2.Y = (T *)A->ue + (size_t)ctx->lev[l].row_base * nsp, c2.ldy = nsp;
        c2.tiles = &L.kept_tiles, c2.rows = L.kept;
        FMM_CUDA_TRY(gemm_simt<T>(ctx, c2, s));
    }
    const Levels L = make_levels(ctx);
    auto go = [&](auto kern, T *g) {
        kern<<<(unsigned)A->n_w, kEvalThreads, 0, s>>>((const typename Pt4<T>::type *)ctx->pts, L, A->off[2], A->idx[2],
                                                       A->begin, A->count, (const T *)ctx->grid_dev, ctx->npts,
                                                       ctx->origin[0], ctx->origin[1], ctx->origin[2], ctx->side,
                                                       (const T *)A->ue, nsp, phi, g, A->wlist);
    };
    grad ? go(wli_kernel<T, true>, grad) : go(wli_kernel<T, false>, nullptr);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t adaptive_uli(const fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s) {
    const AdaptiveState *A = ctx->adaptive;
    if constexpr (sizeof(T) == 4) {   // the packed FP32 kernels of the uniform tree, over the leaves' rows
        return launch_p2p_rows_f32((const float4 *)ctx->pts, ctx->n, A->begin, A->count, A->off[0], A->idx[0],
                                   A->uli_order, A->uli_leaves, (float *)phi, (float *)grad, s);
    } else {   // FP64: one block per leaf, in the ULI schedule's order
        if (A->uli_leaves == 0) return cudaSuccess;
        auto go = [&](auto kern) {
            kern<<<(unsigned)A->uli_leaves, kEvalThreads, 0, s>>>((const typename Pt4<T>::type *)ctx->pts, A->state,
                                                                 A->off[0], A->idx[0], A->begin, A->count, phi, grad,
                                                                 A->uli_order);
        };
        if (phi && grad) go(uli_kernel<T, true, true>);
        else if (grad) go(uli_kernel<T, false, true>);
        else go(uli_kernel<T, true, false>);
        count_launch();
        return cudaGetLastError();
    }
}

// workspaces of the W-list step for the current operators
fmm_status adaptive_prepare(fmm_ctx *ctx) {
    AdaptiveState *A = ctx->adaptive;
    const size_t es = ctx->fp64 ? sizeof(double) : sizeof(float);
    const int D = ctx->opt.depth;
    int64_t maxn = 1;
    int rclup = 16;
    for (int l = 2; l <= D; ++l) {
        maxn = std::max<int64_t>(maxn, ctx->lev[l].n);
        rclup = std::max(rclup, ctx->fwd[l].rclup);
        if (!ctx->fwd[l].uclose1) return afail(ctx, FMM_ESTATE, "the upward closing operators are missing");
    }
    const size_t ue_bytes = (size_t)A->rows * ctx->nsp * es, y1_bytes = (size_t)maxn * rclup * es;
    auto grow = [&](void **p, size_t *have, size_t need) {
        if (*have >= need) return true;
        cudaFree(*p);
        *p = nullptr, *have = 0;
        if (dev_malloc(p, need) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        *have = need;
        return true;
    };
    if (!grow(&A->ue, &A->ue_bytes, ue_bytes) || !grow(&A->y1, &A->y1_bytes, y1_bytes))
        return afail(ctx, FMM_ENOMEM, "adaptive workspace");
    return FMM_OK;
}

// The far field over the adaptive tree (forward, FP32/FP64): far_phi / far_grad (sorted order)
// receive D2T and WLI of every point.
template <typename T>
cudaError_t adaptive_far(fmm_ctx *ctx, T *far_phi, T *far_grad, cudaStream_t s) {
    const AdaptiveState *A = ctx->adaptive;
    const int D = ctx->opt.depth, nsp = ctx->nsp, kw = ctx->ws_kw;
    const T *grid = (const T *)ctx->grid_dev;
    auto at = [&](void *base, int l, int ld) { return (T *)base + (size_t)ctx->lev[l].row_base * ld; };
    auto restrict_to = [](GemmCall &c, const TileSet &ts, const int *rows) { c.tiles = &ts, c.rows = rows; };
    // upward pass (step 1), levels D .. 2: S2U at the leaves of the level, U2U at its refined boxes
    for (int l = D; l >= 2; --l) {
        const AdaptiveLevel &L = A->lv[l];
        const int64_t rb = ctx->lev[l].row_base;
        FMM_CUDA_TRY(launch_leaf_check_rows<T>(ctx, l, L.leaves, L.n_leaves, A->begin + rb, A->count + rb, grid,
                                               at(ctx->Uc, l, nsp), s));
        if (l == D) cudaEventRecord(ctx->ev[2], s);
        if (l < D && L.n_refined) {
            GemmCall c;
            c.mode = GM_CHILDREN, c.level = l, c.n_out = nsp;
            c.X0 = at(ctx->Uc, l + 1, nsp), c.ldx0 = nsp, c.k0 = nsp;
            c.W0 = ctx->fwd[l].up[0], c.w_stride = (int64_t)nsp * nsp;
            c.Y = at(ctx->Uc, l, nsp), c.ldy = nsp;
            restrict_to(c, L.refined_tiles, L.refined);
            FMM_CUDA_TRY(gemm_simt<T>(ctx, c, s));
        }
    }
    cudaEventRecord(ctx->ev[3], s);
    // downward pass (step 2), levels 2 .. D at the kept boxes: the VLI compress and stencil of
    // every level on the level's own stream (over the kept sources), then, level after level,
    // the decompress with D2D from the parent and XLI
    FMM_CUDA_TRY(cudaEventRecord(ctx->fork_ev[0], s));
    for (int l = 2; l <= D; ++l) {
        const AdaptiveLevel &L = A->lv[l];
        cudaStream_t ls = ctx->aux[l];
        FMM_CUDA_TRY(cudaStreamWaitEvent(ls, ctx->fork_ev[0], 0));
        if (L.n_kept) {
            const OpSet &o = ctx->fwd[l];
            GemmCall c;
            c.mode = GM_IDENTITY, c.level = l, c.n_out = o.kinp;
            c.X0 = at(ctx->Uc, l, nsp), c.ldx0 = nsp, c.k0 = nsp, c.W0 = o.compress;
            c.Y = at(ctx->Ut, l, kw), c.ldy = kw;
            restrict_to(c, L.kept_tiles, L.kept);
            FMM_CUDA_TRY(gemm_simt<T>(ctx, c, ls));
            GemmCall st;
            st.mode = GM_STENCIL, st.level = l, st.n_out = o.koutp;
            st.X0 = at(ctx->Ut, l, kw), st.ldx0 = kw, st.k0 = o.kinp;
            st.W0 = o.stencil, st.w_stride = (int64_t)o.koutp * o.kinp;
            st.Y = at(ctx->Ct, l, kw), st.ldy = kw;
            st.dense = A->dense_kept[l];
            restrict_to(st, L.kept_tiles, L.kept);
            FMM_CUDA_TRY(gemm_simt<T>(ctx, st, ls));
        }
        FMM_CUDA_TRY(cudaEventRecord(ctx->join_ev[l], ls));
    }
    for (int l = 2; l <= D; ++l) {
        const AdaptiveLevel &L = A->lv[l];
        FMM_CUDA_TRY(cudaStreamWaitEvent(s, ctx->join_ev[l], 0));
        if (!L.n_kept) continue;
        const OpSet &o = ctx->fwd[l];
        GemmCall dn;
        dn.mode = GM_PARENT2, dn.level = l, dn.n_out = nsp;
        dn.X0 = at(ctx->Ct, l, kw), dn.ldx0 = kw, dn.k0 = o.koutp, dn.W0 = o.decompress;
        if (l >= 3) {
            dn.X1 = at(ctx->Dc, l - 1, nsp), dn.ldx1 = nsp, dn.k1 = nsp;
            dn.W1_by_cls = ctx->fwd[l - 1].down;
        }
        dn.Y = at(ctx->Dc, l, nsp), dn.ldy = nsp;
        restrict_to(dn, L.kept_tiles, L.kept);
        FMM_CUDA_TRY(gemm_simt<T>(ctx, dn, s));
        FMM_CUDA_TRY(adaptive_xli<T>(ctx, l, at(ctx->Dc, l, nsp), nsp, s));
    }
    cudaEventRecord(ctx->ev[4], s);
    // leaf evaluation (step 3): closing and D2T at every leaf of level >= 2 (leaves of levels 0
    // and 1 have no far field), then WLI
    if (far_phi) FMM_CUDA_TRY(cudaMemsetAsync(far_phi, 0, (size_t)ctx->n * sizeof(T), s));
    if (far_grad) FMM_CUDA_TRY(cudaMemsetAsync(far_grad, 0, (size_t)ctx->n * 3 * sizeof(T), s));
    for (int l = 2; l <= D; ++l) {
        const AdaptiveLevel &L = A->lv[l];
        if (!L.n_leaves) continue;
        const OpSet &o = ctx->fwd[l];
        const int64_t rb = ctx->lev[l].row_base;
        GemmCall c1;
        c1.mode = GM_IDENTITY, c1.level = l, c1.n_out = o.rclp;
        c1.X0 = at(ctx->Dc, l, nsp), c1.ldx0 = nsp, c1.k0 = nsp, c1.W0 = o.close1;
        c1.Y = ctx->Yc, c1.ldy = o.rclp;
        restrict_to(c1, L.leaf_tiles, L.leaves);
        FMM_CUDA_TRY(gemm_simt<T>(ctx, c1, s));
        GemmCall c2;
        c2.mode = GM_IDENTITY, c2.level = l, c2.n_out = nsp, c2.alpha = ctx->side / (double)(1 << l) * 0.5;
        c2.X0 = ctx->Yc, c2.ldx0 = o.rclp, c2.k0 = o.rclp, c2.W0 = o.close2;
        c2.Y = ctx->Dq, c2.ldy = nsp;
        restrict_to(c2, L.leaf_tiles, L.leaves);
        FMM_CUDA_TRY(gemm_simt<T>(ctx, c2, s));
        FMM_CUDA_TRY(launch_leaf_eval_rows<T>(ctx, l, L.leaves, L.n_leaves, A->begin + rb, A->count + rb, grid,
                                              (const T *)ctx->Dq, nsp, far_phi, far_grad, s));
    }
    return adaptive_wli<T>(ctx, far_phi, far_grad, s);
}

#define FMM_ADAPTIVE_INST(T)                                                                          \
    template cudaError_t adaptive_far<T>(fmm_ctx *, T *, T *, cudaStream_t);                          \
    template cudaError_t adaptive_xli<T>(const fmm_ctx *, int, T *, int, cudaStream_t);               \
    template cudaError_t adaptive_wli<T>(fmm_ctx *, T *, T *, cudaStream_t);                          \
    template cudaError_t adaptive_uli<T>(const fmm_ctx *, T *, T *, cudaStream_t);
FMM_ADAPTIVE_INST(float)
FMM_ADAPTIVE_INST(double)
#undef FMM_ADAPTIVE_INST

}  // namespace fmm
