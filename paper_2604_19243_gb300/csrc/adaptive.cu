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
#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {

struct AdaptiveState {
    int capacity = 0;
    int64_t rows = 0;
    int *count = nullptr;                  // [rows] points per box
    int *state = nullptr;                  // [rows] 0 not kept, 1 leaf, 2 refined
    int *off[4] = {};                      // U, V, W, X offsets [rows + 1]
    int *idx[4] = {};                      // U, V, W, X members (rows)
    int64_t entries[4] = {};
    std::vector<int> host_state;           // copy of state, for the summary counts
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

__global__ void leaf_count_kernel(const int *leaf_off, int n, int *count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) count[i] = leaf_off[i + 1] - leaf_off[i];
}

__global__ void parent_count_kernel(const int *child, int n, const int *count_child, int *count) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int s = 0;
    for (int c = 0; c < 8; ++c) {
        const int ch = child[(size_t)b * 8 + c];
        if (ch >= 0) s += count_child[ch];
    }
    count[b] = s;
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

unsigned grid_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

fmm_status afail(fmm_ctx *ctx, fmm_status st, const std::string &m) {
    ctx->err = m;
    return st;
}

cudaError_t build(fmm_ctx *ctx, AdaptiveState *A) {
    cudaStream_t s = ctx->stream;
    const int D = ctx->opt.depth;
    const int64_t rows = A->rows;
    FMM_CUDA_TRY(cudaMalloc(&A->count, rows * sizeof(int)));
    FMM_CUDA_TRY(cudaMalloc(&A->state, rows * sizeof(int)));
    for (int k = 0; k < 4; ++k) FMM_CUDA_TRY(cudaMalloc(&A->off[k], (rows + 1) * sizeof(int)));
    Scratch<int> flag;
    FMM_CUDA_TRY(flag.alloc(1, s));
    FMM_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    // point counts, leaves up
    const LevelTables &LD = ctx->lev[D];
    leaf_count_kernel<<<grid_for(LD.n, 256), 256, 0, s>>>(ctx->leaf_off, (int)LD.n, A->count + LD.row_base);
    count_launch();
    for (int l = D - 1; l >= 0; --l) {
        const LevelTables &T = ctx->lev[l];
        parent_count_kernel<<<grid_for(T.n, 256), 256, 0, s>>>(T.child, (int)T.n, A->count + ctx->lev[l + 1].row_base,
                                                                A->count + T.row_base);
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
    Levels L{};
    for (int l = 0; l <= D; ++l) {
        L.keys[l] = ctx->lev[l].keys;
        L.child[l] = ctx->lev[l].child;
        L.dense[l] = ctx->lev[l].dense;
        L.base[l] = (int)ctx->lev[l].row_base;
    }
    L.base[D + 1] = (int)rows;
    L.depth = D;
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
        FMM_CUDA_TRY(cudaMalloc(&A->idx[k], std::max(tot[k], 1) * sizeof(int)));
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
    FMM_CUDA_TRY(cudaMalloc(&A->idx[3], std::max<int64_t>(A->entries[3], 1) * sizeof(int)));
    Scratch<int> cursor;
    FMM_CUDA_TRY(cursor.alloc(rows, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(cursor.p, A->off[3], rows * sizeof(int), cudaMemcpyDeviceToDevice, s));
    x_fill_kernel<<<grid_for(rows, 256), 256, 0, s>>>((int)rows, A->off[2], A->idx[2], cursor.p, A->idx[3]);
    count_launch();
    sort_segments_kernel<<<grid_for(rows, 256), 256, 0, s>>>((int)rows, A->off[3], A->idx[3]);
    count_launch();
    FMM_CUDA_TRY(cudaGetLastError());
    int hflag = 0;
    A->host_state.resize(rows);
    FMM_CUDA_TRY(cudaMemcpyAsync(A->host_state.data(), A->state, rows * sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    return hflag ? cudaErrorInvalidValue : cudaSuccess;
}

}  // namespace

void adaptive_free(fmm_ctx *ctx) {
    AdaptiveState *A = ctx->adaptive;
    if (!A) return;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(A->count);
    cudaFree(A->state);
    for (int k = 0; k < 4; ++k) {
        cudaFree(A->off[k]);
        cudaFree(A->idx[k]);
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

}  // namespace fmm
