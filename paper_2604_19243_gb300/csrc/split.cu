// Partitioned evaluation: the distributed scheme of Section 3 (Box comm-setup and Box
// comm-runtime) with P virtual ranks on one GPU, each holding buffers of its own.
//
// Setup:
//  (1) Tree: the context's tree is split at depth d_global.  Its level-d_global boxes are the
//      local roots, each the root of a local tree down to the leaves.
//  (2) Layout: the local roots go to the ranks in Morton order, in contiguous runs balanced by
//      their point counts (every rank owns at least one root).
//  (3, 4) Queries: for every box a rank owns below d_global, the V-list boxes (levels >
//      d_global) and, for its leaves, the U-list leaves that lie in another rank's subdomain
//      (found through the layout) form the rank's query packets, keyed by Morton key and owner.
//  (5) Neighbourhoods: the owners addressed by a rank's U and by its V packets.
//  (6) Existence: each owner answers with the queried boxes it holds (the non-empty ones).  The
//      answers give every rank its local essential tree (Eq. 3: its own boxes and the ghosts of
//      their U and V lists), the receive rows of its V ghosts and the coordinates of its U-list
//      ghost points.
// Runtime:
//  local stage: densities of the U ghost points; S2U and U2U up to the local roots; VLI compress
//    of the levels below d_global; then the V ghosts' compressed rows (V exchange);
//  global stage: the local roots' u rows gathered into a nominated context, U2U, VLI and D2D over
//    levels 2..d_global there, the local roots' d rows scattered back;
//  local downward stage: VLI stencil, decompress + D2D, leaf closing and D2T of the levels below
//    d_global, and the ULI of the own leaves with the ghost points.
// Every output is computed by the same kernels from the same values in the same order as on the
// unpartitioned tree, so the results are equal bit for bit.  Each exchange is one device copy
// kernel over all ranks (a row gather between the ranks' buffers).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <iterator>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {

namespace {

struct RowCopy {   // one row of one array: context src_ctx, row src_row -> dst_ctx, dst_row
    int src_ctx, src_row, dst_ctx, dst_row;
};
struct PtsCopy {   // the points of one ghost leaf
    int src_ctx, src_pos, dst_ctx, dst_pos, count;
};

// One array as every context holds it: ranks 0..P-1, then the global context (index P).
struct RowArray {
    unsigned char **base = nullptr;   // device [P + 1]
    long long ld = 0;                 // bytes per row
    int row_bytes = 0;
    bool aligned16 = false;           // every base pointer 16-byte aligned (checked on the host)
};

// One warp per row.
template <typename W>
__global__ void copy_rows_kernel(const RowCopy *__restrict__ e, int n, unsigned char *const *__restrict__ base,
                                 long long ld, int words) {
    const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (w >= n) return;
    const RowCopy c = e[w];
    const W *src = reinterpret_cast<const W *>(base[c.src_ctx] + (long long)c.src_row * ld);
    W *dst = reinterpret_cast<W *>(base[c.dst_ctx] + (long long)c.dst_row * ld);
    for (int i = lane; i < words; i += 32) dst[i] = src[i];
}

// Dense key -> row table of one level of a rank's local essential tree (set to -1 before).
__global__ void let_dense_kernel(const uint32_t *__restrict__ keys, int n, int *__restrict__ dense) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dense[keys[i]] = i;
}

// One block per ghost leaf: whole points (setup) or densities only (every evaluation).
template <typename P4>
__global__ void copy_pts_kernel(const PtsCopy *__restrict__ e, P4 *const *__restrict__ base, int whole) {
    const PtsCopy c = e[blockIdx.x];
    const P4 *src = base[c.src_ctx] + c.src_pos;
    P4 *dst = base[c.dst_ctx] + c.dst_pos;
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        if (whole) dst[i] = src[i];
        else dst[i].w = src[i].w;
    }
}

int hw_threads() {
    unsigned n = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(n, 32u));
}

template <class F>
void parallel_for(int n, F f) {
    int nt = std::min(hw_threads(), n);
    if (nt <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int i = t; i < n; i += nt) f(i);
        });
    for (auto &x : th) x.join();
}

}  // namespace

struct SplitState {
    int dg = 0, P = 0;
    std::vector<uint32_t> root_keys;
    std::vector<int> root_owner;
    std::vector<int> rlo;              // [P + 1] first local root of each rank
    std::vector<int64_t> pt_lo;        // [P + 1] first sorted point of each rank
    std::vector<fmm_ctx *> views;      // P rank contexts, then the global context
    std::vector<std::vector<void *>> owned;   // per rank context: its tree tables
    // per rank, per level: own boxes [lo, hi) of the global level, and ghost keys
    std::vector<std::vector<int64_t>> lo, hi;
    std::vector<std::vector<std::vector<uint32_t>>> vghost;   // [rank][level]
    std::vector<std::vector<uint32_t>> ughost;                // [rank]
    std::vector<std::vector<int>> nb_u, nb_v;
    std::vector<int64_t> nq_u, nq_v, n_ghost_pts;
    std::vector<int64_t> bytes_u, bytes_v, bytes_gather, bytes_scatter;
    // exchange tables (device)
    RowCopy *vex = nullptr, *gat = nullptr, *sca = nullptr;
    PtsCopy *uex = nullptr;
    int n_vex = 0, n_gat = 0, n_uex = 0;
    std::vector<RowArray> arr_v, arr_up, arr_dn;
    void *pts_base = nullptr;          // device [P] point arrays of the ranks
    std::vector<void *> allocs;        // the tables above
    cudaEvent_t ev[10] = {};
    bool timed = false;
    // Concurrency: the ranks' chains of launches run on a pool of far-field streams (highest
    // priority) and their ULI on near-field streams (lowest), forked from and joined into a
    // capture stream; the whole evaluation is captured once per output mode as a CUDA graph
    // that reads the densities from q_in and writes phi_out / grad_out.
    static constexpr int kFar = 48, kNear = 8;
    cudaStream_t cap = nullptr, far_s[kFar] = {}, near_s[kNear] = {};
    cudaEvent_t fork = nullptr, ev_far[kFar] = {}, ev_near[kNear] = {}, ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec[4] = {};      // by output mode: 1 potentials, 2 gradients, 3 both
    long long graph_launches[4] = {};  // kernels in each graph
    void *q_in = nullptr, *phi_out = nullptr, *grad_out = nullptr;
};

namespace {

fmm_status sfail(fmm_ctx *ctx, fmm_status st, const std::string &m) {
    ctx->err = m;
    return st;
}

// the shared part of a view: options, streams, operators
fmm_ctx *new_view(const fmm_ctx *ctx) {
    fmm_ctx *v = new fmm_ctx();
    v->opt = ctx->opt;
    v->stream = ctx->stream;
    v->device = ctx->device;
    v->fp64 = ctx->fp64;
    v->tensor = ctx->tensor;
    v->ns = ctx->ns, v->nsp = ctx->nsp, v->npts = ctx->npts;
    v->cplx = ctx->cplx;
    for (int a = 0; a < 3; ++a) v->origin[a] = ctx->origin[a];
    v->side = ctx->side;
    v->grid_dev = ctx->grid_dev;
    for (int l = 0; l <= kMaxDepth; ++l) {
        v->host_ops[l] = ctx->host_ops[l];
        v->fwd[l] = ctx->fwd[l], v->adj[l] = ctx->adj[l];
        v->tc_fwd[l] = ctx->tc_fwd[l], v->tc_adj[l] = ctx->tc_adj[l];
    }
    v->class_slots = ctx->class_slots, v->class_delta = ctx->class_delta;
    v->dev_flag = ctx->dev_flag;
    v->have_ops = true;
    v->have_tree = true;
    return v;
}

void free_view(fmm_ctx *v, std::vector<void *> *owned) {
    free_workspace(v);
    if (owned)
        for (void *p : *owned) cudaFreeAsync(p, v->stream);
    if (v->host_tiles) cudaFreeHost(v->host_tiles);
    if (v->tiles_ev) cudaEventDestroy(v->tiles_ev);
    delete v;
}

template <typename V>
cudaError_t upload(const std::vector<V> &h, V **out, std::vector<void *> &owned, cudaStream_t s) {
    *out = nullptr;
    FMM_CUDA_TRY(pool_alloc((void **)out, std::max<size_t>(h.size() * sizeof(V), 16), s));
    owned.push_back(*out);
    if (!h.empty()) FMM_CUDA_TRY(cudaMemcpyAsync(*out, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
    return cudaSuccess;
}

template <typename V>
cudaError_t download(const V *d, size_t n, std::vector<V> &h, cudaStream_t s) {
    h.resize(n);
    if (n) FMM_CUDA_TRY(cudaMemcpyAsync(h.data(), d, n * sizeof(V), cudaMemcpyDeviceToHost, s));
    return cudaSuccess;
}

cudaError_t copy_rows(const RowCopy *e, int n, const RowArray &a, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 7) / 8);
    if (a.aligned16 && a.row_bytes % 16 == 0 && a.ld % 16 == 0)
        copy_rows_kernel<uint4><<<blocks, 256, 0, s>>>(e, n, a.base, a.ld, a.row_bytes / 16);
    else
        copy_rows_kernel<uint32_t><<<blocks, 256, 0, s>>>(e, n, a.base, a.ld, a.row_bytes / 4);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

void split_free(fmm_ctx *ctx) {
    SplitState *S = ctx->split;
    if (!S) return;
    cudaStreamSynchronize(ctx->stream);
    for (size_t k = 0; k < S->views.size(); ++k)
        free_view(S->views[k], k < S->owned.size() ? &S->owned[k] : nullptr);
    for (void *p : S->allocs) cudaFreeAsync(p, ctx->stream);
    for (auto &e : S->ev)
        if (e) cudaEventDestroy(e);
    for (auto &g : S->exec)
        if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t st : S->far_s)
        if (st) cudaStreamDestroy(st);
    for (cudaStream_t st : S->near_s)
        if (st) cudaStreamDestroy(st);
    if (S->cap) cudaStreamDestroy(S->cap);
    for (cudaEvent_t ev : S->ev_far)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : S->ev_near)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : {S->fork, S->ev_in, S->ev_out})
        if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(ctx->stream);
    delete S;
    ctx->split = nullptr;
}

fmm_status split_setup(fmm_ctx *ctx, int dg, int P) {
    const int d = ctx->opt.depth;
    if (!ctx->have_tree) return sfail(ctx, FMM_ESTATE, "fmm_build_tree has not been called");
    if (!ctx->have_ops) return sfail(ctx, FMM_ESTATE, "fmm_precompute has not been called");
    if (ctx->opt.mean_free) return sfail(ctx, FMM_EUNSUPPORTED, "the partitioned evaluation does not take mean_free");
    if (dg < 2 || dg >= d) return sfail(ctx, FMM_EINVAL, "d_global must satisfy 2 <= d_global < depth");
    const int64_t n_roots = ctx->lev[dg].n;
    if (P < 1 || P > n_roots)
        return sfail(ctx, FMM_EINVAL, "n_ranks must be in [1, " + std::to_string(n_roots) + "] (the local roots)");
    split_free(ctx);
    cudaStream_t s = ctx->stream;
    const int nleaf = ctx->nleaf;
    const size_t psz = ctx->fp64 ? 32 : 16;   // one point (x, y, z, q)

    // host copy of the global tree's levels d_global..d
    std::vector<std::vector<uint32_t>> keys(d + 1);
    std::vector<std::vector<int>> par(d + 1), chi(d + 1);
    std::vector<int> leaf_off, u_off, u_idx;
    cudaError_t e = cudaSuccess;
    for (int l = dg; l <= d && e == cudaSuccess; ++l) {
        const size_t n = (size_t)ctx->lev[l].n;
        e = download(ctx->lev[l].keys, n, keys[l], s);
        if (e == cudaSuccess && l > dg) e = download(ctx->lev[l].parent, n, par[l], s);
        if (e == cudaSuccess && l < d) e = download(ctx->lev[l].child, n * 8, chi[l], s);
    }
    if (e == cudaSuccess) e = download(ctx->leaf_off, (size_t)nleaf + 1, leaf_off, s);
    if (e == cudaSuccess) e = download(ctx->u_off, (size_t)nleaf + 1, u_off, s);
    if (e == cudaSuccess) e = download(ctx->u_idx, (size_t)ctx->n_u, u_idx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sfail(ctx, FMM_ECUDA, std::string("partition setup: ") + cudaGetErrorString(e));

    auto S = new SplitState();
    ctx->split = S;
    S->dg = dg, S->P = P;
    S->root_keys = keys[dg];

    // (2) layout: contiguous runs of local roots balanced by their point counts
    std::vector<int64_t> root_pts(n_roots + 1, 0);
    {
        int64_t li = 0;
        for (int64_t i = 0; i < n_roots; ++i) {
            const int64_t l0 = li;
            while (li < nleaf && (keys[d][li] >> (3 * (d - dg))) == keys[dg][i]) ++li;
            root_pts[i + 1] = root_pts[i] + (leaf_off[li] - leaf_off[l0]);
        }
    }
    S->rlo.assign(P + 1, 0);
    S->rlo[P] = (int)n_roots;
    for (int r = 1; r < P; ++r) {
        const double target = (double)root_pts[n_roots] * r / P;
        int i = (int)(std::lower_bound(root_pts.begin(), root_pts.end(), (int64_t)std::ceil(target)) - root_pts.begin());
        i = std::max(i, S->rlo[r - 1] + 1);
        i = std::min(i, (int)n_roots - (P - r));
        S->rlo[r] = i;
    }
    S->root_owner.assign(n_roots, 0);
    std::vector<int> owner_at((size_t)1 << (3 * dg), -1);   // local root key -> rank
    for (int r = 0; r < P; ++r)
        for (int i = S->rlo[r]; i < S->rlo[r + 1]; ++i) {
            S->root_owner[i] = r;
            owner_at[keys[dg][i]] = r;
        }
    // own boxes of every level: a contiguous run of the level's sorted keys
    S->lo.assign(P, std::vector<int64_t>(d + 1, 0));
    S->hi.assign(P, std::vector<int64_t>(d + 1, 0));
    for (int r = 0; r < P; ++r)
        for (int l = dg; l <= d; ++l) {
            const int sh = 3 * (l - dg);
            auto first = [&](int root) -> int64_t {
                if (root >= n_roots) return (int64_t)keys[l].size();
                const uint32_t rk = keys[dg][root];
                return std::lower_bound(keys[l].begin(), keys[l].end(), rk,
                                        [&](uint32_t k, uint32_t v) { return (k >> sh) < v; }) - keys[l].begin();
            };
            S->lo[r][l] = first(S->rlo[r]);
            S->hi[r][l] = first(S->rlo[r + 1]);
        }
    S->pt_lo.assign(P + 1, 0);
    for (int r = 0; r <= P; ++r) S->pt_lo[r] = r < P ? leaf_off[S->lo[r][d]] : leaf_off[nleaf];

    // (3)-(6) queries, neighbourhoods and existence answers, per rank
    std::vector<int> slots, deltas;
    class_slot_table(slots, deltas);
    S->vghost.assign(P, std::vector<std::vector<uint32_t>>(d + 1));
    S->ughost.assign(P, {});
    S->nb_u.assign(P, {}), S->nb_v.assign(P, {});
    S->nq_u.assign(P, 0), S->nq_v.assign(P, 0);
    auto exists = [&](int owner, int l, uint32_t k) -> bool {   // the owner's answer
        auto b = keys[l].begin() + S->lo[owner][l], en = keys[l].begin() + S->hi[owner][l];
        auto it = std::lower_bound(b, en, k);
        return it != en && *it == k;
    };
    parallel_for(P, [&](int r) {
        std::vector<std::vector<uint32_t>> q(P);
        std::vector<char> nbu(P, 0), nbv(P, 0);
        auto ask = [&](int l, int x, int y, int z) {
            const int m = 1 << l;
            if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) return;
            const uint32_t nk = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
            const int own = owner_at[nk >> (3 * (l - dg))];
            if (own < 0 || own == r) return;   // empty subdomain, or held locally
            q[own].push_back(nk);
        };
        auto answer = [&](int l, std::vector<char> &nb, int64_t &nq, std::vector<uint32_t> &out) {
            for (int o = 0; o < P; ++o) {
                auto &v = q[o];
                if (v.empty()) continue;
                std::sort(v.begin(), v.end());
                v.erase(std::unique(v.begin(), v.end()), v.end());
                nb[o] = 1;
                nq += (int64_t)v.size();
                for (uint32_t k : v)
                    if (exists(o, l, k)) out.push_back(k);
                v.clear();
            }
            std::sort(out.begin(), out.end());
        };
        for (int l = dg + 1; l <= d; ++l) {   // V packets
            for (int64_t i = S->lo[r][l]; i < S->hi[r][l]; ++i) {
                int ax, ay, az;
                const uint32_t k = keys[l][i];
                demorton3(k, ax, ay, az);
                const int c = (int)(k & 7);
                for (int sl = 0; sl < kClassSlots; ++sl) {
                    int dx, dy, dz;
                    unpack_delta(deltas[c * kClassSlots + sl], dx, dy, dz);
                    ask(l, ax + dx, ay + dy, az + dz);
                }
            }
            answer(l, nbv, S->nq_v[r], S->vghost[r][l]);
        }
        for (int64_t i = S->lo[r][d]; i < S->hi[r][d]; ++i) {   // U packets
            int ax, ay, az;
            demorton3(keys[d][i], ax, ay, az);
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz)
                        if (dx || dy || dz) ask(d, ax + dx, ay + dy, az + dz);
        }
        answer(d, nbu, S->nq_u[r], S->ughost[r]);
        for (int o = 0; o < P; ++o) {
            if (nbu[o]) S->nb_u[r].push_back(o);
            if (nbv[o]) S->nb_v[r].push_back(o);
        }
    });

    // local essential trees of the ranks: host tables
    struct LetHost {
        std::vector<uint32_t> keys[kMaxDepth + 1];
        std::vector<int> parent[kMaxDepth + 1], child[kMaxDepth + 1], cls[kMaxDepth + 1];
        int cls_off[kMaxDepth + 1][9] = {};
        int64_t row_base[kMaxDepth + 1] = {};
        int64_t rows = 0;
        std::vector<int> leaf_off, u_off, u_idx, order;
        std::vector<PtsCopy> pts_in;
        int64_t n_pts = 0, n_own_pts = 0;
        bool ok = true;
    };
    std::vector<LetHost> let(P);
    parallel_for(P, [&](int r) {
        LetHost &H = let[r];
        for (int l = dg; l <= d; ++l) {
            const int64_t lo = S->lo[r][l], hi = S->hi[r][l], n_own = hi - lo;
            std::vector<uint32_t> gh;
            if (l > dg) gh = S->vghost[r][l];
            if (l == d) {   // U ghosts join the leaf level's ghosts
                std::vector<uint32_t> m;
                std::merge(gh.begin(), gh.end(), S->ughost[r].begin(), S->ughost[r].end(), std::back_inserter(m));
                m.erase(std::unique(m.begin(), m.end()), m.end());
                gh.swap(m);
            }
            auto &K = H.keys[l];
            K.assign(keys[l].begin() + lo, keys[l].begin() + hi);
            K.insert(K.end(), gh.begin(), gh.end());
            const int64_t n_let = (int64_t)K.size();
            H.parent[l].assign(n_let, -1);
            if (l > dg)
                for (int64_t i = 0; i < n_own; ++i) H.parent[l][i] = (int)(par[l][lo + i] - S->lo[r][l - 1]);
            if (l < d) {
                H.child[l].assign(n_let * 8, -1);
                for (int64_t i = 0; i < n_own; ++i)
                    for (int c = 0; c < 8; ++c) {
                        const int g = chi[l][(lo + i) * 8 + c];
                        H.child[l][i * 8 + c] = g >= 0 ? (int)(g - S->lo[r][l + 1]) : -1;
                    }
            }
            // own boxes in octant-class order (stable)
            auto &C = H.cls[l];
            for (int c = 0; c < 8; ++c) {
                H.cls_off[l][c] = (int)C.size();
                for (int64_t i = 0; i < n_own; ++i)
                    if ((int)(K[i] & 7) == c) C.push_back((int)i);
            }
            H.cls_off[l][8] = (int)C.size();
            H.row_base[l] = H.rows;
            H.rows += n_let;
        }
        // leaves: own points first, then the U ghosts' points in key order
        const int64_t lo = S->lo[r][d], hi = S->hi[r][d], n_own = hi - lo;
        const auto &K = H.keys[d];
        H.n_own_pts = leaf_off[hi] - leaf_off[lo];
        H.leaf_off.assign(K.size() + 1, 0);
        for (int64_t i = 0; i <= n_own; ++i) H.leaf_off[i] = (int)(leaf_off[lo + i] - leaf_off[lo]);
        int64_t pos = H.n_own_pts;
        for (size_t j = n_own; j < K.size(); ++j) {
            int cnt = 0;
            if (std::binary_search(S->ughost[r].begin(), S->ughost[r].end(), K[j])) {
                const int64_t g = std::lower_bound(keys[d].begin(), keys[d].end(), K[j]) - keys[d].begin();
                cnt = leaf_off[g + 1] - leaf_off[g];
                const int o = S->root_owner[std::lower_bound(keys[dg].begin(), keys[dg].end(), K[j] >> (3 * (d - dg))) -
                                            keys[dg].begin()];
                H.pts_in.push_back(PtsCopy{o, (int)(leaf_off[g] - S->pt_lo[o]), r, (int)pos, cnt});
            }
            pos += cnt;
            H.leaf_off[j + 1] = (int)pos;
        }
        H.n_pts = pos;
        // U lists of the own leaves, in the unpartitioned order (ascending Morton key)
        H.u_off.assign(n_own + 1, 0);
        std::vector<int64_t> work(n_own, 0);
        for (int64_t i = 0; i < n_own; ++i) {
            const int64_t g = lo + i;
            int64_t src = leaf_off[g + 1] - leaf_off[g];
            for (int e2 = u_off[g]; e2 < u_off[g + 1]; ++e2) {
                const int a = u_idx[e2];
                int loc;
                if (a >= lo && a < hi) {
                    loc = (int)(a - lo);
                } else {
                    auto it = std::lower_bound(K.begin() + n_own, K.end(), keys[d][a]);
                    if (it == K.end() || *it != keys[d][a]) {
                        H.ok = false;
                        loc = 0;
                    } else {
                        loc = (int)(it - K.begin());
                    }
                }
                H.u_idx.push_back(loc);
                if (a != g) src += leaf_off[a + 1] - leaf_off[a];
            }
            H.u_off[i + 1] = (int)H.u_idx.size();
            work[i] = (leaf_off[g + 1] - leaf_off[g]) * src;
        }
        H.order.resize(n_own);
        for (int64_t i = 0; i < n_own; ++i) H.order[i] = (int)i;
        std::stable_sort(H.order.begin(), H.order.end(), [&](int a, int b) { return work[a] > work[b]; });
    });
    for (int r = 0; r < P; ++r)
        if (!let[r].ok) {
            split_free(ctx);
            return sfail(ctx, FMM_ECUDA, "partition setup: a U-list leaf has no owner answer");
        }

    // rank contexts: their tables, points and workspaces
    S->owned.assign(P, {});
    e = cudaSuccess;
    for (int r = 0; r < P && e == cudaSuccess; ++r) {
        LetHost &H = let[r];
        fmm_ctx *v = new_view(ctx);
        S->views.push_back(v);
        auto &own = S->owned[r];
        for (int l = dg; l <= d && e == cudaSuccess; ++l) {
            LevelTables &L = v->lev[l];
            L.n = S->hi[r][l] - S->lo[r][l];
            L.row_base = H.row_base[l];
            std::memcpy(L.cls_off, H.cls_off[l], sizeof(L.cls_off));
            e = upload(H.keys[l], &L.keys, own, s);
            if (e == cudaSuccess) {   // the dense table is filled on the device (8^l entries)
                const size_t nd = (size_t)1 << (3 * l);
                e = pool_alloc((void **)&L.dense, nd * sizeof(int), s);
                if (e == cudaSuccess) own.push_back(L.dense);
                if (e == cudaSuccess) e = cudaMemsetAsync(L.dense, 0xff, nd * sizeof(int), s);
                const int n_let = (int)H.keys[l].size();
                if (e == cudaSuccess && n_let) {
                    let_dense_kernel<<<(n_let + 255) / 256, 256, 0, s>>>(L.keys, n_let, L.dense);
                    count_launch();
                    e = cudaGetLastError();
                }
            }
            if (e == cudaSuccess) e = upload(H.parent[l], &L.parent, own, s);
            if (e == cudaSuccess && l < d) e = upload(H.child[l], &L.child, own, s);
            if (e == cudaSuccess) e = upload(H.cls[l], &L.cls_rows, own, s);
        }
        v->total_rows = H.rows;
        v->nleaf = (int)(S->hi[r][d] - S->lo[r][d]);
        v->n = H.n_own_pts;
        v->n_pts_all = H.n_pts;
        if (e == cudaSuccess) e = upload(H.leaf_off, &v->leaf_off, own, s);
        if (e == cudaSuccess) e = upload(H.u_off, &v->u_off, own, s);
        if (e == cudaSuccess) e = upload(H.u_idx, &v->u_idx, own, s);
        if (e == cudaSuccess) e = upload(H.order, &v->p2p_order, own, s);
        v->n_u = (int64_t)H.u_idx.size();
        if (e == cudaSuccess) {
            e = pool_alloc(&v->pts, std::max<size_t>(H.n_pts * psz, 16), s);
            if (e == cudaSuccess) own.push_back(v->pts);
        }
        if (e == cudaSuccess && H.n_own_pts)
            e = cudaMemcpyAsync(v->pts, (const unsigned char *)ctx->pts + S->pt_lo[r] * psz, H.n_own_pts * psz,
                                cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) {
        split_free(ctx);
        return sfail(ctx, FMM_ECUDA, std::string("partition setup: ") + cudaGetErrorString(e));
    }
    // the nominated context of the global stage: the tree's levels 0..d_global (tables shared)
    {
        fmm_ctx *g = new_view(ctx);
        for (int l = 0; l <= dg; ++l) g->lev[l] = ctx->lev[l];
        g->total_rows = ctx->lev[dg].row_base + ctx->lev[dg].n;
        g->nleaf = 0;
        g->n = 0;
        S->views.push_back(g);
    }
    for (fmm_ctx *v : S->views) {
        fmm_status st = ensure_workspace(v);
        if (st != FMM_OK) {
            const std::string m = v->err;
            split_free(ctx);
            return sfail(ctx, st, "partition workspaces: " + m);
        }
    }

    // exchange tables
    const int nsp = ctx->nsp, kw = S->views[0]->ws_kw;
    const int es = ctx->fp64 ? 8 : 4;
    const bool f16 = ctx->opt.precision == FMM_FP16X3;
    const int np = ctx->opt.precision == FMM_BF16X6 ? 3 : 2;
    const int pesz = ctx->opt.precision == FMM_TF32X3 ? 4 : 2;
    const int nck_s = (nsp + 63) / 64, nck_k = (kw + 63) / 64;
    std::vector<RowCopy> vex, gat, sca;
    std::vector<PtsCopy> uex;
    S->n_ghost_pts.assign(P, 0);
    for (int r = 0; r < P; ++r) {
        const LetHost &H = let[r];
        for (int l = dg + 1; l <= d; ++l) {
            const int64_t n_own = S->hi[r][l] - S->lo[r][l];
            for (uint32_t k : S->vghost[r][l]) {
                const int64_t g = std::lower_bound(keys[l].begin(), keys[l].end(), k) - keys[l].begin();
                const int o = S->root_owner[std::lower_bound(keys[dg].begin(), keys[dg].end(), k >> (3 * (l - dg))) -
                                            keys[dg].begin()];
                const int64_t j = std::lower_bound(H.keys[l].begin() + n_own, H.keys[l].end(), k) - H.keys[l].begin();
                vex.push_back(RowCopy{o, (int)(let[o].row_base[l] + (g - S->lo[o][l])), r, (int)(H.row_base[l] + j)});
            }
        }
        for (int i = 0; i < S->rlo[r + 1] - S->rlo[r]; ++i) {
            gat.push_back(RowCopy{r, (int)(H.row_base[dg] + i), P, (int)(ctx->lev[dg].row_base + S->rlo[r] + i)});
            sca.push_back(RowCopy{P, (int)(ctx->lev[dg].row_base + S->rlo[r] + i), r, (int)(H.row_base[dg] + i)});
        }
        for (const PtsCopy &c : H.pts_in) {
            uex.push_back(c);
            S->n_ghost_pts[r] += c.count;
        }
    }
    S->n_vex = (int)vex.size(), S->n_gat = (int)gat.size(), S->n_uex = (int)uex.size();
    e = upload(vex, &S->vex, S->allocs, s);
    if (e == cudaSuccess) e = upload(gat, &S->gat, S->allocs, s);
    if (e == cudaSuccess) e = upload(sca, &S->sca, S->allocs, s);
    if (e == cudaSuccess) e = upload(uex, &S->uex, S->allocs, s);
    // the arrays each exchange copies, as base pointers of every context
    auto arr = [&](auto base_of, long long ld, int row_bytes, std::vector<RowArray> &out) {
        if (e != cudaSuccess) return;
        std::vector<unsigned char *> b;
        for (fmm_ctx *v : S->views) b.push_back(base_of(v));
        RowArray a;
        a.ld = ld, a.row_bytes = row_bytes;
        a.aligned16 = true;
        for (unsigned char *p : b) a.aligned16 = a.aligned16 && ((uintptr_t)p & 15) == 0;
        e = upload(b, &a.base, S->allocs, s);
        out.push_back(a);
    };
    if (!ctx->tensor) {
        arr([&](fmm_ctx *v) { return (unsigned char *)v->Ut; }, (long long)kw * es, kw * es, S->arr_v);
    } else {
        for (int p = 0; p < np; ++p)
            arr([&](fmm_ctx *v) { return (unsigned char *)v->UtP + p * v->utp_plane; }, (long long)kw * pesz, kw * pesz,
                S->arr_v);
        if (f16) arr([&](fmm_ctx *v) { return (unsigned char *)v->Uscale; }, nck_k * 4LL, nck_k * 4, S->arr_v);
    }
    arr([&](fmm_ctx *v) { return (unsigned char *)v->Uc; }, (long long)nsp * es, nsp * es, S->arr_up);
    arr([&](fmm_ctx *v) { return (unsigned char *)v->Dc; }, (long long)nsp * es, nsp * es, S->arr_dn);
    if (f16) {
        for (int p = 0; p < 2; ++p) {
            arr([&](fmm_ctx *v) { return (unsigned char *)v->UpP + p * v->upp_plane; }, nsp * 2LL, nsp * 2, S->arr_up);
            arr([&](fmm_ctx *v) { return (unsigned char *)v->DnP + p * v->upp_plane; }, nsp * 2LL, nsp * 2, S->arr_dn);
        }
        arr([&](fmm_ctx *v) { return (unsigned char *)v->Ups; }, nck_s * 4LL, nck_s * 4, S->arr_up);
        arr([&](fmm_ctx *v) { return (unsigned char *)v->Dns; }, nck_s * 4LL, nck_s * 4, S->arr_dn);
    }
    if (e == cudaSuccess) {
        std::vector<void *> pb;
        for (int r = 0; r < P; ++r) pb.push_back(S->views[r]->pts);
        void **d_pb = nullptr;
        e = upload(pb, &d_pb, S->allocs, s);
        S->pts_base = d_pb;
    }
    // coordinates of the U ghost points (once; the densities move at every evaluation)
    if (e == cudaSuccess && S->n_uex) {
        if (ctx->fp64)
            copy_pts_kernel<double4><<<S->n_uex, 128, 0, s>>>(S->uex, (double4 *const *)S->pts_base, 1);
        else
            copy_pts_kernel<float4><<<S->n_uex, 128, 0, s>>>(S->uex, (float4 *const *)S->pts_base, 1);
        count_launch();
        e = cudaGetLastError();
    }
    for (auto &ev : S->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    {   // streams and events of the concurrent schedule; fixed input and output buffers
        int lo_p = 0, hi_p = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo_p, &hi_p);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S->cap, cudaStreamNonBlocking, hi_p);
        for (int k = 0; k < SplitState::kFar && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithPriority(&S->far_s[k], cudaStreamNonBlocking, hi_p);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_far[k], cudaEventDisableTiming);
        }
        for (int k = 0; k < SplitState::kNear && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithPriority(&S->near_s[k], cudaStreamNonBlocking, lo_p);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_near[k], cudaEventDisableTiming);
        }
        for (cudaEvent_t *ev : {&S->fork, &S->ev_in, &S->ev_out})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        const size_t es_b = ctx->fp64 ? 8 : 4;
        const size_t n = (size_t)ctx->n;
        for (auto pr : {std::make_pair(&S->q_in, n), std::make_pair(&S->phi_out, n), std::make_pair(&S->grad_out, 3 * n)})
            if (e == cudaSuccess) {
                e = pool_alloc(pr.first, std::max<size_t>(pr.second * es_b, 16), s);
                if (e == cudaSuccess) S->allocs.push_back(*pr.first);
            }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host tables above are released next
    if (e != cudaSuccess) {
        split_free(ctx);
        return sfail(ctx, FMM_ECUDA, std::string("partition setup: ") + cudaGetErrorString(e));
    }
    // bytes each rank receives (U, V, scatter) or sends (gather) per evaluation
    auto row_bytes = [](const std::vector<RowArray> &v) {
        int64_t b = 0;
        for (const RowArray &a : v) b += a.row_bytes;
        return b;
    };
    S->bytes_u.assign(P, 0), S->bytes_v.assign(P, 0), S->bytes_gather.assign(P, 0), S->bytes_scatter.assign(P, 0);
    for (int r = 0; r < P; ++r) {
        int64_t nv = 0;
        for (int l = dg + 1; l <= d; ++l) nv += (int64_t)S->vghost[r][l].size();
        S->bytes_u[r] = S->n_ghost_pts[r] * es;
        S->bytes_v[r] = nv * row_bytes(S->arr_v);
        S->bytes_gather[r] = (int64_t)(S->rlo[r + 1] - S->rlo[r]) * row_bytes(S->arr_up);
        S->bytes_scatter[r] = (int64_t)(S->rlo[r + 1] - S->rlo[r]) * row_bytes(S->arr_dn);
    }
    return FMM_OK;
}

namespace {

// The evaluation of one output mode, enqueued on the capture stream (it is captured, not run).
template <typename T>
cudaError_t split_enqueue(fmm_ctx *ctx, SplitState &S, bool want_phi, bool want_grad) {
    cudaStream_t s = S.cap;
    const int P = S.P, dg = S.dg, d = ctx->opt.depth;
    const int K = std::min(P, SplitState::kFar), Kn = std::min(P, SplitState::kNear);
    using P4 = typename std::conditional<sizeof(T) == 8, double4, float4>::type;
    T *phi_o = want_phi ? (T *)S.phi_out : nullptr, *grad_o = want_grad ? (T *)S.grad_out : nullptr;
    auto fork = [&](cudaStream_t *to, int n) -> cudaError_t {
        FMM_CUDA_TRY(cudaEventRecord(S.fork, s));
        for (int k = 0; k < n; ++k) FMM_CUDA_TRY(cudaStreamWaitEvent(to[k], S.fork, 0));
        return cudaSuccess;
    };
    // phase boundaries: events the graph records when it runs (external event record nodes)
    auto mark = [&](cudaEvent_t ev) { return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal); };
    auto join = [&](cudaStream_t *from, cudaEvent_t *evs, int n) -> cudaError_t {
        for (int k = 0; k < n; ++k) {
            FMM_CUDA_TRY(cudaEventRecord(evs[k], from[k]));
            FMM_CUDA_TRY(cudaStreamWaitEvent(s, evs[k], 0));
        }
        return cudaSuccess;
    };
    FMM_CUDA_TRY(mark(S.ev[0]));
    // densities: every rank's own points, then its U ghosts' (U exchange)
    FMM_CUDA_TRY(fork(S.far_s, K));
    for (int r = 0; r < P; ++r)
        FMM_CUDA_TRY(launch_gather_points<T>((const T *)S.q_in, ctx->perm + S.pt_lo[r], S.views[r]->pts,
                                             S.views[r]->n, S.far_s[r % K]));
    FMM_CUDA_TRY(join(S.far_s, S.ev_far, K));
    if (S.n_uex) {
        copy_pts_kernel<P4><<<S.n_uex, 128, 0, s>>>(S.uex, (P4 *const *)S.pts_base, 0);
        count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    FMM_CUDA_TRY(mark(S.ev[1]));
    // the ULI of every rank on the near-field streams, beside everything that follows
    FMM_CUDA_TRY(fork(S.near_s, Kn));
    for (int r = 0; r < P; ++r) {
        fmm_ctx *v = S.views[r];
        FMM_CUDA_TRY(launch_p2p<T>(v, want_phi ? (T *)v->near_phi : nullptr, want_grad ? (T *)v->near_grad : nullptr,
                                   S.near_s[r % Kn]));
    }
    // local stage: S2U, U2U up to the local roots, VLI compress below d_global
    FMM_CUDA_TRY(fork(S.far_s, K));
    for (int r = 0; r < P; ++r) {
        FarSteps<T> f(S.views[r], false);
        cudaStream_t fs = S.far_s[r % K];
        FMM_CUDA_TRY(f.leaf_in(fs));
        for (int l = d - 1; l >= dg; --l) FMM_CUDA_TRY(f.up(l, fs));
        for (int l = dg + 1; l <= d; ++l) FMM_CUDA_TRY(f.compress(l, fs));
    }
    FMM_CUDA_TRY(join(S.far_s, S.ev_far, K));
    FMM_CUDA_TRY(mark(S.ev[2]));
    for (const RowArray &a : S.arr_v) FMM_CUDA_TRY(copy_rows(S.vex, S.n_vex, a, s));   // V exchange
    FMM_CUDA_TRY(mark(S.ev[3]));
    for (const RowArray &a : S.arr_up) FMM_CUDA_TRY(copy_rows(S.gat, S.n_gat, a, s));  // gather
    FMM_CUDA_TRY(mark(S.ev[4]));
    {   // global stage on the nominated context
        FarSteps<T> g(S.views[P], false);
        for (int l = dg - 1; l >= 2; --l) FMM_CUDA_TRY(g.up(l, s));
        for (int l = 2; l <= dg; ++l) {
            FMM_CUDA_TRY(g.compress(l, s));
            FMM_CUDA_TRY(g.stencil(l, s));
        }
        for (int l = 2; l <= dg; ++l) FMM_CUDA_TRY(g.down(l, s));
    }
    FMM_CUDA_TRY(mark(S.ev[5]));
    for (const RowArray &a : S.arr_dn) FMM_CUDA_TRY(copy_rows(S.sca, S.n_gat, a, s));  // scatter
    FMM_CUDA_TRY(mark(S.ev[6]));
    // local downward stage
    FMM_CUDA_TRY(fork(S.far_s, K));
    for (int r = 0; r < P; ++r) {
        fmm_ctx *v = S.views[r];
        FarSteps<T> f(v, false);
        cudaStream_t fs = S.far_s[r % K];
        for (int l = dg + 1; l <= d; ++l) FMM_CUDA_TRY(f.stencil(l, fs));
        for (int l = dg + 1; l <= d; ++l) FMM_CUDA_TRY(f.down(l, fs));
        FMM_CUDA_TRY(f.leaf_out(want_phi ? (T *)v->far_phi : nullptr, want_grad ? (T *)v->far_grad : nullptr, fs));
    }
    FMM_CUDA_TRY(join(S.far_s, S.ev_far, K));
    FMM_CUDA_TRY(mark(S.ev[7]));
    FMM_CUDA_TRY(join(S.near_s, S.ev_near, Kn));   // what is left of the ULI
    FMM_CUDA_TRY(mark(S.ev[8]));
    FMM_CUDA_TRY(fork(S.far_s, K));
    for (int r = 0; r < P; ++r) {   // outputs in input order
        fmm_ctx *v = S.views[r];
        FMM_CUDA_TRY(launch_scatter<T>(want_phi ? (const T *)v->near_phi : nullptr,
                                       want_grad ? (const T *)v->near_grad : nullptr,
                                       want_phi ? (const T *)v->far_phi : nullptr,
                                       want_grad ? (const T *)v->far_grad : nullptr, ctx->perm + S.pt_lo[r], phi_o,
                                       grad_o, v->n, S.far_s[r % K], ctx->n));
    }
    FMM_CUDA_TRY(join(S.far_s, S.ev_far, K));
    FMM_CUDA_TRY(mark(S.ev[9]));
    return cudaSuccess;
}

}  // namespace

template <typename T>
fmm_status split_run(fmm_ctx *ctx, const T *q, T *phi, T *grad) {
    SplitState &S = *ctx->split;
    cudaStream_t s = ctx->stream;
    const int mode = (phi ? 1 : 0) | (grad ? 2 : 0);
    const size_t n = (size_t)ctx->n;
    auto bad = [&](cudaError_t e) {
        ctx->err = std::string("partitioned evaluation: ") + cudaGetErrorString(e);
        return FMM_ECUDA;
    };
    cudaError_t e;
    if (!S.exec[mode]) {   // capture this output mode once
        const long long before = launches();
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(S.cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return bad(e);
        cudaError_t ee = split_enqueue<T>(ctx, S, phi != nullptr, grad != nullptr);
        e = cudaStreamEndCapture(S.cap, &graph);
        if (ee != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return bad(ee != cudaSuccess ? ee : e);
        }
        e = cudaGraphInstantiate(&S.exec[mode], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            S.exec[mode] = nullptr;
            return bad(e);
        }
        S.graph_launches[mode] = launches() - before;
        count_launches(-S.graph_launches[mode]);   // captured, not run: counted at every replay
    }
    if ((e = cudaMemcpyAsync(S.q_in, q, n * sizeof(T), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return bad(e);
    if ((e = cudaGraphLaunch(S.exec[mode], s)) != cudaSuccess) return bad(e);
    count_launches(S.graph_launches[mode]);
    if (phi && (e = cudaMemcpyAsync(phi, S.phi_out, n * sizeof(T), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return bad(e);
    if (grad && (e = cudaMemcpyAsync(grad, S.grad_out, 3 * n * sizeof(T), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return bad(e);
    S.timed = true;
    return FMM_OK;
}

template fmm_status split_run<float>(fmm_ctx *, const float *, float *, float *);
template fmm_status split_run<double>(fmm_ctx *, const double *, double *, double *);

// ---- exports ----
fmm_status split_info(fmm_ctx *ctx, int rank, fmm_rank_info *out) {
    const SplitState *S = ctx->split;
    if (!S) return sfail(ctx, FMM_ESTATE, "fmm_partition_setup has not been called");
    if (rank < 0 || rank >= S->P) return sfail(ctx, FMM_EINVAL, "rank out of range");
    std::memset(out, 0, sizeof(*out));
    const int d = ctx->opt.depth;
    out->rank = rank;
    out->n_ranks = S->P;
    out->d_global = S->dg;
    out->first_root = S->rlo[rank];
    out->n_local_roots = S->rlo[rank + 1] - S->rlo[rank];
    out->first_point = S->pt_lo[rank];
    out->n_points = S->pt_lo[rank + 1] - S->pt_lo[rank];
    for (int l = S->dg; l <= d; ++l) {
        out->n_boxes[l] = S->hi[rank][l] - S->lo[rank][l];
        out->n_ghost_v[l] = (int64_t)S->vghost[rank][l].size();
    }
    out->n_ghost_u = (int64_t)S->ughost[rank].size();
    out->n_ghost_points = S->n_ghost_pts[rank];
    out->n_query_u = S->nq_u[rank];
    out->n_query_v = S->nq_v[rank];
    out->n_neighbours_u = (int32_t)S->nb_u[rank].size();
    out->n_neighbours_v = (int32_t)S->nb_v[rank].size();
    out->bytes_u = S->bytes_u[rank];
    out->bytes_v = S->bytes_v[rank];
    out->bytes_gather = S->bytes_gather[rank];
    out->bytes_scatter = S->bytes_scatter[rank];
    return FMM_OK;
}

fmm_status split_export(fmm_ctx *ctx, int rank, int level, int kind, uint64_t *out, int64_t *count) {
    const SplitState *S = ctx->split;
    if (!S) return sfail(ctx, FMM_ESTATE, "fmm_partition_setup has not been called");
    if (!count) return sfail(ctx, FMM_EINVAL, "null count");
    if (kind == FMM_PARTITION_LAYOUT) {
        *count = (int64_t)S->root_keys.size();
        if (out)
            for (size_t i = 0; i < S->root_keys.size(); ++i) out[i] = S->root_keys[i] | ((uint64_t)S->root_owner[i] << 32);
        return FMM_OK;
    }
    if (rank < 0 || rank >= S->P) return sfail(ctx, FMM_EINVAL, "rank out of range");
    const int d = ctx->opt.depth;
    std::vector<uint64_t> v;
    switch (kind) {
        case FMM_PARTITION_OWN:
        case FMM_PARTITION_GHOST_V: {
            if (level < S->dg || level > d) return sfail(ctx, FMM_EINVAL, "level out of [d_global, depth]");
            if (kind == FMM_PARTITION_GHOST_V) {
                for (uint32_t k : S->vghost[rank][level]) v.push_back(k);
            } else {   // own keys: the rank context's first keys of the level
                const int64_t n = S->hi[rank][level] - S->lo[rank][level];
                std::vector<uint32_t> h((size_t)n);
                if (n && (cudaMemcpyAsync(h.data(), S->views[rank]->lev[level].keys, n * 4, cudaMemcpyDeviceToHost,
                                          ctx->stream) != cudaSuccess ||
                          cudaStreamSynchronize(ctx->stream) != cudaSuccess))
                    return sfail(ctx, FMM_ECUDA, "device-to-host copy");
                for (uint32_t k : h) v.push_back(k);
            }
            break;
        }
        case FMM_PARTITION_GHOST_U:
            for (uint32_t k : S->ughost[rank]) v.push_back(k);
            break;
        case FMM_PARTITION_NEIGHBOURS_U:
            for (int o : S->nb_u[rank]) v.push_back((uint64_t)o);
            break;
        case FMM_PARTITION_NEIGHBOURS_V:
            for (int o : S->nb_v[rank]) v.push_back((uint64_t)o);
            break;
        default:
            return sfail(ctx, FMM_EINVAL, "unknown export kind");
    }
    *count = (int64_t)v.size();
    if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(uint64_t));
    return FMM_OK;
}

fmm_status split_timings(fmm_ctx *ctx, double *ms, int n) {
    SplitState *S = ctx->split;
    if (!S) return sfail(ctx, FMM_ESTATE, "fmm_partition_setup has not been called");
    if (!S->timed) return sfail(ctx, FMM_ESTATE, "no partitioned evaluation yet");
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return sfail(ctx, FMM_ECUDA, "synchronize");
    for (int i = 0; i < n && i < 10; ++i) {   // -1 where the driver gives no time
        float t = 0;
        ms[i] = cudaEventElapsedTime(&t, S->ev[i == 9 ? 0 : i], S->ev[i == 9 ? 9 : i + 1]) == cudaSuccess ? t : -1.0;
    }
    cudaGetLastError();
    return FMM_OK;
}

}  // namespace fmm
