// Internal declarations of libfmm (not part of the C ABI).
//
// Representation.  Every box carries *check potentials* instead of equivalent densities:
//   U_l[b] = potential on the upward-check surface of box b due to the sources inside b,
//   D_l[b] = potential on the downward-check surface of b due to the sources far from b.
// The kiFMM operators of Table 1 then become products "evaluation o pseudo-inverse" formed in
// FP64 on the host, which are smooth and bounded, so they can be applied in FP32 or in split
// BF16/TF32 without the rounding amplification an explicit pseudo-inverse would cause:
//   U2U  U_P  = sum_c A_c U_c,        A_c = K(uc_P, ue_c) pinv(K(uc_c, ue_c))
//   VLI  D_b += sum_{a in V(b)} T_t U_a,  T_t = K(dc_b, ue_a) pinv(K(uc_a, ue_a)) ~ Uo C_t Vi^T
//   D2D  D_c += B_c D_P,              B_c = K(dc_c, de_P) pinv(K(dc_P, de_P))
//   D2T  d_b  = pinv(K(dc_b, de_b)) D_b  (factored: (V S^-1)(U^T D_b)), f += K(x, de_b) d_b
// For Laplace all of these are level-invariant in units of the box half-width (K is homogeneous
// of degree -1); only the leaf closing carries the factor r_leaf.  The modified Helmholtz kernel
// at half-width r is (1/r) times the unit-box kernel with kappa r, so it has one operator set per
// level (kappa r_l), with the same M2L ranks on every level, and the same r_leaf closing factor.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fmm.h"

namespace fmm {

constexpr int kMaxDepth = 10;
// device count array of the tree build: boxes per level, U-list entries, a non-finite
// coordinate flag, boxes per child octant per level
constexpr int kCntLevel = 0, kCntU = kMaxDepth + 1, kCntBad = kMaxDepth + 2, kCntOct = kMaxDepth + 3;
constexpr int kCntSize = kCntOct + 8 * (kMaxDepth + 1);
constexpr int kNumTransfer = 316;     // [-3,3]^3 minus [-1,1]^3
constexpr int kClassSlots = 189;      // transfer vectors with adjacent parents, per octant

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Operators of one direction (forward or adjoint) in one arithmetic, device-resident.
// Row-major [rows x cols] with cols padded: a matrix applied to a padded row vector.
struct OpSet {
    // host-side shapes
    int ns = 0, nsp = 0;        // surface size and its padding to 16
    int kin = 0, kinp = 0;      // M2L compressed source rank (Vi^T: kin x ns)
    int kout = 0, koutp = 0;    // M2L compressed target rank (Uo: ns x kout)
    int rcl = 0, rclp = 0;      // leaf-closing rank
    // Device pointers (element type = the context's storage type for SIMT; split planes for
    // tensor-core arithmetic live in TcOps).
    void *up[8] = {};           // U2U (children -> parent) per octant: [nsp x nsp]
    void *down[8] = {};         // D2D (parent -> child) per child octant: [nsp x nsp]
    void *compress = nullptr;   // [kinp x nsp]
    void *stencil = nullptr;    // [316][koutp x kinp]
    void *decompress = nullptr; // [nsp x koutp]
    void *close1 = nullptr;     // [rclp x nsp]  (U^T)          forward: applied before D2T
    void *close2 = nullptr;     // [nsp x rclp]  (V S^-1)
    // upward closing (forward sets only): equivalent densities from the upward check potentials,
    // read by the W-list step of the adaptive evaluation
    int rclu = 0, rclup = 0;
    void *uclose1 = nullptr;    // [rclup x nsp] (U^T)
    void *uclose2 = nullptr;    // [nsp x rclup] (V S^-1)
};

// Split operand planes for the tcgen05 GEMMs (gemm_tc.cu): planes[0] holds `count` operators,
// each `bytes` long, in the stage layout [K chunk][plane][rows x 128 B, SWIZZLE_128B].  Planes:
// BF16x3 {hi, lo}; BF16x6 {hi, lo, third}; TF32x3 {big, small}.
struct TcMat {
    void *planes[1] = {};
    int rows = 0, cols = 0;     // padded N x K
    int nplanes = 0;
    size_t bytes = 0;           // one operator
    float *scale = nullptr;     // FP16 planes: 1 / (power-of-two scale) per operator and K chunk
    int scale_ld = 0;           // K chunks per operator
};

struct TcOpSet {
    TcMat up;                   // 8 operators (children octants)
    TcMat down[8], compress, decompress;
    TcMat stencil;              // 316 operators
};

struct HostOps;  // FP64 host operators (precompute.cpp)
struct SplitState;  // virtual-rank partition (split.cu)
struct AdaptiveState;  // adaptive tree and its lists (adaptive.cu)

// Tile of output rows for the GEMM kernels: rows [row0, row0+nrows) of a level's row list,
// all of one child octant class `cls` (or -1 when not class-ordered); `mask` indexes the
// 6-word active-transfer bitmask of the tile (stencil GEMMs only).
struct Tile {
    int row0, nrows, cls, mask;
};

// Stream-ordered allocation from the library's per-device pool (memory is kept cached for
// reuse); freed with cudaFreeAsync.  pool_trim returns the unused memory to the driver.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
// cudaMalloc under the process-wide cap of fmm_set_alloc_limit (the library's other allocations)
cudaError_t dev_malloc(void **p, size_t bytes);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
void pool_trim();

struct LevelTables {
    int64_t n = 0;              // non-empty boxes
    uint32_t *keys = nullptr;   // ascending Morton keys
    int *parent = nullptr;      // index into level-1
    int *child = nullptr;       // [n x 8] index into level+1, -1 if empty
    int *dense = nullptr;       // [8^l] key -> index or -1 (levels >= 2)
    int *cls_rows = nullptr;    // box indices ordered by octant (stable)
    int cls_off[9] = {};        // host copy: class c rows are cls_rows[cls_off[c] .. cls_off[c+1])
    int64_t row_base = 0;       // first row of this level in the all-level arrays
};

struct TileSet {                // tiles of one level for one tile height
    int ntiles = 0;
    int tile_m = 0;             // rows per tile at most (0: the context's tile_m)
    Tile *tiles = nullptr;      // device
    uint32_t *masks = nullptr;  // device [ntiles x 6] (stencil active-slot bits)
    std::vector<Tile> host;
};

}  // namespace fmm

struct fmm_ctx {
    fmm_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    bool fp64 = false;
    bool tensor = false;        // tcgen05 contractions
    bool cplx = false;          // complex densities and outputs (FMM_HELMHOLTZ)
    bool fft = false;           // M2L by FFT (FMM_M2L_FFT)
    void *fft_ghat = nullptr;   // FFT M2L: the kernel's transforms [316][n n (n/2+1)] complex, storage type
    int *fft_surf = nullptr;    // FFT M2L: p^3 grid index of every surface point
    int *fft_tindex = nullptr;  // FFT M2L: transfer index of (neighbour offset, source octant, target octant), -1 near
    int npts = 0;               // surface points, 6(p-1)^2+2
    int ns = 0, nsp = 0;        // box vector length (npts, or 2 npts: real then imaginary parts), padded

    // tree
    bool have_tree = false;
    int64_t n = 0;
    double origin[3] = {0, 0, 0};
    double side = 1.0;
    int nleaf = 0;
    void *pts = nullptr;        // sorted (x, y, z, q) as float4 or double4
    int64_t n_pts_all = -1;     // points in pts when it holds more than n (a rank view's ghosts)
    int *perm = nullptr;        // sorted position -> input index
    int *inv_perm = nullptr;    // input index -> sorted position (made by the first evaluation with host outputs)
    int *leaf_off = nullptr;    // [nleaf+1]
    int *u_off = nullptr, *u_idx = nullptr;
    int64_t n_u = 0;
    int64_t p2p_pairs = 0;
    fmm::LevelTables lev[fmm::kMaxDepth + 1];
    int64_t total_rows = 0;     // sum of boxes over levels
    // tiles per level: [0] plain order (children gather), [1] class order with stencil masks
    fmm::TileSet tiles_plain[fmm::kMaxDepth + 1];
    fmm::TileSet tiles_cls[fmm::kMaxDepth + 1];
    int tile_m = 0;             // tile height the tile sets were built for
    int *class_slots = nullptr; // device [8][189] transfer index of each slot (per context)
    int *class_delta = nullptr; // device [8][189] packed (dx, dy, dz) of each slot (per context)
    // counts the tree build produces on the device, read back once per build (layout: kCnt*)
    int *dev_counts = nullptr, *host_counts = nullptr;   // device / pinned host [kCntSize]
    unsigned long long *dev_pairs = nullptr;              // device: near-field pair count
    fmm::Tile *host_tiles = nullptr;                      // pinned staging of the tile lists
    size_t host_tiles_cap = 0;
    cudaEvent_t tiles_ev = nullptr;                       // completion of the last tile copies
    cudaEvent_t masks_fork_ev = nullptr, masks_ev = nullptr;   // stencil masks: inputs ready / done
    // P2P schedule: leaves in decreasing work order
    int *p2p_order = nullptr;
    // class order of every level in one allocation (lev[l].cls_rows point into it); null when
    // each level owns its own array (the contexts of virtual ranks)
    int *cls_all = nullptr;

    // evaluate workspaces (allocated with the tree once operators are known)
    bool have_ws = false;
    bool tiles_ok = false;          // tiles of the current tree built
    int64_t ws_rows = 0, ws_nleaf = 0, ws_n = 0;   // capacity of the workspaces
    void *Uc = nullptr, *Dc = nullptr;   // [total_rows x nsp] upward / downward check potentials
    void *Ut = nullptr, *Ct = nullptr;   // [total_rows x ws_kw] compressed M2L vectors
    void *UtP = nullptr;                 // tensor-core modes: Ut as split planes [plane][rows x ws_kw]
    long long utp_plane = 0;             // bytes per plane
    void *Yc = nullptr;                  // [nleaf x rclp] closing intermediate
    void *Dq = nullptr;                  // [nleaf x nsp] leaf equivalent densities
    void *Cmean = nullptr;               // [total_rows] FP64 constant part of the downward check potentials
    float *Uscale = nullptr;             // FMM_FP16X3: 1 / scale of UtP per row and 64-column chunk
    // FMM_FP16X3: FP16 hi/lo planes (and scales) of the upward-side rows of the current direction
    // (UpP, [rows x nsp]), of its downward-side rows (DnP) and of the stencil output (CtP, [rows x ws_kw])
    void *UpP = nullptr, *DnP = nullptr, *CtP = nullptr;
    long long upp_plane = 0, ctp_plane = 0;   // bytes per plane (UpP and DnP share the first)
    float *Ups = nullptr, *Dns = nullptr, *Cts = nullptr;
    void *pts_qi = nullptr;              // FMM_HELMHOLTZ: imaginary parts of the sorted densities [n]
    void *near_phi = nullptr, *near_grad = nullptr;  // sorted-order outputs [n], [n x 3] (complex: x2)
    void *far_phi = nullptr, *far_grad = nullptr;
    size_t ws_bytes = 0;
    int ws_kw = 0;
    void *grid_dev = nullptr;            // unit surface grid [ns x 3] in the storage type
    // host-pointer staging
    void *stage_in = nullptr, *stage_out = nullptr, *stage_grad = nullptr;

    // operators
    bool have_ops = false;
    // one set per level (Laplace: every entry the same set; levels that no step uses alias a
    // used one); uniform shapes across levels
    const fmm::HostOps *host_ops[fmm::kMaxDepth + 1] = {};
    fmm::OpSet fwd[fmm::kMaxDepth + 1], adj[fmm::kMaxDepth + 1];
    fmm::TcOpSet *tc_fwd[fmm::kMaxDepth + 1] = {}, *tc_adj[fmm::kMaxDepth + 1] = {};
    std::vector<fmm::TcOpSet *> tc_owned;
    std::vector<void *> op_allocs;

    fmm::SplitState *split = nullptr;   // partitioned evaluation on virtual ranks (split.cu)
    fmm::AdaptiveState *adaptive = nullptr;   // adaptive tree and its lists (adaptive.cu)
    bool adaptive_eval = false;               // an evaluation over the adaptive tree is running

    bool last_adjoint = false;  // what the last evaluation left in the workspaces
    bool last_far = false;

    // concurrency: side streams for the near field and the per-level VLI (Section 2.2: the ULI is
    // independent of the far field and the VLI of different levels are independent)
    cudaStream_t aux[fmm::kMaxDepth + 2] = {};
    cudaEvent_t fork_ev[fmm::kMaxDepth + 2] = {}, join_ev[fmm::kMaxDepth + 2] = {};

    // timings
    cudaEvent_t ev[8] = {};
    float last_ms[5] = {};
    int *dev_flag = nullptr;    // device error flag (bounded waits, bounds checks)
    unsigned long long tc_wait_ns = 1000000000ull;   // bound on the tensor-core kernels' barrier waits
};

namespace fmm {

// Process-wide count of kernels launched by the library (every launch site calls it).
void count_launch();
long long launches();
void count_launches(long long n);   // the kernels of a replayed CUDA graph

// ---- precompute.cpp ----
struct HostOps {
    int p = 0;
    int ns = 0;                                       // box vector length (npts, or 2 npts if complex)
    int npts = 0;                                     // surface points
    int kernel = FMM_LAPLACE;
    double kappa_u = 0;                               // kernel's kappa (or wavenumber) x the half-width
    int kin = 0, kout = 0, rcl = 0;
    std::vector<double> surf_inner, surf_outer;       // [ns x 3] unit grids scaled by alpha
    std::vector<double> up[8], down[8];               // [ns x ns]
    std::vector<double> compress;                     // [kin x ns]   Vi^T
    std::vector<double> stencil;                      // [316][kout x kin]
    std::vector<double> decompress;                   // [ns x kout]  Uo
    std::vector<double> close1, close2;               // [rcl x ns], [ns x rcl] (unit box)
    int rclu = 0;                                     // rank of the upward check-to-equivalent map
    std::vector<double> uclose1, uclose2;             // [rclu x ns], [ns x rclu] (unit box)
    // adjoint (transposes)
    std::vector<double> a_up[8], a_down[8], a_compress, a_stencil, a_decompress, a_close1,
        a_close2;
    double alpha_inner = 1.05;                        // radius of the upward-equivalent / downward-check surfaces
    // FFT form of the M2L: transform size n = 2p per axis and the lattice kernel's transforms of
    // the 316 transfer vectors on the unit box, [316][n][n][n/2 + 1] (re, im)
    int fft_n = 0;
    std::vector<double> fft_ghat;
};
// Build (or fetch from the process-wide cache) the FP64 operators for (p, pinv_rtol, svd_rtol).
const HostOps *host_operators(int p, double pinv_rtol, double svd_rtol, std::string *err);
// One operator set per entry of kappa_u (the kernel's kappa times a level's half-width; 0 =
// Laplace), all with the M2L ranks of the entry that needs the largest; cached per argument list.
std::vector<const HostOps *> host_operator_levels(int p, double pinv_rtol, double svd_rtol, int kernel,
                                                  const std::vector<double> &kappa_u, std::string *err,
                                                  bool fft = false);
// Unit surface grid of order p (lexicographic), [n x 3] in [-1,1]^3.
std::vector<double> surface_grid(int p);

// ---- api.cpp ----
// Workspaces of a context for its tree (allocated once, reused while they fit; tiles rebuilt).
fmm_status ensure_workspace(fmm_ctx *ctx);
void free_workspace(fmm_ctx *ctx);

// ---- split.cu ----
// Partitioned evaluation on virtual ranks; the message of a failure goes to ctx->err.
fmm_status split_setup(fmm_ctx *ctx, int d_global, int n_ranks);
template <typename T>
fmm_status split_run(fmm_ctx *ctx, const T *q, T *phi, T *grad);
void split_free(fmm_ctx *ctx);
fmm_status split_info(fmm_ctx *ctx, int rank, fmm_rank_info *out);
fmm_status split_export(fmm_ctx *ctx, int rank, int level, int kind, uint64_t *out, int64_t *count);
fmm_status split_timings(fmm_ctx *ctx, double *ms, int n);

// ---- adaptive.cu ----
// Adaptive tree of the current uniform tree and its U, V, W and X lists; the message of a
// failure goes to ctx->err.
fmm_status adaptive_setup(fmm_ctx *ctx, int capacity);
void adaptive_free(fmm_ctx *ctx);
fmm_status adaptive_export(fmm_ctx *ctx, int kind, int64_t *offsets, int64_t *idx, int64_t *count);
fmm_status adaptive_info(fmm_ctx *ctx, int32_t *capacity, int64_t *leaves, int64_t *refined, int64_t *entries);
// Evaluation over the adaptive tree (FMM_FP32 / FMM_FP64, Laplace): workspaces, then the far
// and near fields that run_far and run_evaluate call while ctx->adaptive_eval is set.
fmm_status adaptive_prepare(fmm_ctx *ctx);
template <typename T>
cudaError_t adaptive_far(fmm_ctx *ctx, T *far_phi, T *far_grad, cudaStream_t s);
template <typename T>
cudaError_t adaptive_xli(const fmm_ctx *ctx, int level, T *D, int ld, cudaStream_t s);
template <typename T>
cudaError_t adaptive_wli(fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s);
template <typename T>
cudaError_t adaptive_uli(const fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s);

// ---- tree.cu ----
cudaError_t build_tree(fmm_ctx *ctx, const void *d_xyz);
// Class slot table: for child octant c, the 189 transfer indices (and packed deltas) of the
// V-list sources whose parent is adjacent to the target's parent.
void class_slot_table(std::vector<int> &slots, std::vector<int> &deltas);
cudaError_t export_v_lists(fmm_ctx *ctx, int level, int64_t *off, int64_t *idx, int32_t *tv,
                           int64_t *count);
cudaError_t build_tiles(fmm_ctx *ctx, int tile_m);
// fmm_debug_check: the tree's index tables against their bounds and definitions (fmm_debug_bits)
cudaError_t validate_tree(const fmm_ctx *ctx, uint32_t *flags);
// the in-kernel checks recorded by a translation unit of the FMM_DEBUG build (0 otherwise)
uint32_t debug_word_tree(bool clear);
uint32_t debug_word_p2p(bool clear);
uint32_t debug_word_output(bool clear);

// ---- kernels ----
// Point kernels (p2p.cu).  T = float or double.
template <typename T>
cudaError_t launch_gather_points(const T *q_in, const int *perm, void *pts, int64_t n,
                                 cudaStream_t s);
// phi[perm[i]] = near_phi[i] + far_phi[i] (either may be null), same for grad if non-null
template <typename T>
cudaError_t launch_scatter(const T *near_phi, const T *near_grad, const T *far_phi,
                           const T *far_grad, const int *perm, T *phi, T *grad, int64_t n,
                           cudaStream_t s, int64_t n_out = -1);   // n_out: output length (-1: n)
// the same sums into the caller's order through the inverse permutation inv (input index ->
// sorted position), written coalesced: for outputs in mapped host memory
template <typename T>
cudaError_t launch_gather_out(const T *near_phi, const T *near_grad, const T *far_phi, const T *far_grad,
                              const int *inv, T *phi, T *grad, int64_t n, cudaStream_t s);
cudaError_t launch_invert_perm(const int *perm, int64_t n, int *inv, cudaStream_t s);
// ULI near field in sorted order (phi and grad each written if non-null, one of them non-null)
template <typename T>
cudaError_t launch_p2p(const fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s);
// S2U check potentials of the boxes list[0 .. n) of one level (box b's points [begin[b], begin[b]
// + count[b]), begin and count indexed by the level's box index) into out[b x nsp]; Laplace
template <typename T>
cudaError_t launch_leaf_check_rows(const fmm_ctx *ctx, int level, const int *list, int n, const int *begin,
                                   const int *count, const T *grid, T *out, cudaStream_t s);
// D2T at the points of the boxes list[0 .. n) of one level from the densities dens[b x ldd] on
// their 2.95 surfaces (phi and grad written, not added); Laplace
template <typename T>
cudaError_t launch_leaf_eval_rows(const fmm_ctx *ctx, int level, const int *list, int n, const int *begin,
                                  const int *count, const T *grid, const T *dens, int ldd, T *phi, T *grad,
                                  cudaStream_t s);
// the FP32 ULI (Laplace) over nrows boxes of any level, box order[i] for CTA i: box r holds the
// sorted points [begin[r], begin[r] + count[r]), its U list is u_idx[u_off[r] .. u_off[r + 1])
cudaError_t launch_p2p_rows_f32(const float4 *pts, int64_t n_points, const int *begin, const int *count, const int *u_off,
                                const int *u_idx, const int *order, int nrows, float *phi, float *grad,
                                cudaStream_t s);
// check potentials on the 2.95 surface of every leaf from its own points -> rows [nleaf x nsp]
template <typename T>
cudaError_t launch_leaf_check(const fmm_ctx *ctx, const T *grid, T *out, cudaStream_t s);
// potentials (and gradients) at the points of every leaf from densities on its 2.95 surface
// shift (nullable): per-leaf constant added to the potentials (not the gradients)
template <typename T>
cudaError_t launch_leaf_eval(const fmm_ctx *ctx, const T *grid, const T *dens, int ldd, T scale,
                             T *phi, T *grad, cudaStream_t s, const double *shift);

// Helmholtz point kernels (helm.cu): complex densities (Re in pts, Im in pts_qi), complex outputs
// interleaved (re, im); the S2U rows hold [Re | Im] of the surface values, as do the D2T densities.
template <typename T>
cudaError_t launch_gather_points_c(const T *q, const int *perm, void *pts, T *qi, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_scatter_c(const T *np, const T *ng, const T *fp, const T *fg, const int *perm, T *phi, T *grad,
                             int64_t n, cudaStream_t s);
template <typename T>
cudaError_t helm_p2p(const fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s);
template <typename T>
cudaError_t helm_leaf_check(const fmm_ctx *ctx, const T *grid, T *out, cudaStream_t s);
template <typename T>
cudaError_t helm_leaf_eval(const fmm_ctx *ctx, const T *grid, const T *dens, int ldd, T *phi, T *grad, cudaStream_t s);

// Generic gathered GEMM (gemm_simt.cu / gemm_tc.cu): Y[rows] (+)= alpha sum_seg W_seg X[src(row,seg)].
enum GatherMode { GM_IDENTITY = 0, GM_CHILDREN = 1, GM_PARENT2 = 2, GM_STENCIL = 3 };
// operator ids (tensor-core operand planes); the adjoint set adds OP_COUNT
enum OpId { OP_UP = 0, OP_COMPRESS, OP_STENCIL, OP_DECOMPRESS, OP_CLOSE1, OP_CLOSE2, OP_COUNT };
struct GemmCall {
    int mode = GM_IDENTITY;
    int level = 0;               // level of the output rows
    int accumulate = 0;          // Y += ... instead of Y = ...
    int n_out = 0;               // padded N (columns of Y, rows of W)
    double alpha = 1.0;
    // segment 0 (and the only one for IDENTITY / STENCIL); CHILDREN uses W0 + c * w_stride,
    // STENCIL uses W0 + t * w_stride
    const void *X0 = nullptr; int ldx0 = 0; int k0 = 0;   // input rows, padded K
    const void *W0 = nullptr; int64_t w_stride = 0;
    // segment 1 (PARENT2 only): X1 rows of the parent level, W chosen by child octant class
    const void *X1 = nullptr; int ldx1 = 0; int k1 = 0;
    void *const *W1_by_cls = nullptr;                     // array of 8 device pointers
    void *Y = nullptr; int ldy = 0;
    const int *dense = nullptr;  // GM_STENCIL: source lookup table in place of the level's own
    // a subset of the level's boxes in place of all of them (SIMT form): the tiles, and the box
    // index of every tile row (tile.row0 + r indexes `rows`; class-ordered for STENCIL / PARENT2)
    const TileSet *tiles = nullptr;
    const int *rows = nullptr;
    // tensor-core only: A rows read from split planes through TMA row gathers (segment 0), and/or
    // the output written as split planes instead of FP32 Y.  Plane p of row r, column k is at
    // byte (r * ld + k) * esize + p * plane within the buffer (esize 2 for BF16, 4 for TF32).
    const void *Xp = nullptr; int xp_ld = 0; int xp_rows = 0; long long xp_plane = 0;
    void *Yp = nullptr; int yp_ld = 0; long long yp_plane = 0;
    // FP16 split planes (FMM_FP16X3): 1 / scale per row and 64-column chunk of Xp / Yp
    const float *xp_scale = nullptr; int xp_scale_ld = 0;
    float *yp_scale = nullptr; int yp_scale_ld = 0;
    // PARENT2 segment 1 from split planes (FMM_FP16X3): the parent rows
    const void *Xp1 = nullptr; int xp1_ld = 0; long long xp1_plane = 0;
    const float *xp1_scale = nullptr; int xp1_scale_ld = 0;
};
template <typename T>
cudaError_t gemm_simt(const fmm_ctx *ctx, const GemmCall &g, cudaStream_t s);
cudaError_t gemm_tc(const fmm_ctx *ctx, const GemmCall &g, int op_id, cudaStream_t s);
// FP32 rows (nrows x ncols, stride ldx) -> FP16 hi/lo planes (stride ldp, planes plane_bytes
// apart) and 1 / scale per row and 64-column chunk (stride lds), as FMM_FP16X3 contractions read
cudaError_t launch_rows_to_planes(const float *x, int ldx, int64_t nrows, int ncols, void *planes,
                                  long long plane_bytes, int ldp, float *scales, int lds, cudaStream_t s);
cudaError_t tc_upload_operators(fmm_ctx *ctx);
void tc_free(fmm_ctx *ctx);

// ---- fft.cu ----
cudaError_t fft_upload(fmm_ctx *ctx);
template <typename T>
cudaError_t fft_vli(fmm_ctx *ctx, int level, const T *U, T *D, cudaStream_t s);

// ---- evaluate.cu ----
cudaError_t upload_operators(fmm_ctx *ctx);
template <typename T>
cudaError_t run_far(fmm_ctx *ctx, bool adjoint, T *far_phi, T *far_grad, cudaStream_t s);
// The far-field steps of one context, each on the given stream (run_far orders them for a whole
// tree; the partitioned evaluation orders them across rank contexts).
template <typename T>
struct FarSteps {
    fmm_ctx *ctx;
    bool adjoint;
    int d = 0, nsp = 0, kw = 0, nck_s = 0, nck_k = 0;
    bool f16 = false;
    void *A = nullptr, *B = nullptr;   // upward- and downward-side rows of this direction
    FarSteps(fmm_ctx *c, bool adj);
    cudaError_t leaf_in(cudaStream_t s);                 // S2U (+ leaf planes)
    cudaError_t up(int l, cudaStream_t s);               // U2U into level l
    cudaError_t compress(int l, cudaStream_t s);         // VLI compress of level l
    cudaError_t stencil(int l, cudaStream_t s);          // VLI stencil of level l
    cudaError_t down(int l, cudaStream_t s);             // decompress + D2D into level l
    cudaError_t leaf_out(T *far_phi, T *far_grad, cudaStream_t s);   // closing + D2T
    size_t base(int l) const { return (size_t)ctx->lev[l].row_base; }
    const OpSet &O(int l) const;
    unsigned char *upP(int l) const;
    unsigned char *dnP(int l) const;
    unsigned char *ctP(int l) const;
    unsigned char *utP(int l) const;
    float *upS(int l) const;
    float *dnS(int l) const;
    float *ctS(int l) const;
    float *utS(int l) const;
};

}  // namespace fmm
