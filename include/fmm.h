/*
 * fmm.h - C ABI of libfmm: a kernel-independent fast multipole method (kiFMM) for the 3D
 * Laplace kernel K(x, y) = 1 / (4 pi |x - y|) over a Morton-keyed uniform octree, evaluated on
 * one NVIDIA GB300 (sm_103a).  The same steps also run with the modified Helmholtz (Yukawa)
 * kernel K(x, y) = exp(-kappa |x - y|) / (4 pi |x - y|) (option `kernel`), a second real kernel
 * of Eq. 1 that the kernel-independent method of Section 2.1 takes without change.
 *
 * What is computed (the paper's problem statement, Section 1, Eq. 1 with the kernel of Eq. 2
 * normalised by 4 pi): for N points x_i that are both sources and targets, given in arbitrary
 * order (Section 2.3), and densities s_j,
 *     phi_i = sum_{j != i} K(x_i, x_j) s_j,   grad_i = grad_x phi(x_i),
 * approximated by Algorithm 1 (uniform branches: S2U, U2U, VLI, D2D, D2T, ULI).  A built tree
 * can be re-used with new densities (Section 3.1, step 6).
 *
 * Calling conventions shared by every entry point:
 *  - Status codes only; nothing throws across the ABI.  After an error, fmm_last_error(ctx)
 *    returns a message; the context stays usable unless the status is FMM_ECUDA.
 *  - All GPU work is ordered on the CUDA stream given to fmm_create (NULL = legacy default).
 *  - Array arguments may be device pointers or host pointers (pageable or pinned); the library
 *    detects which with cudaPointerGetAttributes.  With device pointers a call returns as soon
 *    as its work is enqueued; with host pointers it copies through library-owned device
 *    buffers and returns after the results are back in host memory.  Outputs of an evaluation
 *    (fmm_evaluate, fmm_evaluate_parts, fmm_adjoint's psi, fmm_adaptive_evaluate; real
 *    kernels) that are all in pinned host memory are written there directly by a kernel, in the
 *    caller's order, with no staging buffer.
 *  - Floating-point arrays are float (4 bytes) unless the context's precision is FMM_FP64,
 *    in which case they are double.  Coordinates are N x 3 row-major (x0 y0 z0 x1 y1 z1 ...).
 *  - The caller owns every array it passes; the library keeps no caller pointer after a call
 *    returns.  The library owns the tree, the operators and all workspaces (allocated with
 *    cudaMalloc by fmm_build_tree and fmm_precompute, released by fmm_destroy).
 *  - One context must not be used by two host threads at the same time.
 */
#ifndef FMM_H
#define FMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx fmm_ctx;

typedef enum {
    FMM_OK = 0,
    FMM_EINVAL = 1,        /* bad argument (null pointer, size, option out of range, NaN input) */
    FMM_ENOMEM = 2,        /* a device or host allocation failed */
    FMM_ECUDA = 3,         /* a CUDA call or kernel failed; the context should be destroyed */
    FMM_ESTATE = 4,        /* call out of order (e.g. evaluate before build_tree/precompute) */
    FMM_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    FMM_EUNSUPPORTED = 6   /* option combination not available in this library */
} fmm_status;

/* Arithmetic of the surface contractions (U2U, VLI, D2D and the check-to-equivalent steps).
 * The near field (ULI), the S2U check potentials and D2T always run in FP32 SIMT arithmetic,
 * except under FMM_FP64 where everything is FP64. */
typedef enum {
    FMM_FP32 = 0,          /* FP32 SIMT everywhere */
    FMM_FP64 = 1,          /* FP64 SIMT everywhere; inputs and outputs are double */
    FMM_TF32X3 = 2,        /* contractions on tcgen05 tensor cores, 3 TF32 products (big/small split) */
    FMM_BF16X3 = 3,        /* contractions on tcgen05 tensor cores, 3 BF16 products (hi/lo split) */
    FMM_BF16X6 = 4,        /* contractions on tcgen05 tensor cores, 6 BF16 products (hi/mid/lo split) */
    FMM_FP16X3 = 5         /* contractions on tcgen05 tensor cores from FP16 hi/lo splits of power-of-two
                              scaled operands (every box row scaled per box and 64-column chunk by the
                              step that writes it, the operators per chunk), 3 FP16 products, about
                              2^-22 relative per term, scales applied in FP32.  The leaf closing (the
                              pseudo-inverse of the downward check potentials) stays in FP32 SIMT, as
                              in every tensor-core mode.  No mean_free (FMM_EUNSUPPORTED). */
} fmm_precision;

/* Kernel of Eq. 1 (option `kernel`). */
typedef enum {
    FMM_LAPLACE = 0,       /* 1 / (4 pi r) (Eq. 2, normalised by 4 pi) */
    FMM_YUKAWA = 1,        /* exp(-kappa r) / (4 pi r), kappa > 0; gradient -(1 + kappa r) exp(-kappa r) d / (4 pi r^3) */
    FMM_HELMHOLTZ = 2      /* exp(i k r) / (4 pi r), wavenumber k = `kappa` > 0 (Eq. 1 with F = C); gradient
                              (i k r - 1) exp(i k r) d / (4 pi r^3).  Densities and outputs are complex,
                              stored interleaved (re, im): q and phi hold 2n values, grad 6n
                              (d/dx re, d/dx im, d/dy re, ... per point).  Box vectors hold the real
                              and imaginary parts of the surface values (2 (6(p-1)^2+2) entries). */
} fmm_kernel;

typedef struct {
    int order_p;           /* expansion order p >= 2; each box vector has 6(p-1)^2+2 entries
                              (Section 4, global portion).  Supported: 2..10. */
    int depth;             /* uniform tree depth d, 0..10 (level 0 = root, d = leaves; Section 2.1) */
    int precision;         /* an fmm_precision value */
    double svd_rtol;       /* M2L operator compression: keep singular values >= svd_rtol * sigma_1 */
    double pinv_rtol;      /* check-to-equivalent pseudo-inverse cutoff relative to sigma_1 */
    int with_gradient;     /* nonzero: fmm_evaluate may be asked for gradients */
    int has_domain;        /* nonzero: use origin/side below as the bounding cube */
    double origin[3];      /* bounding cube corner (has_domain) */
    double side;           /* bounding cube side > 0 (has_domain) */
    int mean_free;         /* nonzero: keep each box's downward check potential without its mean,
                              carrying the means down the tree in FP64 and adding them to the leaf
                              potentials only.  The stored values then have the size of the field's
                              variation across a box instead of the potential itself, so FP32 or
                              split-precision rounding no longer grows into gradient error as the
                              boxes shrink (deep trees).  It treats a constant potential as exactly
                              constant, where the textbook operators reproduce it only up to their
                              fit error, so results differ from the textbook kiFMM by about that
                              error (1e-7 relative at p >= 6, 1e-4 at p = 4).  Default 0. */
    int kernel;            /* an fmm_kernel value.  Default FMM_LAPLACE.  FMM_YUKAWA and FMM_HELMHOLTZ need
                              has_domain: these kernels are not homogeneous, so their operators depend
                              on the physical box sizes and are built per level by fmm_precompute from
                              `side` (fmm_create returns FMM_EUNSUPPORTED without a domain, and with
                              mean_free, whose constant-potential argument holds for Laplace only).
                              FMM_HELMHOLTZ has no fmm_adjoint and no partitioned evaluation
                              (FMM_EUNSUPPORTED). */
    double kappa;          /* FMM_YUKAWA: screening constant; FMM_HELMHOLTZ: wavenumber; finite and > 0,
                              in inverse units of the coordinates.  Ignored for FMM_LAPLACE. */
    int m2l;               /* an fmm_m2l_form value.  Default FMM_M2L_DENSE. */
} fmm_options;

/* Form of the M2L (VLI) translation (option `m2l`; Section 2.2 names both). */
typedef enum {
    FMM_M2L_DENSE = 0,     /* SVD-compressed operators applied as batched contractions (BLAS form) */
    FMM_M2L_FFT = 1        /* lattice convolution by FFT: the upward-equivalent and downward-check
                              surfaces on radius (p-1)/(p-2) half-widths, whose grid spacing divides
                              the box width; each box's equivalent densities are transformed once
                              (n = 2p points per axis, zero-padded), the products with the kernel's
                              transforms summed over the V list, and the sum transformed back at the
                              check surface.  FMM_FP32 / FMM_FP64 and FMM_LAPLACE with p >= 4 only;
                              no mean_free, fmm_adjoint, partitioned or adaptive evaluation
                              (FMM_EUNSUPPORTED). */
} fmm_m2l_form;

/* Part selectors for fmm_evaluate_parts (Section 1, Eq. 3: near field + far field). */
#define FMM_PART_NEAR 1    /* ULI: direct sums over the U lists */
#define FMM_PART_FAR 2     /* S2U, U2U, VLI, D2D, D2T */
#define FMM_PART_ALL 3

/* Tree and operator sizes, filled by fmm_get_tree_info. */
typedef struct {
    int64_t n_points;
    int32_t depth;
    int32_t n_surface;         /* 6(p-1)^2+2 surface points (a box vector holds twice that under FMM_HELMHOLTZ) */
    int32_t m2l_rank_in;       /* rank of the compressed M2L on the source side (0 before precompute) */
    int32_t m2l_rank_out;      /* rank on the target side (0 before precompute) */
    int64_t n_boxes[11];       /* non-empty boxes per level 0..depth */
    int64_t n_u_entries;       /* total length of all U lists */
    int64_t p2p_pairs;         /* sum over leaves of |leaf| * sum_{a in U(leaf)} |a| */
    double origin[3];          /* the bounding cube actually used */
    double side;
} fmm_tree_info;

/* Fill *opt with defaults: p = 6, depth = 4, FMM_FP32, svd_rtol = 1e-6, pinv_rtol = 1e-7,
 * with_gradient = 1, no domain (the cube is taken from the points). */
fmm_status fmm_default_options(fmm_options *opt);

/* Create a context bound to the current CUDA device and `cuda_stream` (a cudaStream_t, may be
 * NULL).  Validates the options (EINVAL) and allocates nothing on the device. */
fmm_status fmm_create(const fmm_options *opt, void *cuda_stream, fmm_ctx **out);

/* Build the octree over n points (Section 2.1): Morton keys at depth d, a stable radix sort,
 * leaf ranges, per-level box tables and the U lists; V lists are stencil lookups (Section 2.2).
 * xyz: n x 3 coordinates (float, or double under FMM_FP64), host or device.
 * Errors: EINVAL for n <= 0, n > 2^31 - 1 or a non-finite coordinate; ENOMEM. */
fmm_status fmm_build_tree(fmm_ctx *ctx, const void *xyz, int64_t n);

/* Host FP64 precompute of every operator (check-to-equivalent pseudo-inverses, U2U, D2D,
 * the 316 M2L operators and their SVD compression) and upload in the context's precision.
 * Independent of the points; may be called before or after fmm_build_tree.  Laplace: one set for
 * every level (homogeneity); FMM_YUKAWA and FMM_HELMHOLTZ: one set per level from the domain's box
 * sizes, all with the M2L ranks of the level that needs the largest.  Cached per process. */
fmm_status fmm_precompute(fmm_ctx *ctx);

/* phi = A q (Algorithm 1), and grad phi if `grad` is non-NULL (requires with_gradient).
 * q: n densities; phi: n outputs; grad: n x 3 outputs; all in the input order of the points
 * (FMM_HELMHOLTZ: complex values, interleaved re, im: 2n, 2n and 6n numbers).
 * phi may be NULL when grad is not: the gradient-only ("force") evaluation of N-body codes, which
 * skips the potential sums of the near field and the potential outputs; its gradients are those
 * of the full evaluation bit for bit.
 * Errors: ESTATE before fmm_build_tree and fmm_precompute; EINVAL for null q, for phi and grad
 * both NULL, and for grad with with_gradient = 0. */
fmm_status fmm_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad);

/* As fmm_evaluate, restricted to the parts in `parts` (FMM_PART_NEAR | FMM_PART_FAR). */
fmm_status fmm_evaluate_parts(fmm_ctx *ctx, const void *q, void *phi, void *grad, int parts);

/* psi = A^T g: the transpose of the map q -> phi computed by fmm_evaluate (the FMM is not
 * exactly symmetric), by running every step of Algorithm 1 transposed in reverse order.
 * If grad_psi is non-NULL it receives grad phi_g(x_i), the gradient of the potential generated
 * by densities g (a forward pass); with it, d/dx_k of a loss L(phi) is
 * g_k grad phi_q(x_k) + q_k grad phi_g(x_k) with g = dL/dphi and the tree held fixed.
 * Same argument rules and errors as fmm_evaluate. */
fmm_status fmm_adjoint(fmm_ctx *ctx, const void *g, void *psi, void *grad_psi);

/* ---- Partitioned evaluation on virtual ranks (Section 3: Box comm-setup, Box comm-runtime) ----
 *
 * The tree is split at depth d_global: its level-d_global boxes are the local roots, each the
 * root of a local tree.  n_ranks virtual ranks on this GPU each own a contiguous Morton run of
 * local roots (the layout, balanced by point counts) and hold their own buffers: their points,
 * the rows of their local trees, and receive rows for the ghost boxes of their local essential
 * tree (Eq. 3).  Setup forms each rank's U and V query packets from the layout, the owners'
 * existence answers, the neighbourhoods and the ghost points' coordinates.  An evaluation runs
 * the local upward stage of every rank, the exchanges (U: ghost densities; V: the ghosts'
 * compressed upward rows), the gather of the local roots' upward rows into a nominated global
 * context, the global upward and downward passes over levels 2..d_global there, the scatter of
 * the local roots' downward rows, and the local downward stage with the ULI.  Every output is
 * computed by the same kernels from the same values in the same order as by fmm_evaluate, so the
 * two agree bit for bit.  Exchanges are device copies between the ranks' buffers.
 */
typedef enum {
    FMM_PARTITION_OWN = 0,           /* keys of the rank's own boxes at `level` (d_global..depth) */
    FMM_PARTITION_GHOST_V = 1,       /* keys of its V-list ghost boxes at `level` (d_global+1..depth) */
    FMM_PARTITION_GHOST_U = 2,       /* keys of its U-list ghost leaves (level ignored) */
    FMM_PARTITION_NEIGHBOURS_U = 3,  /* ranks its U query packets address, ascending (level ignored) */
    FMM_PARTITION_NEIGHBOURS_V = 4,  /* ranks its V query packets address, ascending (level ignored) */
    FMM_PARTITION_LAYOUT = 5         /* per local root in Morton order: key | (owner rank << 32)
                                        (rank and level ignored) */
} fmm_partition_export_kind;

typedef struct {
    int32_t rank, n_ranks, d_global;
    int32_t n_local_roots;         /* local roots owned */
    int64_t first_root;            /* index of its first local root among the level-d_global boxes */
    int64_t first_point;           /* its points are sorted positions first_point .. + n_points - 1 */
    int64_t n_points;
    int64_t n_boxes[11];           /* own boxes per level (levels d_global..depth; 0 above) */
    int64_t n_ghost_v[11];         /* V-list ghost boxes per level (levels d_global+1..depth) */
    int64_t n_ghost_u;             /* U-list ghost leaves */
    int64_t n_ghost_points;        /* their points */
    int64_t n_query_u, n_query_v;  /* keys in its U and V query packets (before the existence answers) */
    int32_t n_neighbours_u, n_neighbours_v;   /* ranks its U and V packets address */
    int64_t bytes_u;               /* received per evaluation: densities of the ghost points */
    int64_t bytes_v;               /* received per evaluation: the V ghosts' compressed upward rows */
    int64_t bytes_gather;          /* sent per evaluation: its local roots' upward rows */
    int64_t bytes_scatter;         /* received per evaluation: its local roots' downward rows */
} fmm_rank_info;

/* Build the partition: 2 <= d_global < depth, 1 <= n_ranks <= the number of local roots.
 * Needs fmm_build_tree and fmm_precompute; a new fmm_build_tree drops the partition.
 * Errors: ESTATE, EINVAL (ranges), EUNSUPPORTED (mean_free, FMM_HELMHOLTZ), ENOMEM, ECUDA. */
fmm_status fmm_partition_setup(fmm_ctx *ctx, int d_global, int n_ranks);

/* fmm_evaluate through the partition (same arguments and output rules; phi may be NULL when grad
 * is not).  ESTATE before fmm_partition_setup. */
fmm_status fmm_partition_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad);

/* Sizes, neighbourhoods and exchange volumes of one rank.  ESTATE before fmm_partition_setup;
 * EINVAL for a rank out of range. */
fmm_status fmm_partition_info(fmm_ctx *ctx, int rank, fmm_rank_info *info);

/* Export one list of a rank (an fmm_partition_export_kind) into out[*count]; with out == NULL
 * only *count is set.  EINVAL for a bad rank, level or kind. */
fmm_status fmm_partition_export(fmm_ctx *ctx, int rank, int level, int kind, uint64_t *out, int64_t *count);

/* Device times (ms) of the last partitioned evaluation, up to n of: densities and U exchange,
 * local upward stage, V exchange, gather, global stage, scatter, local downward stage, the part
 * of the ULI still running after it (the ULI runs beside all the stages from the local upward
 * one on), output, total.  Waits for that evaluation.
 *
 * Concurrency: the ranks' chains of launches run on a pool of far-field streams and their ULI
 * on near-field streams of lower priority; each output mode's evaluation is captured once as a
 * CUDA graph (densities read from, and outputs written to, buffers of the partition, with one
 * device copy in and out per call) and replayed. */
fmm_status fmm_partition_timings(fmm_ctx *ctx, double *ms, int n);

/* ---- Adaptive tree and its interaction lists (Section 2.1: adaptive refinement; Table 1 and
 * Algorithm 1: the U, V, W and X lists of the adaptive branches) ----
 *
 * Built on the device from the uniform tree of fmm_build_tree (its depth D is the deepest level
 * allowed).  The adaptive tree keeps the root and the children of every kept box of level < D
 * that holds more than `capacity` points; a kept box that is not refined is a leaf.
 *   U(b), leaf b:      kept leaves adjacent to b (sharing a vertex, edge or face), b included;
 *   V(b), level >= 2:  kept boxes of b's level whose parents are adjacent to b's parent and that
 *                      are not adjacent to b;
 *   W(b), leaf b:      kept boxes below b's colleagues that are not adjacent to b while their
 *                      parents are;
 *   X(b):              the leaves whose W list holds b.
 * Boxes are named by their row: the boxes of the uniform tree, level by level from the root,
 * ascending Morton key within a level (fmm_export_level gives each level's keys); rows of boxes
 * that the adaptive tree does not keep have empty lists.  Every list is sorted by row. */
typedef enum {
    FMM_ADAPTIVE_STATE = 0,   /* per row: 0 not kept, 1 leaf, 2 refined */
    FMM_ADAPTIVE_COUNT = 1,   /* per row: points in the box */
    FMM_ADAPTIVE_U = 2,       /* U lists (CSR over rows) */
    FMM_ADAPTIVE_V = 3,       /* V lists */
    FMM_ADAPTIVE_W = 4,       /* W lists */
    FMM_ADAPTIVE_X = 5        /* X lists */
} fmm_adaptive_export_kind;

typedef struct {
    int32_t capacity;
    int64_t n_rows;            /* boxes of the uniform tree over all levels (the row space) */
    int64_t n_leaves[11];      /* leaves of the adaptive tree per level 0..depth */
    int64_t n_refined[11];     /* refined boxes of the adaptive tree per level */
    int64_t n_entries[4];      /* total lengths of the U, V, W and X lists */
} fmm_adaptive_tree_info;

/* Refine by `capacity` (>= 0) and build the four lists; replaces an earlier adaptive tree of this
 * context.  It belongs to the current tree: fmm_build_tree discards it.
 * Errors: ESTATE before fmm_build_tree; EINVAL for capacity < 0; ECUDA, ENOMEM. */
fmm_status fmm_adaptive_setup(fmm_ctx *ctx, int capacity);

/* Summary counts of the adaptive tree.  ESTATE before fmm_adaptive_setup. */
fmm_status fmm_adaptive_info(fmm_ctx *ctx, fmm_adaptive_tree_info *info);

/* Copy one fmm_adaptive_export_kind to host arrays (any pointer may be NULL to skip it):
 *  count[0] = rows, count[1] = entries (rows for STATE and COUNT, the list length otherwise);
 *  offsets[rows + 1]: the CSR offsets (lists only); idx[entries]: the per-row values or the
 *  members (rows).  ESTATE before fmm_adaptive_setup; EINVAL for an unknown kind. */
fmm_status fmm_adaptive_export(fmm_ctx *ctx, int kind, int64_t *offsets, int64_t *idx, int64_t *count);

/* phi = A q over the adaptive tree (Algorithm 1 with its adaptive branches), and grad phi if `grad`
 * is non-NULL; arguments, layouts and the gradient-only form (phi == NULL) as fmm_evaluate, with
 * `parts` as fmm_evaluate_parts: FMM_PART_NEAR is the ULI over the adaptive U lists, FMM_PART_FAR
 * the rest:
 *   S2U and U2U   as the uniform tree's (the check potentials of a leaf above the deepest level
 *                 come from its descendants' by U2U, which represents the same sources);
 *   VLI           over the adaptive V lists (kept boxes only);
 *   XLI (2b)      the sources of X(b) added to b's downward check potentials before D2D;
 *   D2D           down to the deepest level: the boxes below a leaf of the adaptive tree take no
 *                 VLI of their own and carry the leaf's local field to its points by D2D alone;
 *   D2T           at the deepest level;
 *   WLI (3a)      the upward equivalent densities of W(b), r (V S^-1)(U^T u) of the upward
 *                 check potentials, evaluated at the points of leaf b.
 * Requires fmm_adaptive_setup on the current tree and fmm_precompute.  FMM_FP32 and FMM_FP64 with
 * the Laplace kernel only (EUNSUPPORTED for the tensor-core precisions, the other kernels and
 * mean_free).  Errors otherwise as fmm_evaluate_parts. */
fmm_status fmm_adaptive_evaluate(fmm_ctx *ctx, const void *q, void *phi, void *grad, int parts);

/* Sizes of the built tree and operators.  ESTATE before fmm_build_tree. */
fmm_status fmm_get_tree_info(const fmm_ctx *ctx, fmm_tree_info *info);

/* Copy the tree to host arrays (any pointer may be NULL to skip it):
 *  perm[n]                  sorted position -> input index (stable sort by leaf key)
 *  leaf_keys[n_leaf]        Morton keys of the non-empty leaves, ascending
 *  leaf_offsets[n_leaf+1]   points of leaf b are sorted positions leaf_offsets[b] .. [b+1]-1
 *  u_offsets[n_leaf+1], u_idx[n_u_entries]  U lists (CSR), leaf indices ascending
 * Morton keys interleave x, y, z bits with x most significant in every triple. */
fmm_status fmm_export_tree(fmm_ctx *ctx, int64_t *perm, uint64_t *leaf_keys,
                           int64_t *leaf_offsets, int64_t *u_offsets, int64_t *u_idx);

/* Copy one level's boxes and V lists to host arrays (pointers may be NULL):
 *  keys[n_boxes[level]]     ascending Morton keys of the level's non-empty boxes
 *  v_offsets[n+1], v_idx[], v_tvec[]   V lists (CSR) for level >= 2, box indices ascending;
 *  v_tvec holds the transfer-vector index t in [0, 316): (source - target) in box units, in
 *  the enumeration of [-3,3]^3 minus [-1,1]^3 with x slowest and z fastest.
 * *n_v_entries receives the total V length (call once with v_idx = NULL to size the arrays).
 * The V lists are built on the device for this call and freed before it returns. */
fmm_status fmm_export_level(fmm_ctx *ctx, int level, uint64_t *keys, int64_t *v_offsets,
                            int64_t *v_idx, int32_t *v_tvec, int64_t *n_v_entries);

/* Copy the check potentials of the last fmm_evaluate (with its far field) at `level` in [2, d]
 * to host memory: n_boxes[level] x n_surface values, row-major, float or double (FMM_HELMHOLTZ:
 * n_boxes[level] x 2 n_surface, each row the real parts then the imaginary parts).
 *  kind 0 (upward): row b approximates sum_{j in b} K(x^{uc}_b, x_j) s_j, the potential of the
 *          sources inside box b on its upward check surface (exact at the leaf level);
 *  kind 1 (downward): row b approximates the potential on b's downward check surface of the
 *          sources outside b's colleagues and b itself (its far field, Section 1 Eq. 3).
 * The surfaces: centre c_b + alpha r_b g, g the order-p grid on the boundary of [-1,1]^3 in
 * lexicographic order, alpha = 2.95 (upward check) or 1.05 (downward check), r_b the half-width.
 * Errors: ESTATE without such an evaluation; EINVAL for a bad level or kind. */
fmm_status fmm_export_check(fmm_ctx *ctx, int level, int kind, void *host_out);

/* Milliseconds spent in each phase of the last fmm_evaluate or fmm_adjoint, measured with CUDA
 * events: [0] near field (the ULI kernel, on the side stream it runs on), [1] upward pass (S2U
 * and U2U), [2] VLI (M2L compress and stencil products of all levels, with the downward steps
 * of the levels above the leaves that overlap them), [3] the leaf level's downward step and
 * D2T, [4] whole call.  [1] to [3] are consecutive on the far-field stream; the near field runs
 * concurrently with them at a lower stream priority, so [0] + [1] + [2] + [3] may exceed [4].
 * n <= 5 values are written. */
fmm_status fmm_last_timings(fmm_ctx *ctx, double *ms, int n);

/* Wait for all work of ctx and report device-side failures since the last fmm_sync:
 * FMM_ETIMEOUT if a tensor-core kernel's bounded wait on a shared-memory barrier expired (the
 * kernel then skipped its remaining work, so the outputs of those calls are invalid); FMM_ECUDA
 * for a CUDA error.  Calls with host pointers already synchronize but do not read the flag. */
fmm_status fmm_sync(fmm_ctx *ctx);

/* Failure injection for tests and deployment checks (no counterpart in the paper).
 *
 * fmm_set_wait_limit: the bound on every barrier wait of ctx's tensor-core kernels (default 1 s;
 * seconds in [0, 60], else EINVAL).  A wait that exceeds it makes the kernel record FMM_ETIMEOUT,
 * stop issuing copies and MMAs, wait for the copies and MMAs it already issued, free its tensor
 * memory and return; fmm_sync then reports FMM_ETIMEOUT and the outputs of that call are
 * invalid.  0 gives up at the first wait that does not complete at once, which forces the
 * failure path; the context stays usable and later calls with a normal limit are correct.
 *
 * fmm_set_alloc_limit: process-wide cap on any single device allocation the library makes
 * (SIZE_MAX, the default, is no cap).  A larger request fails as out of memory: the call that
 * needed it returns FMM_ENOMEM (fmm_build_tree leaves the context without a tree, fmm_precompute
 * without operators) and frees what it had allocated, so the same call succeeds once the cap is
 * lifted. */
fmm_status fmm_set_wait_limit(fmm_ctx *ctx, double seconds);
void fmm_set_alloc_limit(size_t bytes);

/* Consistency checks in place of a memory checker (no counterpart in the paper).
 *
 * fmm_debug_check validates every index table of ctx's tree on the device against its bounds
 * and its definition: the sort permutation, the leaf offsets (increasing from 0 to n), the U
 * lists (in range, ascending, adjacent, the leaf itself included), every level's keys, dense
 * table, parent and child indices and class order, and the near-field schedule.  The library
 * also exists as libfmm_debug.so, built with FMM_DEBUG: there the kernels that compute indices
 * (the radix scatter, the near-field and leaf kernels' point ranges, the output scatter) check
 * each one before using it and, instead of trapping, skip the access and record the check; this
 * call then also returns the checks recorded since its last call, and clears them.
 * *flags (not NULL) receives the OR of the fmm_debug_bits that failed, 0 if none; *in_kernel (may
 * be NULL) is set to 1 in libfmm_debug.so, else 0.  ESTATE before fmm_build_tree; ECUDA for a
 * CUDA error.  It synchronizes ctx's stream. */
typedef enum {
    FMM_DEBUG_PERM = 1 << 0,     /* sort permutation */
    FMM_DEBUG_LEAF = 1 << 1,     /* leaf offsets */
    FMM_DEBUG_ULIST = 1 << 2,    /* U lists */
    FMM_DEBUG_KEYS = 1 << 3,     /* level keys and dense tables */
    FMM_DEBUG_TREE = 1 << 4,     /* parent and child indices */
    FMM_DEBUG_CLASS = 1 << 5,    /* class (octant) order of a level */
    FMM_DEBUG_ORDER = 1 << 6,    /* near-field schedule */
    FMM_DEBUG_P2P = 1 << 7,      /* in-kernel: a point range outside the points */
    FMM_DEBUG_SCATTER = 1 << 8,  /* in-kernel: an output position outside [0, n) */
    FMM_DEBUG_SORT = 1 << 9      /* in-kernel: a radix scatter position outside [0, n) */
} fmm_debug_bits;
fmm_status fmm_debug_check(fmm_ctx *ctx, uint32_t *flags, int32_t *in_kernel);

/* Morton keys and stable sort of n points, allocating nothing.  The paper has no counterpart:
 * this entry point is for callers that cannot let a library allocate device memory, because
 * one allocator owns all of their device memory or because they reserve their whole budget at
 * start-up.  It performs the first step of fmm_build_tree (the leaf key of every point at
 * `depth` in the cube [origin, origin + side)^3, computed as fmm_build_tree does, and a stable
 * sort by key) on caller-owned device arrays:
 *   xyz[n x 3]  float coordinates (device);  perm[n]  receives the input index of each sorted
 *   position;  keys[n]  receives the sorted Morton keys (x bit most significant per triple).
 * Its scratch is a file-scope device array of 8,651,012 bytes (every GPU that loads the library
 * holds it until the process exits), so n is limited to 1,048,576: larger n, n <= 0, a
 * depth outside 0..10, a non-positive side or a non-finite origin return FMM_EINVAL.
 * A non-finite coordinate also returns FMM_EINVAL, as in fmm_build_tree; perm and keys are
 * then written but meaningless.
 * The first call on a device (and the first after a device reset) looks up the array's device
 * address (cudaGetSymbolAddress), so make that first call before any stream capture.  Every
 * call shares the array: calls that overlap on the GPU (different streams, or different threads
 * on one device) race and must be serialised by the caller.  Work is enqueued on `cuda_stream`,
 * and the call waits for that stream once at the end to read the non-finite flag back.
 * FMM_ECUDA reports a CUDA failure. */
fmm_status fmm_sort_points_noalloc(const float *xyz, int64_t n, int depth, const double origin[3],
                                   double side, int32_t *perm, uint32_t *keys, void *cuda_stream);

/* Number of CUDA kernels this library has launched in the process so far (all contexts). */
long long fmm_kernel_launches(void);

/* Measurement utility (no counterpart in the paper): the FP32 fused multiply-add throughput of
 * the current device in TFLOP/s (2 flops per FMA), as scalar FP32 (*tflops_scalar) and in the
 * two-wide float2 form (*tflops_pair), each from the second of two launches of `iters`
 * iterations of 8 independent FMA chains per thread on 8 x 256 threads per SM.  It is the
 * measured denominator of the near-field roofline and depends on the clock at the time.
 * Synchronous; uses its own stream.  EINVAL for iters <= 0 or a null output; ECUDA on a CUDA
 * failure. */
fmm_status fmm_measure_fp32_peak(int iters, double *tflops_scalar, double *tflops_pair);

/* Message for the last failed call on ctx ("" if none).  Never NULL. */
const char *fmm_last_error(const fmm_ctx *ctx);

/* Release every device and host resource of ctx (waits for its stream).  NULL is allowed. */
void fmm_destroy(fmm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H */
