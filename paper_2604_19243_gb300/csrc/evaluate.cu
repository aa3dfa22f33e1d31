// Evaluation pipeline (Algorithm 1, uniform branches) and its transpose.
//
// Forward, with boxes holding check potentials (fmm_internal.h):
//   S2U   U_d  = K(uc, y) s                          leaf check kernel
//   U2U   U_l  = sum_c A_c U_{l+1}[child_c]          l = d-1 .. 2 (levels 0-1 take no part)
//   VLI   Ut_l = Vi^T U_l ; Ct_l[b] = sum_t C_t Ut_l[b + t] ; D_l = Uo Ct_l   l = 2 .. d
//   D2D   D_l += B_c D_{l-1}[parent]                 fused with the VLI decompress, l >= 3
//   D2T   d = r_d (V S^-1)(U^T D_d) ; f = K(x, de) d
//   ULI   f += near-field sums                       independent of the rest (Section 2.2)
// Adjoint (psi = A^T g): the same sequence with every operator transposed and the roles of the
// upward and downward arrays exchanged: D2T^T is the leaf check kernel on the 2.95 surface,
// the closing pseudo-inverse is applied transposed, D2D^T gathers children like U2U, the VLI
// runs with C_{-t}^T, U2U^T gathers the parent like D2D and S2U^T evaluates the 2.95 surface
// at the points like D2T.  ULI is symmetric.
#include <algorithm>
#include <cmath>
#include <vector>

#include "devutil.cuh"
#include "gemm_common.cuh"

namespace fmm {

GemmDev make_gemm_dev(const fmm_ctx *ctx, const GemmCall &c) {
    GemmDev g{};
    g.mode = c.mode;
    g.accumulate = c.accumulate;
    g.n_out = c.n_out;
    g.level = c.level;
    g.alpha = (float)c.alpha;
    g.alpha_d = c.alpha;
    g.X0 = c.X0, g.ldx0 = c.ldx0, g.k0 = c.k0;
    g.W0 = c.W0, g.w_stride = c.w_stride;
    g.X1 = c.X1, g.ldx1 = c.ldx1, g.k1 = c.k1;
    for (int i = 0; i < 8; ++i) g.W1[i] = c.W1_by_cls ? c.W1_by_cls[i] : nullptr;
    g.Y = c.Y, g.ldy = c.ldy;
    const LevelTables &L = ctx->lev[c.level];
    const bool cls = c.mode == GM_STENCIL || c.mode == GM_PARENT2;
    g.rows = c.rows ? c.rows : cls ? L.cls_rows : nullptr;
    g.child = L.child;
    g.parent = L.parent;
    g.keys = L.keys;
    g.dense = c.dense ? c.dense : L.dense;
    g.class_slots = ctx->class_slots;
    g.class_delta = ctx->class_delta;
    return g;
}

namespace {

// Option mean_free.  Downward check potentials carry the whole far-field potential, whose size
// is that of the potential itself while the gradients at a leaf depend only on its variation
// across the leaf.  Taking the per-box mean off after every downward step keeps the stored
// values at the size of that variation, so their rounding no longer grows into gradient error
// as boxes shrink.  A constant potential has zero gradient and D2D maps it onto itself up to the
// operators' fit error, so the means are carried down the tree separately (FP64) and added back
// to the leaf potentials only.
template <typename T>
__global__ void remove_mean_kernel(T *__restrict__ D, int n, int ns, int ld, const int *__restrict__ parent,
                                   const double *__restrict__ c_parent, double *__restrict__ c_out) {
    const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (b >= n) return;
    T *row = D + (size_t)b * ld;
    double sum = 0;
    for (int j = lane; j < ns; j += 32) sum += (double)row[j];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const double m = sum / ns;
    for (int j = lane; j < ns; j += 32) row[j] = (T)((double)row[j] - m);
    if (lane == 0) c_out[b] = m + (c_parent ? c_parent[parent[b]] : 0.0);
}

// Tensor-core contractions in the split-precision modes, except the leaf closing: its second
// factor (V S^-1) carries the inverse singular values of the check-to-equivalent map and stays
// in FP32 so that its rounding is attenuated by the D2T evaluation as analysed for FP32.
template <typename T>
cudaError_t gemm(const fmm_ctx *ctx, const GemmCall &c, int op_id, cudaStream_t s) {
    const int op = op_id % OP_COUNT;
    if (ctx->tensor && op != OP_CLOSE1 && op != OP_CLOSE2) return gemm_tc(ctx, c, op_id, s);
    return gemm_simt<T>(ctx, c, s);
}

template <typename T>
T *rows_at(void *base, const fmm_ctx *ctx, int level, int ld) {
    return (T *)base + (size_t)ctx->lev[level].row_base * ld;
}

}  // namespace

template <typename T>
FarSteps<T>::FarSteps(fmm_ctx *c, bool adj) : ctx(c), adjoint(adj) {
    d = ctx->opt.depth;
    nsp = ctx->nsp;
    kw = ctx->ws_kw;
    A = adjoint ? ctx->Dc : ctx->Uc;
    B = adjoint ? ctx->Uc : ctx->Dc;
    f16 = ctx->opt.precision == FMM_FP16X3;
    nck_s = (nsp + 63) / 64, nck_k = (kw + 63) / 64;
}

// FMM_FP16X3: every contraction reads FP16 planes, which the step producing its input writes
// beside (or instead of) the FP32 rows: level l's rows of the upward side (UpP), of the
// downward side (DnP), of the compressed vectors (UtP) and of the stencil output (CtP)
template <typename T> unsigned char *FarSteps<T>::upP(int l) const {
    return (unsigned char *)ctx->UpP + base(l) * nsp * 2;
}
template <typename T> unsigned char *FarSteps<T>::dnP(int l) const {
    return (unsigned char *)ctx->DnP + base(l) * nsp * 2;
}
template <typename T> unsigned char *FarSteps<T>::ctP(int l) const {
    return (unsigned char *)ctx->CtP + base(l) * kw * 2;
}
template <typename T> float *FarSteps<T>::upS(int l) const { return ctx->Ups + base(l) * nck_s; }
template <typename T> float *FarSteps<T>::dnS(int l) const { return ctx->Dns + base(l) * nck_s; }
template <typename T> float *FarSteps<T>::ctS(int l) const { return ctx->Cts + base(l) * nck_k; }

// operators of level l (one set for Laplace; per level for the modified Helmholtz kernel)
template <typename T> const OpSet &FarSteps<T>::O(int l) const { return adjoint ? ctx->adj[l] : ctx->fwd[l]; }

// S2U (forward) or D2T^T and the transposed closing (adjoint) on the leaves, and the leaf
// rows' planes
template <typename T>
cudaError_t FarSteps<T>::leaf_in(cudaStream_t s) {
    const OpSet &o = O(d);
    const T *grid = (const T *)ctx->grid_dev;
    const double r_leaf = ctx->side / (double)(1 << d) * 0.5;
    const int dir = adjoint ? 1 : 0;
    if (!adjoint) {
        FMM_CUDA_TRY(launch_leaf_check<T>(ctx, grid, rows_at<T>(A, ctx, d, nsp), s));
    } else {
        FMM_CUDA_TRY(launch_leaf_check<T>(ctx, grid, (T *)ctx->Dq, s));
        GemmCall c1;
        c1.mode = GM_IDENTITY, c1.level = d, c1.n_out = o.rclp;
        c1.X0 = ctx->Dq, c1.ldx0 = nsp, c1.k0 = nsp, c1.W0 = o.close1;
        c1.Y = ctx->Yc, c1.ldy = o.rclp;
        FMM_CUDA_TRY(gemm<T>(ctx, c1, OP_CLOSE1 + dir * OP_COUNT, s));
        GemmCall c2;
        c2.mode = GM_IDENTITY, c2.level = d, c2.n_out = nsp, c2.alpha = r_leaf;
        c2.X0 = ctx->Yc, c2.ldx0 = o.rclp, c2.k0 = o.rclp, c2.W0 = o.close2;
        c2.Y = rows_at<T>(A, ctx, d, nsp), c2.ldy = nsp;
        FMM_CUDA_TRY(gemm<T>(ctx, c2, OP_CLOSE2 + dir * OP_COUNT, s));
    }
    if (f16)
        FMM_CUDA_TRY(launch_rows_to_planes((const float *)rows_at<T>(A, ctx, d, nsp), nsp, ctx->lev[d].n, nsp, upP(d),
                                           ctx->upp_plane, nsp, upS(d), nck_s, s));
    return cudaSuccess;
}

// U2U: level l's upward-side rows from level l + 1's
template <typename T>
cudaError_t FarSteps<T>::up(int l, cudaStream_t s) {
    GemmCall c;
    c.mode = GM_CHILDREN, c.level = l, c.n_out = nsp;
    c.X0 = rows_at<T>(A, ctx, l + 1, nsp), c.ldx0 = nsp, c.k0 = nsp;
    c.W0 = O(l).up[0], c.w_stride = (int64_t)nsp * nsp;
    c.Y = rows_at<T>(A, ctx, l, nsp), c.ldy = nsp;
    if (f16) {
        c.Xp = upP(l + 1), c.xp_ld = nsp, c.xp_plane = ctx->upp_plane, c.xp_scale = upS(l + 1), c.xp_scale_ld = nck_s;
        c.Yp = upP(l), c.yp_ld = nsp, c.yp_plane = ctx->upp_plane, c.yp_scale = upS(l), c.yp_scale_ld = nck_s;
    }
    return gemm<T>(ctx, c, OP_UP + (adjoint ? OP_COUNT : 0), s);
}

// VLI compress: Ut_l = Vi^T U_l.  Tensor-core modes pass the compressed vectors to the stencil
// as split planes, so that it copies its source rows instead of converting them itself.
template <typename T>
cudaError_t FarSteps<T>::compress(int l, cudaStream_t s) {
    const OpSet &o = O(l);
    GemmCall c;
    c.mode = GM_IDENTITY, c.level = l, c.n_out = o.kinp;
    c.X0 = rows_at<T>(A, ctx, l, nsp), c.ldx0 = nsp, c.k0 = nsp, c.W0 = o.compress;
    c.Y = ctx->tensor ? nullptr : rows_at<T>(ctx->Ut, ctx, l, kw), c.ldy = kw;   // tensor modes: planes only
    if (ctx->tensor) {
        c.Yp = utP(l), c.yp_ld = kw, c.yp_plane = ctx->utp_plane;
        c.yp_scale = utS(l), c.yp_scale_ld = nck_k;
    }
    if (f16) c.Xp = upP(l), c.xp_ld = nsp, c.xp_plane = ctx->upp_plane, c.xp_scale = upS(l), c.xp_scale_ld = nck_s;
    return gemm<T>(ctx, c, OP_COMPRESS + (adjoint ? OP_COUNT : 0), s);
}

template <typename T> unsigned char *FarSteps<T>::utP(int l) const {
    const int pesz = ctx->opt.precision == FMM_TF32X3 ? 4 : 2;
    return (unsigned char *)ctx->UtP + base(l) * kw * pesz;
}
template <typename T> float *FarSteps<T>::utS(int l) const { return ctx->Uscale ? ctx->Uscale + base(l) * nck_k : nullptr; }

// VLI stencil: Ct_l[b] = sum_t C_t Ut_l[b + t]
template <typename T>
cudaError_t FarSteps<T>::stencil(int l, cudaStream_t s) {
    const OpSet &o = O(l);
    GemmCall st;
    st.mode = GM_STENCIL, st.level = l, st.n_out = o.koutp;
    st.X0 = rows_at<T>(ctx->Ut, ctx, l, kw), st.ldx0 = kw, st.k0 = o.kinp;
    st.W0 = o.stencil, st.w_stride = (int64_t)o.koutp * o.kinp;
    st.Y = rows_at<T>(ctx->Ct, ctx, l, kw), st.ldy = kw;
    if (ctx->tensor) {
        st.Xp = utP(l), st.xp_ld = kw, st.xp_rows = (int)ctx->lev[l].n, st.xp_plane = ctx->utp_plane;
        st.xp_scale = utS(l), st.xp_scale_ld = nck_k;
    }
    if (f16) {   // the decompress reads the stencil output as planes
        st.Y = nullptr;
        st.Yp = ctP(l), st.yp_ld = kw, st.yp_plane = ctx->ctp_plane, st.yp_scale = ctS(l), st.yp_scale_ld = nck_k;
    }
    return gemm<T>(ctx, st, OP_STENCIL + (adjoint ? OP_COUNT : 0), s);
}

// downward step of level l: decompress fused with the parent's D2D contribution (l >= 3)
template <typename T>
cudaError_t FarSteps<T>::down(int l, cudaStream_t s) {
    const OpSet &o = O(d);
    GemmCall c;
    c.mode = GM_PARENT2, c.level = l, c.n_out = nsp;
    c.X0 = rows_at<T>(ctx->Ct, ctx, l, kw), c.ldx0 = kw, c.k0 = o.koutp, c.W0 = O(l).decompress;
    if (l >= 3) {   // D2D from the parent level: that level's operators
        c.X1 = rows_at<T>(B, ctx, l - 1, nsp), c.ldx1 = nsp, c.k1 = nsp;
        c.W1_by_cls = O(l - 1).down;
    }
    c.Y = rows_at<T>(B, ctx, l, nsp), c.ldy = nsp;
    if (f16) {
        c.Xp = ctP(l), c.xp_ld = kw, c.xp_plane = ctx->ctp_plane, c.xp_scale = ctS(l), c.xp_scale_ld = nck_k;
        if (l >= 3)
            c.Xp1 = dnP(l - 1), c.xp1_ld = nsp, c.xp1_plane = ctx->upp_plane, c.xp1_scale = dnS(l - 1),
            c.xp1_scale_ld = nck_s;
        if (l < d)   // the leaves' rows have no children to read them as planes
            c.Yp = dnP(l), c.yp_ld = nsp, c.yp_plane = ctx->upp_plane, c.yp_scale = dnS(l), c.yp_scale_ld = nck_s;
    }
    FMM_CUDA_TRY(gemm<T>(ctx, c, OP_DECOMPRESS + (adjoint ? OP_COUNT : 0), s));
    if (!adjoint && ctx->opt.mean_free) {
        const LevelTables &L = ctx->lev[l];
        double *cm = (double *)ctx->Cmean;
        remove_mean_kernel<T><<<(unsigned)((L.n + 7) / 8), 256, 0, s>>>(
            rows_at<T>(B, ctx, l, nsp), (int)L.n, ctx->ns, nsp, L.parent,
            l >= 3 ? cm + ctx->lev[l - 1].row_base : nullptr, cm + L.row_base);
        count_launch();
        FMM_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

// leaf output: closing pseudo-inverse and D2T (forward), or the S2U^T evaluation (adjoint)
template <typename T>
cudaError_t FarSteps<T>::leaf_out(T *far_phi, T *far_grad, cudaStream_t s) {
    const OpSet &o = O(d);
    const T *grid = (const T *)ctx->grid_dev;
    const double r_leaf = ctx->side / (double)(1 << d) * 0.5;
    if (!adjoint) {
        GemmCall c1;
        c1.mode = GM_IDENTITY, c1.level = d, c1.n_out = o.rclp;
        c1.X0 = rows_at<T>(B, ctx, d, nsp), c1.ldx0 = nsp, c1.k0 = nsp, c1.W0 = o.close1;
        c1.Y = ctx->Yc, c1.ldy = o.rclp;
        FMM_CUDA_TRY(gemm<T>(ctx, c1, OP_CLOSE1, s));
        GemmCall c2;
        c2.mode = GM_IDENTITY, c2.level = d, c2.n_out = nsp, c2.alpha = r_leaf;
        c2.X0 = ctx->Yc, c2.ldx0 = o.rclp, c2.k0 = o.rclp, c2.W0 = o.close2;
        c2.Y = ctx->Dq, c2.ldy = nsp;
        FMM_CUDA_TRY(gemm<T>(ctx, c2, OP_CLOSE2, s));
        return launch_leaf_eval<T>(ctx, grid, (const T *)ctx->Dq, nsp, (T)1, far_phi, far_grad, s,
                                   ctx->opt.mean_free ? (const double *)ctx->Cmean + ctx->lev[d].row_base : nullptr);
    }
    return launch_leaf_eval<T>(ctx, grid, rows_at<T>(B, ctx, d, nsp), nsp, (T)1, far_phi, nullptr, s, nullptr);
}

// Downward pass with the FFT form of the M2L (forward only): per level, D2D from the parent (or
// zero at level 2), then the lattice convolution of the V list added in (fft.cu).
template <typename T>
cudaError_t run_far_fft(fmm_ctx *ctx, FarSteps<T> &f, T *far_phi, T *far_grad, cudaStream_t s) {
    const int d = f.d, nsp = f.nsp;
    for (int l = 2; l <= d; ++l) {
        if (l == d) cudaEventRecord(ctx->ev[4], s);
        T *D = rows_at<T>(f.B, ctx, l, nsp);
        if (l >= 3) {   // D2D alone: PARENT2 with an empty first segment
            GemmCall c;
            c.mode = GM_PARENT2, c.level = l, c.n_out = nsp;
            c.X0 = D, c.ldx0 = nsp, c.k0 = 0, c.W0 = f.O(l).up[0];
            c.X1 = rows_at<T>(f.B, ctx, l - 1, nsp), c.ldx1 = nsp, c.k1 = nsp;
            c.W1_by_cls = f.O(l - 1).down;
            c.Y = D, c.ldy = nsp;
            FMM_CUDA_TRY(gemm_simt<T>(ctx, c, s));
        } else {
            FMM_CUDA_TRY(cudaMemsetAsync(D, 0, (size_t)ctx->lev[l].n * nsp * sizeof(T), s));
        }
        FMM_CUDA_TRY(fft_vli<T>(ctx, l, rows_at<T>(f.A, ctx, l, nsp), D, s));
    }
    return f.leaf_out(far_phi, far_grad, s);
}

template <typename T>
cudaError_t run_far(fmm_ctx *ctx, bool adjoint, T *far_phi, T *far_grad, cudaStream_t s) {
    if (ctx->adaptive_eval) return adaptive_far<T>(ctx, far_phi, far_grad, s);   // forward only
    FarSteps<T> f(ctx, adjoint);
    const int d = f.d;
    if (ctx->fft) {
        FMM_CUDA_TRY(f.leaf_in(s));
        cudaEventRecord(ctx->ev[2], s);
        for (int l = d - 1; l >= 2; --l) FMM_CUDA_TRY(f.up(l, s));
        cudaEventRecord(ctx->ev[3], s);
        return run_far_fft<T>(ctx, f, far_phi, far_grad, s);
    }
    FMM_CUDA_TRY(f.leaf_in(s));
    cudaEventRecord(ctx->ev[2], s);
    for (int l = d - 1; l >= 2; --l) FMM_CUDA_TRY(f.up(l, s));
    cudaEventRecord(ctx->ev[3], s);
    // VLI of every level on its own stream (levels are independent once the upward pass is
    // done); the downward sweep below waits for each level's VLI just before using it
    FMM_CUDA_TRY(cudaEventRecord(ctx->fork_ev[0], s));
    for (int l = 2; l <= d; ++l) {
        cudaStream_t ls = ctx->aux[l];
        FMM_CUDA_TRY(cudaStreamWaitEvent(ls, ctx->fork_ev[0], 0));
        FMM_CUDA_TRY(f.compress(l, ls));
        FMM_CUDA_TRY(f.stencil(l, ls));
        FMM_CUDA_TRY(cudaEventRecord(ctx->join_ev[l], ls));
    }
    for (int l = 2; l <= d; ++l) {
        FMM_CUDA_TRY(cudaStreamWaitEvent(s, ctx->join_ev[l], 0));
        if (l == d) cudaEventRecord(ctx->ev[4], s);
        FMM_CUDA_TRY(f.down(l, s));
    }
    return f.leaf_out(far_phi, far_grad, s);
}

template struct FarSteps<float>;
template struct FarSteps<double>;
template cudaError_t run_far<float>(fmm_ctx *, bool, float *, float *, cudaStream_t);
template cudaError_t run_far<double>(fmm_ctx *, bool, double *, double *, cudaStream_t);

// ---------------------------------------------------------------------------------------
// operator upload (SIMT layouts: row-major, zero padded)
// ---------------------------------------------------------------------------------------
namespace {

template <typename T>
cudaError_t upload_padded(fmm_ctx *ctx, const std::vector<double> &w, int rows, int cols,
                          int rows_p, int cols_p, int count, void **out) {
    std::vector<T> h((size_t)count * rows_p * cols_p, (T)0);
    for (int m = 0; m < count; ++m)
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < cols; ++j)
                h[(size_t)m * rows_p * cols_p + (size_t)i * cols_p + j] =
                    (T)w[(size_t)m * rows * cols + (size_t)i * cols + j];
    void *p = nullptr;
    FMM_CUDA_TRY(dev_malloc(&p, h.size() * sizeof(T)));
    ctx->op_allocs.push_back(p);
    FMM_CUDA_TRY(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *out = p;
    return cudaSuccess;
}

template <typename T>
cudaError_t upload_set(fmm_ctx *ctx, const HostOps &h, bool adjoint, OpSet &o) {
    const int ns = h.ns, nsp = round_up(ns, 16);
    o.ns = ns, o.nsp = nsp;
    o.kin = adjoint ? h.kout : h.kin;
    o.kout = adjoint ? h.kin : h.kout;
    o.kinp = round_up(o.kin, 16), o.koutp = round_up(o.kout, 16);
    o.rcl = h.rcl, o.rclp = round_up(h.rcl, 16);
    const auto &up = adjoint ? h.a_up : h.up;
    const auto &down = adjoint ? h.a_down : h.down;
    // the 8 U2U operators contiguous so that W0 + c * nsp * nsp addresses octant c
    std::vector<double> ups;
    for (int c = 0; c < 8; ++c) ups.insert(ups.end(), up[c].begin(), up[c].end());
    FMM_CUDA_TRY(upload_padded<T>(ctx, ups, ns, ns, nsp, nsp, 8, &o.up[0]));
    for (int c = 1; c < 8; ++c) o.up[c] = (T *)o.up[0] + (size_t)c * nsp * nsp;
    for (int c = 0; c < 8; ++c) FMM_CUDA_TRY(upload_padded<T>(ctx, down[c], ns, ns, nsp, nsp, 1, &o.down[c]));
    if (!h.fft_n) {   // the compressed M2L (the FFT form has its own transforms, fft.cu)
        FMM_CUDA_TRY(upload_padded<T>(ctx, adjoint ? h.a_compress : h.compress, o.kin, ns, o.kinp, nsp, 1, &o.compress));
        FMM_CUDA_TRY(upload_padded<T>(ctx, adjoint ? h.a_stencil : h.stencil, o.kout, o.kin, o.koutp, o.kinp,
                                      kNumTransfer, &o.stencil));
        FMM_CUDA_TRY(upload_padded<T>(ctx, adjoint ? h.a_decompress : h.decompress, ns, o.kout, nsp, o.koutp, 1,
                                      &o.decompress));
    }
    FMM_CUDA_TRY(upload_padded<T>(ctx, adjoint ? h.a_close1 : h.close1, h.rcl, ns, o.rclp, nsp, 1, &o.close1));
    FMM_CUDA_TRY(upload_padded<T>(ctx, adjoint ? h.a_close2 : h.close2, ns, h.rcl, nsp, o.rclp, 1, &o.close2));
    if (!adjoint && h.rclu > 0) {
        o.rclu = h.rclu, o.rclup = round_up(h.rclu, 16);
        FMM_CUDA_TRY(upload_padded<T>(ctx, h.uclose1, h.rclu, ns, o.rclup, nsp, 1, &o.uclose1));
        FMM_CUDA_TRY(upload_padded<T>(ctx, h.uclose2, ns, h.rclu, nsp, o.rclup, 1, &o.uclose2));
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t upload_operators(fmm_ctx *ctx) {
    // every distinct host set once; levels sharing a set share its device copy
    for (int l = 0; l <= kMaxDepth; ++l) {
        int first = -1;
        for (int k = 0; k < l && first < 0; ++k)
            if (ctx->host_ops[k] == ctx->host_ops[l]) first = k;
        if (first >= 0) {
            ctx->fwd[l] = ctx->fwd[first];
            ctx->adj[l] = ctx->adj[first];
            continue;
        }
        const HostOps &h = *ctx->host_ops[l];
        if (ctx->fp64) {
            FMM_CUDA_TRY(upload_set<double>(ctx, h, false, ctx->fwd[l]));
            FMM_CUDA_TRY(upload_set<double>(ctx, h, true, ctx->adj[l]));
        } else {
            FMM_CUDA_TRY(upload_set<float>(ctx, h, false, ctx->fwd[l]));
            FMM_CUDA_TRY(upload_set<float>(ctx, h, true, ctx->adj[l]));
        }
    }
    if (ctx->tensor) FMM_CUDA_TRY(tc_upload_operators(ctx));
    if (ctx->fft) FMM_CUDA_TRY(fft_upload(ctx));
    // unit surface grid in the storage type
    std::vector<double> g = surface_grid(ctx->opt.order_p);
    size_t bytes = g.size() * (ctx->fp64 ? sizeof(double) : sizeof(float));
    FMM_CUDA_TRY(dev_malloc(&ctx->grid_dev, bytes));
    ctx->op_allocs.push_back(ctx->grid_dev);
    if (ctx->fp64) {
        FMM_CUDA_TRY(cudaMemcpy(ctx->grid_dev, g.data(), bytes, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(g.begin(), g.end());
        FMM_CUDA_TRY(cudaMemcpy(ctx->grid_dev, f.data(), bytes, cudaMemcpyHostToDevice));
    }
    return cudaSuccess;
}

}  // namespace fmm
