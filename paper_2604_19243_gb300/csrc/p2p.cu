// Point kernels of the kiFMM (Algorithm 1): the near-field ULI sums (step 3c), the S2U check
// potentials of the leaves (step 1a, before the pseudo-inverse) and the D2T evaluation of the
// leaves' far field (step 3b).  Points live in Morton order as (x, y, z, q) vectors.
//
// Kernel: K(x, y) = 1/(4 pi |x - y|) (Eq. 2 normalised by 4 pi); the gradient with respect to
// the target is (y - x) q / (4 pi |x - y|^3).  With YUK the modified Helmholtz kernel
// exp(-kappa r) / (4 pi r), r = |x - y|, whose gradient is (y - x) q (1 + kappa r) exp(-kappa r)
// / (4 pi r^3); the screening factor is exp2(-kappa log2(e) r) (FP32) or exp(-kappa r) (FP64).
// Pairs at distance zero are skipped (the self interaction and coincident points, which share a
// leaf).
#include <algorithm>
#include <type_traits>

#include "debugcheck.cuh"
#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };

template <typename T> __device__ inline T rsqrt_t(T x);
template <> __device__ inline float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ inline double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename T> __host__ __device__ constexpr T inv4pi() { return (T)0.079577471545947667884441881686257181; }
constexpr double kLog2E = 1.44269504088896340736;   // log2(e)

// screening factor exp(-kappa r) of the modified Helmholtz kernel
__device__ __forceinline__ float screen(float r, float kappa) { return exp2f(-(kappa * (float)kLog2E) * r); }
__device__ __forceinline__ double screen(double r, double kappa) { return exp(-kappa * r); }

// ---------------------------------------------------------------------------------------
// ULI: one CTA (4 warps) per target leaf.  The leaf's targets are cut into chunks of 32 (one
// target per lane).  Each warp holds R chunks at once, so every source read from shared memory
// serves R targets per lane, and works through one of S slices of the sources; R and S are
// chosen per leaf so that the four warps stay busy with little padding (Section 2.2: the ULI is
// the compute-bound kernel the method leans on).
// ---------------------------------------------------------------------------------------
constexpr int kP2PThreads = 128;
constexpr int kP2PChunk = 1024;     // sources staged per pass (16 KB as float4)

// one (target, source) interaction; `checked` skips pairs at distance zero
template <typename T, bool checked, bool YUK = false>
__device__ __forceinline__ void interact(const typename Vec4<T>::type &sp, T xi, T yi, T zi,
                                         T &pot, T &gx, T &gy, T &gz, T kappa = (T)0) {
    const T dx = sp.x - xi, dy = sp.y - yi, dz = sp.z - zi;
    const T r2 = dx * dx + dy * dy + dz * dz;
    T rinv = rsqrt_t<T>(r2);
    if (checked) rinv = r2 > (T)0 ? rinv : (T)0;
    T qr = sp.w * rinv;
    T qr3 = qr * rinv * rinv;
    if (YUK) {
        const T r = r2 * rinv;
        qr *= screen(r, kappa);
        qr3 = qr * rinv * rinv * (kappa * r + (T)1);
    }
    pot += qr;
    gx += qr3 * dx;
    gy += qr3 * dy;
    gz += qr3 * dz;
}

constexpr int kRangeWin = 32;   // source ranges staged per window (one per lane of a warp)

struct P2PRanges {
    int beg[kRangeWin], len[kRangeWin];
    int n, total, self_len;
};

// One round: chunks [cbase, cbase + nch) of the leaf with R chunks per warp group and S source
// slices (4 / S groups of S warps).
template <typename T, int R, bool GRAD, bool YUK>
__device__ __forceinline__ void p2p_round(const typename Vec4<T>::type *__restrict__ pts,
                                          typename Vec4<T>::type *src, T *red, const P2PRanges &rg,
                                          int t0, int t1, int cbase, int nch, int S, T *__restrict__ phi,
                                          T *__restrict__ grad, T kappa) {
    using P = typename Vec4<T>::type;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp / S, slice = warp % S;
    T xi[R], yi[R], zi[R], pot[R], gx[R], gy[R], gz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = t0 + (cbase + grp * R + r) * 32 + lane;
        const P p = pts[min(i, t1 - 1)];
        xi[r] = p.x, yi[r] = p.y, zi[r] = p.z;
        pot[r] = gx[r] = gy[r] = gz[r] = (T)0;
    }
    for (int c0 = 0; c0 < rg.total; c0 += kP2PChunk) {
        const int c1 = min(rg.total, c0 + kP2PChunk);
        __syncthreads();
        int pos = 0;
        for (int k = 0; k < rg.n; ++k) {
            const int lo = max(pos, c0), hi = min(pos + rg.len[k], c1);
            for (int e = lo + (int)threadIdx.x; e < hi; e += kP2PThreads) src[e - c0] = pts[rg.beg[k] + (e - pos)];
            pos += rg.len[k];
        }
        __syncthreads();
        const int n = c1 - c0;
        const int per = (n + S - 1) / S;
        const int s0 = slice * per, s1 = min(n, s0 + per);
        const int chk_end = min(s1, max(s0, rg.self_len - c0));     // [s0, chk_end) may hold self
        for (int e = s0; e < chk_end; ++e) {
            const P sp = src[e];
#pragma unroll
            for (int r = 0; r < R; ++r) interact<T, true, YUK>(sp, xi[r], yi[r], zi[r], pot[r], gx[r], gy[r], gz[r], kappa);
        }
        int e = chk_end;
        for (; e + 4 <= s1; e += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const P sp = src[e + u];
#pragma unroll
                for (int r = 0; r < R; ++r) interact<T, false, YUK>(sp, xi[r], yi[r], zi[r], pot[r], gx[r], gy[r], gz[r], kappa);
            }
        }
        for (; e < s1; ++e) {
            const P sp = src[e];
#pragma unroll
            for (int r = 0; r < R; ++r) interact<T, false, YUK>(sp, xi[r], yi[r], zi[r], pot[r], gx[r], gy[r], gz[r], kappa);
        }
    }
    if (S > 1) {   // reduce the S slices of every group
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T *o = red + ((size_t)(warp * R + r) * 32 + lane) * 4;
            o[0] = pot[r], o[1] = gx[r], o[2] = gy[r], o[3] = gz[r];
        }
        __syncthreads();
        if (slice == 0)
            for (int sl = 1; sl < S; ++sl)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T *o = red + ((size_t)((warp + sl) * R + r) * 32 + lane) * 4;
                    pot[r] += o[0], gx[r] += o[1], gy[r] += o[2], gz[r] += o[3];
                }
    }
    if (slice == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int ch = grp * R + r;
            const int i = t0 + (cbase + ch) * 32 + lane;
            if (ch < nch && i < t1) {
                if (phi) phi[i] = pot[r] * inv4pi<T>();
                if (GRAD) {
                    grad[3 * (int64_t)i] = gx[r] * inv4pi<T>();
                    grad[3 * (int64_t)i + 1] = gy[r] * inv4pi<T>();
                    grad[3 * (int64_t)i + 2] = gz[r] * inv4pi<T>();
                }
            }
        }
    }
    __syncthreads();   // src / red are reused by the next round
}

// ---------------------------------------------------------------------------------------
// FP32 form on pairs of sources.  The two-wide FP32 instructions of sm_100 and later (add, mul
// and fma on float2) do the arithmetic of two (target, source) pairs in one issue slot, so the
// 13 FP32 operations of a pair cost 6.5 issue slots instead of 13 and the FP32 pipe, not the
// instruction issue, bounds the sum.  Sources are staged per pair (j, k) as two float4,
// [x_j x_k y_j y_k] [z_j z_k q_j q_k], padded with zero charges to an even number of pairs.
// Targets are held negated so that one add forms y - x.
// ---------------------------------------------------------------------------------------
template <bool checked, bool YUK = false, bool POT = true>
__device__ __forceinline__ void interact2(const float4 &a, const float4 &b, float2 nx, float2 ny,
                                          float2 nz, float2 &pot, float2 &gx, float2 &gy, float2 &gz,
                                          float kappa = 0.f) {
    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
    const float2 dz = __fadd2_rn(make_float2(b.x, b.y), nz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    if (checked) {
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    float2 qr = __fmul2_rn(make_float2(b.z, b.w), ri);
    float2 qr3;
    if (YUK) {   // r = r2 / r (0 for a skipped pair), q exp(-kappa r) / r, times (1 + kappa r) / r^2
        const float2 r = __fmul2_rn(r2, ri);
        qr = __fmul2_rn(qr, make_float2(screen(r.x, kappa), screen(r.y, kappa)));
        const float2 f = __ffma2_rn(make_float2(kappa, kappa), r, make_float2(1.f, 1.f));
        qr3 = __fmul2_rn(__fmul2_rn(__fmul2_rn(qr, ri), ri), f);
    } else {
        qr3 = __fmul2_rn(__fmul2_rn(qr, ri), ri);
    }
    if (POT) pot = __fadd2_rn(pot, qr);
    gx = __ffma2_rn(qr3, dx, gx);
    gy = __ffma2_rn(qr3, dy, gy);
    gz = __ffma2_rn(qr3, dz, gz);
}

template <int R, bool checked, bool YUK = false, bool POT = true>
__device__ __forceinline__ void pair_step(const float4 *__restrict__ sp, int e, const float2 *nx,
                                          const float2 *ny, const float2 *nz, float2 *pot, float2 *gx,
                                          float2 *gy, float2 *gz, float kappa = 0.f) {
    const float4 a = sp[2 * e], b = sp[2 * e + 1];
#pragma unroll
    for (int r = 0; r < R; ++r)
        interact2<checked, YUK, POT>(a, b, nx[r], ny[r], nz[r], pot[r], gx[r], gy[r], gz[r], kappa);
}

// FP32 ULI kernel.  Targets go to half-warps 16 at a time (the padding of a leaf's last group
// is then 6.7% of the sphere workload's pairs instead of 14% with whole warps), and the work of
// a leaf, (groups of targets) x (source pairs), is cut into four equal contiguous ranges, one
// per warp, so no warp waits on another for more than one pair step.  The two half-warps of a
// warp always walk the same pair indices: they hold two target groups, or, for a leaf with an
// odd number of groups, the two halves of the sources of its last group.  A range may start or
// end inside a group's sweep; the partial sums go to shared memory and are added up per target
// in a fixed order, so the results do not depend on timing.
constexpr int kSmallLeaf = 8;                   // leaves up to this many points: p2p_small_f32_kernel
constexpr int kSub = 16;                        // targets per half-warp
constexpr int kRoundSub = 16;                   // target groups per round
constexpr int kRoundT = kSub * kRoundSub;       // 256 targets per round
constexpr int kSlots = kRoundSub / 2 + 4;       // partial-sum slots: one per (unit, warp) piece

__device__ __forceinline__ void build_ranges(P2PRanges &rg, int b, const int *__restrict__ leaf_off,
                                             const int *__restrict__ u_off, const int *__restrict__ u_idx) {
    // the target leaf first (the only one that can hold a zero distance), then its U list
    const int t0 = leaf_off[b], nt = leaf_off[b + 1] - t0;
    int k = 0, tot = nt;
    rg.beg[k] = t0;
    rg.len[k++] = nt;
    for (int e = u_off[b]; e < u_off[b + 1]; ++e) {
        const int a = u_idx[e];
        if (a == b) continue;
        rg.beg[k] = leaf_off[a];
        rg.len[k] = leaf_off[a + 1] - leaf_off[a];
        tot += rg.len[k++];
    }
    rg.n = k;
    rg.total = tot;
    rg.self_len = nt;
}

// Where the points of a box lie in the sorted order.  Leaves of the uniform tree: box b holds
// [leaf_off[b], leaf_off[b + 1]).  Rows of the adaptive tree (any level): [begin[r], begin[r] +
// count[r]).
struct LeafBoxes {
    const int *leaf_off;
    int npts;                   // points of the sorted arrays (bound of the debug checks)
    __device__ int first(int b) const { return leaf_off[b]; }
    __device__ int size(int b) const { return leaf_off[b + 1] - leaf_off[b]; }
};
struct RowBoxes {
    const int *begin, *count;
    int npts;
    __device__ int first(int b) const { return begin[b]; }
    __device__ int size(int b) const { return count[b]; }
};

// a box's point range, checked against the point arrays in FMM_DEBUG builds (empty if outside)
template <typename Boxes>
__device__ __forceinline__ void box_range(const Boxes &bx, int b, int &beg, int &len) {
    beg = bx.first(b), len = bx.size(b);
    if (!dbg_ok(beg >= 0 && len >= 0 && beg + len <= bx.npts, kDbgP2P)) len = 0;
}

// The sources of target box b in order: b itself (the only box that can hold a zero distance),
// then the other members of its U list in list order; range k >= 1 is list entry k - 1, or k
// once past b's own entry (at position ps of the list, nl if absent).  One warp fills ranges
// [w0, w0 + 32) with their lengths summed by a shuffle scan.
template <typename Boxes>
__device__ __forceinline__ void window_ranges(P2PRanges &rg, const Boxes &bx, int b, const int *__restrict__ list,
                                              int ps, int nr, int w0, int lane) {
    const int k = w0 + lane;
    int beg = 0, len = 0;
    if (k < nr) {
        int a = b;
        if (k > 0) {
            const int m = k - 1;
            a = list[m + (m >= ps ? 1 : 0)];
        }
        box_range(bx, a, beg, len);
    }
    int incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const int len0 = __shfl_sync(0xffffffffu, len, 0);
    rg.beg[lane] = beg, rg.len[lane] = len;
    if (lane == 31) {
        rg.n = min(kRangeWin, nr - w0);
        rg.total = incl;
        rg.self_len = w0 == 0 ? len0 : 0;
    }
}

// OUT: bit 0 potentials, bit 1 gradients (gradient only: the "force" evaluation of N-body codes)
constexpr int kOutPhi = 1, kOutGrad = 2;

// The sources of a box come in windows of up to 32 ranges (one window for every leaf of the
// uniform tree, whose U lists hold at most 27 leaves; adaptive U lists can be longer).
template <int OUT, bool YUK, typename Boxes>
__global__ void __launch_bounds__(kP2PThreads)
p2p_f32_kernel(const float4 *__restrict__ pts, Boxes bx, const int *__restrict__ u_off,
               const int *__restrict__ u_idx, const int *__restrict__ order, float *__restrict__ phi,
               float *__restrict__ grad, float kappa) {
    __shared__ __align__(16) float4 src[kP2PChunk];       // sources, pair layout
    __shared__ __align__(16) float4 tgt[kRoundT];
    __shared__ __align__(16) float4 acc[kRoundT];         // (pot, gx, gy, gz) per target
    __shared__ __align__(16) float4 part[kSlots * 32];
    __shared__ P2PRanges rg;
    __shared__ int s_ps;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, half = lane >> 4, hl = lane & 15;
    const int b = order[blockIdx.x];
    int t0, tn;
    box_range(bx, b, t0, tn);
    const int t1 = t0 + tn;
    if (tn <= kSmallLeaf) return;   // p2p_small_f32_kernel
    const int lo = u_off[b], nl = u_off[b + 1] - lo;
    if (warp == 0) {   // position of b in its own U list (nl if absent); a single window now
        int ps = nl;
        for (int m0 = 0; m0 < nl; m0 += 32) {
            const unsigned hit = __ballot_sync(0xffffffffu, m0 + lane < nl && u_idx[lo + m0 + lane] == b);
            if (hit) {
                ps = m0 + __ffs(hit) - 1;
                break;
            }
        }
        if (lane == 0) s_ps = ps;
        const int nr0 = 1 + nl - (ps < nl ? 1 : 0);
        if (nr0 <= kRangeWin) window_ranges(rg, bx, b, u_idx + lo, ps, nr0, 0, lane);
    }
    __syncthreads();
    const int ps = s_ps, nr = 1 + nl - (ps < nl ? 1 : 0);
    const bool one_window = nr <= kRangeWin;   // every leaf of the uniform tree
    const int groups = (t1 - t0 + kSub - 1) / kSub;
    float *sf = reinterpret_cast<float *>(src);
    for (int gb = 0; gb < groups; gb += kRoundSub) {
        const int m = min(kRoundSub, groups - gb), mt = m * kSub, tb = t0 + gb * kSub;
        __syncthreads();   // tgt / acc of the previous round consumed
        for (int j = tid; j < mt; j += kP2PThreads) {
            tgt[j] = pts[min(tb + j, t1 - 1)];
            acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int npair = m >> 1;                          // units holding two groups
        for (int w0 = 0; w0 < nr; w0 += kRangeWin) {
            if (!one_window) {
                __syncthreads();   // the previous window's ranges are no longer read
                if (warp == 0) window_ranges(rg, bx, b, u_idx + lo, ps, nr, w0, lane);
                __syncthreads();
            }
            for (int c0 = 0; c0 < rg.total; c0 += kP2PChunk) {
                const int c1 = min(rg.total, c0 + kP2PChunk), n = c1 - c0;
                const int L = (((n + 1) >> 1) + 1) & ~1;      // source pairs, even
                __syncthreads();
                int pos = 0;
                for (int k = 0; k < rg.n; ++k) {
                    const int lo = max(pos, c0), hi = min(pos + rg.len[k], c1);
                    for (int e = lo + tid; e < hi; e += kP2PThreads) {
                        const float4 v = pts[rg.beg[k] + (e - pos)];
                        const int j = e - c0;
                        float *o = sf + 8 * (j >> 1) + (j & 1);
                        o[0] = v.x, o[2] = v.y, o[4] = v.z, o[6] = v.w;
                    }
                    pos += rg.len[k];
                }
                for (int j = n + tid; j < 2 * L; j += kP2PThreads) {   // zero charges up to 2L
                    float *o = sf + 8 * (j >> 1) + (j & 1);
                    o[0] = 0.f, o[2] = 0.f, o[4] = 0.f, o[6] = 0.f;
                }
                __syncthreads();
                const int T = npair * L + (m & 1) * (L >> 1);
                const int self_pairs = (max(0, min(n, rg.self_len - c0)) + 1) >> 1;
                const int pad_pair = n >> 1, pad_split = max(0, pad_pair - (L >> 1));
                const int W = (T + 3) >> 2;
                int at = warp * W;
                const int end = min(T, at + W);
                while (at < end) {
                    int u, e0, e1, g, soff;
                    if (at < npair * L) {
                        u = at / L, e0 = at - u * L, e1 = min(L, e0 + (end - at));
                        g = 2 * u + half, soff = 0;
                    } else {
                        u = npair, e0 = at - npair * L, e1 = min(L >> 1, e0 + (end - at));
                        g = m - 1, soff = half * (L >> 1);
                    }
                    const float4 t = tgt[g * kSub + hl];
                    const float2 nx = make_float2(-t.x, -t.x), ny = make_float2(-t.y, -t.y),
                                 nz = make_float2(-t.z, -t.z);
                    float2 pot = make_float2(0.f, 0.f), gx = pot, gy = pot, gz = pot;
                    const float4 *sp = src + 2 * soff;
                    // checked: pairs that may hold a target (the leaf's own points lead the list)
                    // or a padding charge at the origin; the bounds are the same for both halves
                    const int ce = min(e1, max(e0, self_pairs)), ue = max(ce, min(e1, u == npair ? pad_split : pad_pair));
                    constexpr bool POT = OUT & kOutPhi;
                    for (int e = e0; e < ce; ++e)
                        pair_step<1, true, YUK, POT>(sp, e, &nx, &ny, &nz, &pot, &gx, &gy, &gz, kappa);
                    int e = ce;
                    for (; e + 4 <= ue; e += 4) {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            pair_step<1, false, YUK, POT>(sp, e + v, &nx, &ny, &nz, &pot, &gx, &gy, &gz, kappa);
                    }
                    for (; e < ue; ++e) pair_step<1, false, YUK, POT>(sp, e, &nx, &ny, &nz, &pot, &gx, &gy, &gz, kappa);
                    for (e = ue; e < e1; ++e) pair_step<1, true, YUK, POT>(sp, e, &nx, &ny, &nz, &pot, &gx, &gy, &gz, kappa);
                    part[(u + warp) * 32 + lane] =
                        make_float4(pot.x + pot.y, gx.x + gx.y, gy.x + gy.y, gz.x + gz.y);
                    at += e1 - e0;
                }
                __syncthreads();
                for (int j = tid; j < mt; j += kP2PThreads) {   // fixed-order sum of the pieces
                    const int g = j / kSub, h = j % kSub;
                    const bool two = g < 2 * npair;
                    const int u = two ? g >> 1 : npair;
                    const int start = two ? u * L : npair * L, len = two ? L : (L >> 1);
                    float4 s = acc[j];
                    for (int w = start / W; w <= (start + len - 1) / W; ++w) {
                        const float4 *pp = part + (u + w) * 32;
                        const float4 a = two ? pp[(g & 1) * kSub + h] : pp[h];
                        s.x += a.x, s.y += a.y, s.z += a.z, s.w += a.w;
                        if (!two) {
                            const float4 c = pp[kSub + h];
                            s.x += c.x, s.y += c.y, s.z += c.z, s.w += c.w;
                        }
                    }
                    acc[j] = s;
                }
            }
        }
        // acc[j] is read back by the thread that wrote it
        for (int j = tid; j < mt; j += kP2PThreads) {
            const int i = tb + j;
            if (i < t1) {
                const float4 s = acc[j];
                if (OUT & kOutPhi) phi[i] = s.x * inv4pi<float>();
                if (OUT & kOutGrad) {
                    grad[3 * (int64_t)i] = s.y * inv4pi<float>();
                    grad[3 * (int64_t)i + 1] = s.z * inv4pi<float>();
                    grad[3 * (int64_t)i + 2] = s.w * inv4pi<float>();
                }
            }
        }
    }
}

// ULI of the leaves with at most kSmallLeaf targets (the two-point leaves of deep trees): one
// warp per leaf, where the CTA-per-leaf kernel above would leave most of its 128 threads idle.
// Lane l takes target l mod T (T: the leaf's count rounded up to a power of two) and every S-th
// source (S = 32 / T) of the leaf's source list (the leaf itself, then the other members of its
// U list), read through the L1 cache; the S partial sums of a target are then added by a
// butterfly over the lanes, in a fixed order.  The U list is read 32 entries at a time, one per
// lane, and its ranges are passed around by shuffles.
constexpr int kSmallWarps = 8;

template <int OUT, bool YUK, typename Boxes>
__global__ void __launch_bounds__(kSmallWarps * 32)
p2p_small_f32_kernel(const float4 *__restrict__ pts, Boxes bx, const int *__restrict__ u_off,
                     const int *__restrict__ u_idx, const int *__restrict__ order, int n,
                     float *__restrict__ phi, float *__restrict__ grad, float kappa) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kSmallWarps + (threadIdx.x >> 5);
    if (i >= n) return;
    const int b = order ? order[i] : i;
    int t0, nt;
    box_range(bx, b, t0, nt);
    if (nt > kSmallLeaf || nt <= 0) return;
    int lt = 0;
    while ((1 << lt) < nt) ++lt;
    const int T = 1 << lt, S = 32 >> lt, ti = lane & (T - 1), sl = lane >> lt;
    const float4 x = pts[t0 + min(ti, nt - 1)];
    float pot = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    int pos = 0;   // position of the current range's first source in the whole list
    auto range = [&](int beg, int len) {
        for (int e = (sl - pos) & (S - 1); e < len; e += S)
            interact<float, true, YUK>(pts[beg + e], x.x, x.y, x.z, pot, gx, gy, gz, kappa);
        pos += len;
    };
    range(t0, nt);
    const int lo = u_off[b], nl = u_off[b + 1] - lo;
    for (int w0 = 0; w0 < nl; w0 += 32) {
        int beg = 0, len = 0;
        if (w0 + lane < nl) {
            const int a = u_idx[lo + w0 + lane];
            if (a != b) box_range(bx, a, beg, len);
        }
        const int kn = min(32, nl - w0);
        for (int k = 0; k < kn; ++k) {
            const int bg = __shfl_sync(0xffffffffu, beg, k), ln = __shfl_sync(0xffffffffu, len, k);
            if (ln) range(bg, ln);
        }
    }
    for (int o = T; o < 32; o <<= 1) {
        pot += __shfl_xor_sync(0xffffffffu, pot, o);
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
    }
    if (sl == 0 && ti < nt) {
        const int64_t k = t0 + ti;
        if (OUT & kOutPhi) phi[k] = pot * inv4pi<float>();
        if (OUT & kOutGrad) {
            grad[3 * k] = gx * inv4pi<float>();
            grad[3 * k + 1] = gy * inv4pi<float>();
            grad[3 * k + 2] = gz * inv4pi<float>();
        }
    }
}

template <typename T, bool GRAD, bool YUK>
__global__ void __launch_bounds__(kP2PThreads)
p2p_kernel(const typename Vec4<T>::type *__restrict__ pts, const int *__restrict__ leaf_off,
           const int *__restrict__ u_off, const int *__restrict__ u_idx,
           const int *__restrict__ order, T *__restrict__ phi, T *__restrict__ grad, T kappa) {
    using P = typename Vec4<T>::type;
    __shared__ __align__(16) unsigned char smem_raw[kP2PChunk * sizeof(P)];
    __shared__ P2PRanges rg;
    P *src = reinterpret_cast<P *>(smem_raw);
    T *red = reinterpret_cast<T *>(smem_raw);   // [4 warps][R][32][4] after the sources are used

    const int b = order[blockIdx.x];
    const int t0 = leaf_off[b], t1 = leaf_off[b + 1];
    const int nt = t1 - t0;
    if (threadIdx.x == 0) build_ranges(rg, b, leaf_off, u_off, u_idx);
    __syncthreads();
    const int C = (nt + 31) / 32;   // target chunks
    for (int cbase = 0; cbase < C; cbase += 16) {
        const int nch = min(16, C - cbase);
        int R, S;
        if (nch <= 4) R = nch, S = 4;
        else if (nch <= 8) R = (nch + 1) / 2, S = 2;
        else R = (nch + 3) / 4, S = 1;
        switch (R) {
            case 1: p2p_round<T, 1, GRAD, YUK>(pts, src, red, rg, t0, t1, cbase, nch, S, phi, grad, kappa); break;
            case 2: p2p_round<T, 2, GRAD, YUK>(pts, src, red, rg, t0, t1, cbase, nch, S, phi, grad, kappa); break;
            case 3: p2p_round<T, 3, GRAD, YUK>(pts, src, red, rg, t0, t1, cbase, nch, S, phi, grad, kappa); break;
            default: p2p_round<T, 4, GRAD, YUK>(pts, src, red, rg, t0, t1, cbase, nch, S, phi, grad, kappa); break;
        }
    }
}

// ---------------------------------------------------------------------------------------
// S2U check potentials: row b = K(x^{uc}_b, y_b) s_b on the 2.95 surface of leaf b.
// ---------------------------------------------------------------------------------------
constexpr int kLeafThreads = 128;
constexpr int kLeafChunk = 1024;

// The leaf kernels take box b = list[blockIdx.x] (blockIdx.x without a list), its points from
// `bx` (LeafBoxes for the leaves of the uniform tree, RowBoxes for the leaves of one level of the
// adaptive tree) and its Morton key from the level's keys.
template <typename T, bool YUK, typename Boxes>
__global__ void __launch_bounds__(kLeafThreads)
leaf_check_kernel(const typename Vec4<T>::type *__restrict__ pts, Boxes bx, const int *__restrict__ list,
                  const uint32_t *__restrict__ keys, const T *__restrict__ grid, int ns, int nsp,
                  double ox, double oy, double oz, double width, double radius,
                  T *__restrict__ out, T kappa) {
    using P = typename Vec4<T>::type;
    __shared__ P src[kLeafChunk];
    const int b = list ? list[blockIdx.x] : (int)blockIdx.x;
    int s0, sn;
    box_range(bx, b, s0, sn);
    const int s1 = s0 + sn;
    int ax, ay, az;
    demorton3(keys[b], ax, ay, az);
    const double cx = ox + (ax + 0.5) * width, cy = oy + (ay + 0.5) * width,
                 cz = oz + (az + 0.5) * width;
    for (int i0 = 0; i0 < nsp; i0 += kLeafThreads) {
        const int i = i0 + threadIdx.x;
        T px = 0, py = 0, pz = 0;
        if (i < ns) {
            px = (T)(cx + radius * (double)grid[3 * i]);
            py = (T)(cy + radius * (double)grid[3 * i + 1]);
            pz = (T)(cz + radius * (double)grid[3 * i + 2]);
        }
        T acc = 0;
        for (int c0 = s0; c0 < s1; c0 += kLeafChunk) {
            const int c1 = min(s1, c0 + kLeafChunk);
            __syncthreads();
            for (int e = c0 + threadIdx.x; e < c1; e += kLeafThreads) src[e - c0] = pts[e];
            __syncthreads();
            if (i < ns)
                for (int e = 0; e < c1 - c0; ++e) {
                    const P sp = src[e];
                    const T dx = sp.x - px, dy = sp.y - py, dz = sp.z - pz;
                    const T r2 = dx * dx + dy * dy + dz * dz, ri = rsqrt_t<T>(r2);
                    acc += YUK ? sp.w * ri * screen(r2 * ri, kappa) : sp.w * ri;
                }
        }
        if (i < nsp) out[(int64_t)b * nsp + i] = i < ns ? acc * inv4pi<T>() : (T)0;
    }
}

// FP32 form: one thread per surface point (160 threads cover the 152 points of p = 6 in one
// pass), the leaf's points staged as pairs and summed with the two-wide FP32 instructions.  An
// odd count is padded with a copy of the last point carrying zero charge: every source lies in
// the leaf box and every target on the 2.95 surface outside it, so no distance is zero.
constexpr int kCheckThreads = 160;

template <bool YUK, typename Boxes>
__global__ void __launch_bounds__(kCheckThreads)
leaf_check_f32_kernel(const float4 *__restrict__ pts, Boxes bx, const int *__restrict__ list,
                      const uint32_t *__restrict__ keys, const float *__restrict__ grid, int ns, int nsp,
                      double ox, double oy, double oz, double width, double radius, float *__restrict__ out,
                      float kappa) {
    __shared__ __align__(16) float4 src[kLeafChunk];   // kLeafChunk sources as pairs
    __shared__ float cen[3];
    float *sf = reinterpret_cast<float *>(src);
    const int b = list ? list[blockIdx.x] : (int)blockIdx.x;
    int s0, sn;
    box_range(bx, b, s0, sn);
    const int s1 = s0 + sn;
    if (threadIdx.x == 0) {   // the box centre in FP64 once, rounded to FP32
        int ax, ay, az;
        demorton3(keys[b], ax, ay, az);
        cen[0] = (float)(ox + (ax + 0.5) * width), cen[1] = (float)(oy + (ay + 0.5) * width);
        cen[2] = (float)(oz + (az + 0.5) * width);
    }
    __syncthreads();
    const float r32 = (float)radius;
    for (int i0 = 0; i0 < nsp; i0 += kCheckThreads) {
        const int i = i0 + threadIdx.x;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (i < ns) {   // centre + radius * grid point: two FP32 roundings, no FP64 per thread
            px = fmaf(r32, grid[3 * i], cen[0]);
            py = fmaf(r32, grid[3 * i + 1], cen[1]);
            pz = fmaf(r32, grid[3 * i + 2], cen[2]);
        }
        const float2 nx = make_float2(-px, -px), ny = make_float2(-py, -py), nz = make_float2(-pz, -pz);
        float2 acc = make_float2(0.f, 0.f);
        for (int c0 = s0; c0 < s1; c0 += kLeafChunk) {
            const int c1 = min(s1, c0 + kLeafChunk), n = c1 - c0;
            __syncthreads();
            for (int e = threadIdx.x; e < n + (n & 1); e += kCheckThreads) {
                const float4 v = pts[c0 + min(e, n - 1)];
                float *o = sf + 8 * (e >> 1) + (e & 1);
                o[0] = v.x, o[2] = v.y, o[4] = v.z, o[6] = e < n ? v.w : 0.f;
            }
            __syncthreads();
            if (i < ns)
                for (int e = 0; e < (n + 1) >> 1; ++e) {
                    const float4 a = src[2 * e], c = src[2 * e + 1];
                    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
                    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
                    const float2 dz = __fadd2_rn(make_float2(c.x, c.y), nz);
                    float2 r2 = __fmul2_rn(dx, dx);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dz, dz, r2);
                    float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                    if (YUK) {
                        const float2 r = __fmul2_rn(r2, ri);
                        ri = __fmul2_rn(ri, make_float2(screen(r.x, kappa), screen(r.y, kappa)));
                    }
                    acc = __ffma2_rn(make_float2(c.z, c.w), ri, acc);
                }
        }
        if (i < nsp) out[(int64_t)b * nsp + i] = i < ns ? (acc.x + acc.y) * inv4pi<float>() : 0.f;
    }
}

// ---------------------------------------------------------------------------------------
// D2T: potentials (and gradients) at the points of leaf b from densities on its 2.95 surface.
// ---------------------------------------------------------------------------------------
template <typename T, bool GRAD, bool YUK, typename Boxes>
__global__ void __launch_bounds__(kLeafThreads)
leaf_eval_kernel(const typename Vec4<T>::type *__restrict__ pts, Boxes bx, const int *__restrict__ list,
                 const uint32_t *__restrict__ keys, const T *__restrict__ grid, int ns,
                 const T *__restrict__ dens, int ldd, T scale, double ox, double oy, double oz,
                 double width, double radius, T *__restrict__ phi, T *__restrict__ grad,
                 const double *__restrict__ shift, T kappa) {
    using P = typename Vec4<T>::type;
    extern __shared__ unsigned char smem_raw[];
    P *src = reinterpret_cast<P *>(smem_raw);    // [ns]
    __shared__ double cen[3];
    __shared__ float cenf[3];
    const int b = list ? list[blockIdx.x] : (int)blockIdx.x;
    if (threadIdx.x == 0) {   // the box centre once per leaf
        int ax, ay, az;
        demorton3(keys[b], ax, ay, az);
        cen[0] = ox + (ax + 0.5) * width, cen[1] = oy + (ay + 0.5) * width, cen[2] = oz + (az + 0.5) * width;
        cenf[0] = (float)cen[0], cenf[1] = (float)cen[1], cenf[2] = (float)cen[2];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ns; j += kLeafThreads) {
        P p;
        if constexpr (std::is_same<T, float>::value) {   // FP32: no FP64 arithmetic per surface point
            const float r32 = (float)radius;
            p.x = fmaf(r32, grid[3 * j], cenf[0]);
            p.y = fmaf(r32, grid[3 * j + 1], cenf[1]);
            p.z = fmaf(r32, grid[3 * j + 2], cenf[2]);
        } else {
            p.x = (T)(cen[0] + radius * (double)grid[3 * j]);
            p.y = (T)(cen[1] + radius * (double)grid[3 * j + 1]);
            p.z = (T)(cen[2] + radius * (double)grid[3 * j + 2]);
        }
        p.w = dens[(int64_t)b * ldd + j];
        src[j] = p;
    }
    __syncthreads();
    int t0, tn;
    box_range(bx, b, t0, tn);
    const int t1 = t0 + tn;
    if constexpr (std::is_same<T, float>::value) {
        // FP32: the (even) surface count re-staged as pairs, two-wide FP32 arithmetic; the
        // surface lies outside the leaf box, so no distance is zero
        float4 *pr = reinterpret_cast<float4 *>(smem_raw) + ns;   // [ns] float4 = ns / 2 pairs
        float *sf = reinterpret_cast<float *>(pr);
        for (int j = threadIdx.x; j < ns; j += kLeafThreads) {
            const float4 v = src[j];
            float *o = sf + 8 * (j >> 1) + (j & 1);
            o[0] = v.x, o[2] = v.y, o[4] = v.z, o[6] = v.w;
        }
        __syncthreads();
        for (int i = t0 + threadIdx.x; i < t1; i += kLeafThreads) {
            const float4 x = pts[i];
            const float2 nx = make_float2(-x.x, -x.x), ny = make_float2(-x.y, -x.y), nz = make_float2(-x.z, -x.z);
            float2 pot = make_float2(0.f, 0.f), gx = pot, gy = pot, gz = pot;
            for (int e = 0; e < ns / 2; ++e) pair_step<1, false, YUK>(pr, e, &nx, &ny, &nz, &pot, &gx, &gy, &gz, kappa);
            const float f = scale * inv4pi<float>();
            if (phi) phi[i] = (pot.x + pot.y) * f + (shift ? (float)shift[b] : 0.f);   // the leaf's constant part
            if (GRAD) {
                grad[3 * (int64_t)i] = (gx.x + gx.y) * f;
                grad[3 * (int64_t)i + 1] = (gy.x + gy.y) * f;
                grad[3 * (int64_t)i + 2] = (gz.x + gz.y) * f;
            }
        }
        return;
    }
    for (int i = t0 + threadIdx.x; i < t1; i += kLeafThreads) {
        const P x = pts[i];
        T pot = 0, gx = 0, gy = 0, gz = 0;
        for (int e = 0; e < ns; ++e) interact<T, false, YUK>(src[e], x.x, x.y, x.z, pot, gx, gy, gz, kappa);
        const T f = scale * inv4pi<T>();
        if (phi) phi[i] = pot * f + (shift ? (T)shift[b] : (T)0);   // the leaf's constant potential part
        if (GRAD) {
            grad[3 * (int64_t)i] = gx * f;
            grad[3 * (int64_t)i + 1] = gy * f;
            grad[3 * (int64_t)i + 2] = gz * f;
        }
    }
}

template <typename T>
__global__ void gather_q_kernel(const T *__restrict__ q, const int *__restrict__ perm,
                                typename Vec4<T>::type *__restrict__ pts, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) pts[i].w = q[perm[i]];
}

template <typename T>
__global__ void scatter_kernel(const T *__restrict__ near_phi, const T *__restrict__ near_grad,
                               const T *__restrict__ far_phi, const T *__restrict__ far_grad,
                               const int *__restrict__ perm, T *__restrict__ phi,
                               T *__restrict__ grad, int64_t n, int64_t n_out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = perm[i];
    if (!dbg_ok(o >= 0 && o < n_out, kDbgScatter)) return;
    if (phi) {
        T v = 0;
        if (near_phi) v += near_phi[i];
        if (far_phi) v += far_phi[i];
        phi[o] = v;
    }
    if (grad) {
        for (int a = 0; a < 3; ++a) {
            T g = 0;
            if (near_grad) g += near_grad[3 * i + a];
            if (far_grad) g += far_grad[3 * i + a];
            grad[3 * (int64_t)o + a] = g;
        }
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t launch_gather_points(const T *q_in, const int *perm, void *pts, int64_t n,
                                 cudaStream_t s) {
    gather_q_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(q_in, perm, (typename Vec4<T>::type *)pts, n); count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter(const T *near_phi, const T *near_grad, const T *far_phi,
                           const T *far_grad, const int *perm, T *phi, T *grad, int64_t n,
                           cudaStream_t s, int64_t n_out) {
    scatter_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(near_phi, near_grad, far_phi, far_grad,
                                                         perm, phi, grad, n, n_out < 0 ? n : n_out); count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p2p(const fmm_ctx *ctx, T *phi, T *grad, cudaStream_t s) {
    if (ctx->cplx) return helm_p2p<T>(ctx, phi, grad, s);
    if (ctx->nleaf == 0) return cudaSuccess;
    using P = typename Vec4<T>::type;
    const P *pts = (const P *)ctx->pts;
    const bool yuk = ctx->opt.kernel == FMM_YUKAWA;
    const T kappa = (T)ctx->opt.kappa;
    auto go = [&](auto kern, T *g) {
        kern<<<ctx->nleaf, kP2PThreads, 0, s>>>(pts, ctx->leaf_off, ctx->u_off, ctx->u_idx, ctx->p2p_order, phi, g,
                                                 kappa);
    };
    if constexpr (std::is_same<T, float>::value) {
        const LeafBoxes bx{ctx->leaf_off, (int)std::max<int64_t>(ctx->n, ctx->n_pts_all)};
        const unsigned small_grid = (unsigned)((ctx->nleaf + kSmallWarps - 1) / kSmallWarps);
        // leaves of more than kSmallLeaf points in decreasing work, the others one warp each in
        // Morton order
        auto gf = [&](auto kern, auto small, float *g) {
            kern<<<ctx->nleaf, kP2PThreads, 0, s>>>(pts, bx, ctx->u_off, ctx->u_idx, ctx->p2p_order, phi, g, kappa);
            count_launch();
            small<<<small_grid, kSmallWarps * 32, 0, s>>>(pts, bx, ctx->u_off, ctx->u_idx, nullptr, ctx->nleaf, phi, g,
                                                          kappa);
        };
        if (grad && phi)
            yuk ? gf(p2p_f32_kernel<3, true, LeafBoxes>, p2p_small_f32_kernel<3, true, LeafBoxes>, grad)
                : gf(p2p_f32_kernel<3, false, LeafBoxes>, p2p_small_f32_kernel<3, false, LeafBoxes>, grad);
        else if (grad)
            yuk ? gf(p2p_f32_kernel<kOutGrad, true, LeafBoxes>, p2p_small_f32_kernel<kOutGrad, true, LeafBoxes>, grad)
                : gf(p2p_f32_kernel<kOutGrad, false, LeafBoxes>, p2p_small_f32_kernel<kOutGrad, false, LeafBoxes>, grad);
        else
            yuk ? gf(p2p_f32_kernel<kOutPhi, true, LeafBoxes>, p2p_small_f32_kernel<kOutPhi, true, LeafBoxes>, nullptr)
                : gf(p2p_f32_kernel<kOutPhi, false, LeafBoxes>, p2p_small_f32_kernel<kOutPhi, false, LeafBoxes>, nullptr);
        (void)go;
    } else {
        if (grad) yuk ? go(p2p_kernel<T, true, true>, grad) : go(p2p_kernel<T, true, false>, grad);
        else yuk ? go(p2p_kernel<T, false, true>, nullptr) : go(p2p_kernel<T, false, false>, nullptr);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_p2p_rows_f32(const float4 *pts, int64_t n_points, const int *begin, const int *count, const int *u_off,
                                const int *u_idx, const int *order, int nrows, float *phi, float *grad,
                                cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    const RowBoxes bx{begin, count, (int)n_points};
    const unsigned small_grid = (unsigned)((nrows + kSmallWarps - 1) / kSmallWarps);
    auto go = [&](auto kern, auto small, float *g) {
        kern<<<nrows, kP2PThreads, 0, s>>>(pts, bx, u_off, u_idx, order, phi, g, 0.f);
        count_launch();
        small<<<small_grid, kSmallWarps * 32, 0, s>>>(pts, bx, u_off, u_idx, order, nrows, phi, g, 0.f);
    };
    if (grad && phi) go(p2p_f32_kernel<3, false, RowBoxes>, p2p_small_f32_kernel<3, false, RowBoxes>, grad);
    else if (grad) go(p2p_f32_kernel<kOutGrad, false, RowBoxes>, p2p_small_f32_kernel<kOutGrad, false, RowBoxes>, grad);
    else go(p2p_f32_kernel<kOutPhi, false, RowBoxes>, p2p_small_f32_kernel<kOutPhi, false, RowBoxes>, nullptr);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_check(const fmm_ctx *ctx, const T *grid, T *out, cudaStream_t s) {
    if (ctx->cplx) return helm_leaf_check<T>(ctx, grid, out, s);
    if (ctx->nleaf == 0) return cudaSuccess;
    const int d = ctx->opt.depth;
    const double width = ctx->side / (double)(1 << d);
    const double radius = 2.95 * 0.5 * width;
    const bool yuk = ctx->opt.kernel == FMM_YUKAWA;
    const T kappa = (T)ctx->opt.kappa;
    const LeafBoxes bx{ctx->leaf_off, (int)std::max<int64_t>(ctx->n, ctx->n_pts_all)};
    auto go = [&](auto kern, int threads) {
        kern<<<ctx->nleaf, threads, 0, s>>>((const typename Vec4<T>::type *)ctx->pts, bx, nullptr, ctx->lev[d].keys,
                                            grid, ctx->npts, ctx->nsp, ctx->origin[0], ctx->origin[1], ctx->origin[2],
                                            width, radius, out, kappa);
    };
    if constexpr (std::is_same<T, float>::value)
        yuk ? go(leaf_check_f32_kernel<true, LeafBoxes>, kCheckThreads)
            : go(leaf_check_f32_kernel<false, LeafBoxes>, kCheckThreads);
    else
        yuk ? go(leaf_check_kernel<T, true, LeafBoxes>, kLeafThreads) : go(leaf_check_kernel<T, false, LeafBoxes>, kLeafThreads);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_check_rows(const fmm_ctx *ctx, int level, const int *list, int n, const int *begin,
                                   const int *count, const T *grid, T *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const double width = ctx->side / (double)(1 << level);
    const double radius = 2.95 * 0.5 * width;
    const RowBoxes bx{begin, count, (int)std::max<int64_t>(ctx->n, ctx->n_pts_all)};
    auto go = [&](auto kern, int threads) {
        kern<<<n, threads, 0, s>>>((const typename Vec4<T>::type *)ctx->pts, bx, list, ctx->lev[level].keys, grid,
                                   ctx->npts, ctx->nsp, ctx->origin[0], ctx->origin[1], ctx->origin[2], width, radius,
                                   out, (T)0);
    };
    if constexpr (std::is_same<T, float>::value) go(leaf_check_f32_kernel<false, RowBoxes>, kCheckThreads);
    else go(leaf_check_kernel<T, false, RowBoxes>, kLeafThreads);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_eval(const fmm_ctx *ctx, const T *grid, const T *dens, int ldd, T scale,
                             T *phi, T *grad, cudaStream_t s, const double *shift) {
    if (ctx->cplx) return helm_leaf_eval<T>(ctx, grid, dens, ldd, phi, grad, s);   // scale 1, no shift
    if (ctx->nleaf == 0) return cudaSuccess;
    const int d = ctx->opt.depth;
    const double width = ctx->side / (double)(1 << d);
    const double radius = 2.95 * 0.5 * width;
    using P = typename Vec4<T>::type;
    size_t smem = sizeof(P) * ctx->npts * (std::is_same<T, float>::value ? 2 : 1);   // FP32: + the pair layout
    const bool yuk = ctx->opt.kernel == FMM_YUKAWA;
    const T kappa = (T)ctx->opt.kappa;
    const LeafBoxes bx{ctx->leaf_off, (int)std::max<int64_t>(ctx->n, ctx->n_pts_all)};
    auto go = [&](auto kern, T *g) {
        kern<<<ctx->nleaf, kLeafThreads, smem, s>>>((const P *)ctx->pts, bx, nullptr, ctx->lev[d].keys, grid,
                                                    ctx->npts, dens, ldd, scale, ctx->origin[0], ctx->origin[1],
                                                    ctx->origin[2], width, radius, phi, g, shift, kappa);
    };
    if (grad)
        yuk ? go(leaf_eval_kernel<T, true, true, LeafBoxes>, grad) : go(leaf_eval_kernel<T, true, false, LeafBoxes>, grad);
    else
        yuk ? go(leaf_eval_kernel<T, false, true, LeafBoxes>, nullptr)
            : go(leaf_eval_kernel<T, false, false, LeafBoxes>, nullptr);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_eval_rows(const fmm_ctx *ctx, int level, const int *list, int n, const int *begin,
                                  const int *count, const T *grid, const T *dens, int ldd, T *phi, T *grad,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const double width = ctx->side / (double)(1 << level);
    const double radius = 2.95 * 0.5 * width;
    using P = typename Vec4<T>::type;
    size_t smem = sizeof(P) * ctx->npts * (std::is_same<T, float>::value ? 2 : 1);
    const RowBoxes bx{begin, count, (int)std::max<int64_t>(ctx->n, ctx->n_pts_all)};
    auto go = [&](auto kern, T *g) {
        kern<<<n, kLeafThreads, smem, s>>>((const P *)ctx->pts, bx, list, ctx->lev[level].keys, grid, ctx->npts, dens,
                                           ldd, (T)1, ctx->origin[0], ctx->origin[1], ctx->origin[2], width, radius,
                                           phi, g, nullptr, (T)0);
    };
    if (grad) go(leaf_eval_kernel<T, true, false, RowBoxes>, grad);
    else go(leaf_eval_kernel<T, false, false, RowBoxes>, nullptr);
    count_launch();
    return cudaGetLastError();
}

#define FMM_INST(T)                                                                                \
    template cudaError_t launch_gather_points<T>(const T *, const int *, void *, int64_t, cudaStream_t); \
    template cudaError_t launch_scatter<T>(const T *, const T *, const T *, const T *, const int *,   \
                                           T *, T *, int64_t, cudaStream_t, int64_t);               \
    template cudaError_t launch_p2p<T>(const fmm_ctx *, T *, T *, cudaStream_t);                    \
    template cudaError_t launch_leaf_check<T>(const fmm_ctx *, const T *, T *, cudaStream_t);       \
    template cudaError_t launch_leaf_check_rows<T>(const fmm_ctx *, int, const int *, int, const int *, \
                                                   const int *, const T *, T *, cudaStream_t);      \
    template cudaError_t launch_leaf_eval_rows<T>(const fmm_ctx *, int, const int *, int, const int *, \
                                                  const int *, const T *, const T *, int, T *, T *, cudaStream_t); \
    template cudaError_t launch_leaf_eval<T>(const fmm_ctx *, const T *, const T *, int, T, T *, T *, \
                                             cudaStream_t, const double *);
FMM_INST(float)
FMM_INST(double)
#undef FMM_INST

FMM_DEBUG_UNIT(p2p)

}  // namespace fmm
