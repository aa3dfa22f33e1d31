// Tensor-core (tcgen05, sm_103a) form of the gathered GEMM of gemm_common.cuh, with split-
// precision operands: the FP32 inputs are split into BF16 (hi, lo[, mid]) or TF32 (big, small)
// planes and the products a_i b_j with i + j below the split order are accumulated in FP32 in
// tensor memory.  This carries the surface contractions and the M2L (VLI) of the FMM.
//
// Layout.  One CTA computes a 128-row tile (M = 128 boxes) for all N output columns.  The K
// dimension of every segment is cut into chunks of one 128-byte swizzle atom (64 BF16 or 32
// TF32 values).  A stage holds the A planes (128 rows x 128 B each, K-major, SWIZZLE_128B:
// 16-byte unit j of row r sits at (j ^ (r % 8)) * 16 within the row's 128 bytes, rows 128 B
// apart, 8-row groups 1024 B apart) and the B planes (N rows, same layout).  B (the operator) is
// stored in global memory already in this layout, chunk by chunk, so one bulk copy per stage
// moves it; A rows are gathered by the producer warps, split and written with st.shared.
//
// Warp roles (256 threads, two warps per SM sub-partition so that the accumulator warps can hold
// 160 FP32 partial sums in registers): warps 4-7 drain the tensor memory accumulators (warp w
// owns TMEM lanes 32(w-4).. = tile rows) into FP32 registers and write Y; warp 0 owns the tensor
// memory allocation.  A rows from FP32 (gathered and split in registers): warps 0-3 produce the
// stages and lane 0 of warp 4 issues every tcgen05.mma (item i), after which its warp drains item
// i - 1.  A rows from split planes (copies only): warps 0-2 produce and lane 0 of warp 3 issues,
// so the tensor pipe keeps running while all four accumulator warps drain (issuing an item's
// MMAs takes as long as the tensor pipe needs for them).
//
// Accumulation.  The tensor core adds an MMA's products into the FP32 accumulator with
// truncation, so a long chain of MMAs into one accumulator drifts toward zero by about one
// half-ulp per step.  Every stage (at most 4 k-steps x the split products) therefore gets a
// fresh accumulator (two alternate in tensor memory) and its partial sum is added, correctly
// rounded, into registers of the accumulator warps.  A CTA covers at most 160 output columns;
// wider outputs are split over blockIdx.y.
//
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the kernel records an error
// code in a device flag, stops producing/issuing, still releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gemm_common.cuh"

namespace fmm {

constexpr int kTcThreads = 256;           // 4 producer warps, 4 accumulator warps (one issues MMAs)
constexpr int kTcRows = 128;
constexpr int kTcMaxN = 160;               // output columns per CTA (wider N: several CTAs)
constexpr int kAtomBytes = 128;            // one swizzle atom row
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr int kPlaneProducers = 96;        // plane mode: warps 0-2 copy, warp 3 issues the MMAs
constexpr int kPlaneStages = 2;            // plane mode: stages in shared memory

struct TcDev {
    GemmDev g;                      // gather description (W fields unused)
    const unsigned char *Wt0;       // tensor-core operand of segment 0 (or of segment index * stride)
    long long wt_stride;            // bytes between consecutive operators (CHILDREN, STENCIL)
    const unsigned char *Wt1[8];    // PARENT2 segment 1 by class
    int nplanes;                    // 2 (x3) or 3 (x6)
    int tf32;                       // 1: kind::tf32 planes (4-byte); 0: BF16 planes (2-byte)
    int nprod;                      // products per k-step
    int prod_a[6], prod_b[6];       // plane pairs
    int nstages;
    int ncta;                       // output columns per CTA (grid.y splits wider N)
    int tmem_cols;
    int *err;                       // device error flag
    unsigned long long wait_ns;     // bound on every pipeline barrier wait (default 1 s)
    // Segment accumulation (plane layout): all K chunks of one segment go into one of three
    // accumulators, drained once per segment; the rows and operators then carry one FP16 scale
    // each (uniform over their chunks).
    int seg_acc;
    int yp_row_scale;               // FP16 output planes: one scale per row (every chunk's entry equal)
    int a_planes;                   // A rows arrive pre-split from xp (cp.async copies)
    const unsigned char *xp;        // split planes of the A rows
    long long xp_plane;             // bytes between planes
    int xp_ld;                      // row stride in elements
    unsigned char *yp;              // split-plane output (instead of FP32 Y) if non-null
    long long yp_plane;             // bytes between output planes
    int yp_ld;                      // output row stride in elements
    // FP16 operands (FMM_FP16X3 stencil): power-of-two scaled hi/lo planes; the partial sum of
    // every stage item is multiplied by a_scale[src row][chunk] * b_scale[operator][chunk]
    int f16;
    const float *a_scale;
    int a_scale_ld;
    const float *b_scale;
    int b_scale_ld;
    // PARENT2 segment 1 (the parent rows): its own planes, row scales and, per octant class,
    // operator scales
    const unsigned char *xp1;
    long long xp1_plane;
    int xp1_ld;
    const float *a_scale1;
    int a_scale1_ld;
    const float *b_scale1;
    int b_scale1_ld;
    // FP16 output planes: each row scaled by a power of two per 64-column chunk, 1 / scale
    // written to yp_scale[row][chunk]
    int yp_f16;
    float *yp_scale;
    int yp_scale_ld;
};

namespace {

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the barrier's phase with the given parity has completed; false once limit_ns of
// %globaltimer have passed (checked every 16 polls; a limit of 0 gives up at the first poll
// that finds the phase incomplete).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint32_t a = smem_u32(bar);
    uint32_t ready = 0;   // a phase that is already complete costs one non-blocking probe
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ready)
        : "r"(a), "r"(parity)
        : "memory");
    if (ready) return true;
    // Each poll may suspend the thread until the phase completes (at most `hint` ns), so that
    // waiting warps take no issue slots from the warps they wait for on the same SM
    // sub-partition (the MMA issuer above all).
    const uint32_t hint = limit_ns < 1000000ull ? (uint32_t)limit_ns : 1000000u;
    uint32_t done = 0;
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(hint)
            : "memory");
        if (done) return true;
        if (limit_ns == 0) return false;
        if (it == 0) t0 = global_ns();
        else if ((it & 15) == 0 && global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte asynchronous global -> shared copy; src_bytes < 16 zero-fills the rest
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// arrive on the barrier once all of this thread's earlier cp.async copies have completed
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// wait for all of this thread's cp.async copies (the hardware tracks them; no polling)
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// K-major, SWIZZLE_128B shared-memory matrix descriptor: start address, LBO = 16 B (unused for
// this layout), SBO = 1024 B between 8-row groups, version 1, layout type 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: D = F32, A/B format (1 = BF16 for kind::f16, 2 = TF32 for kind::tf32),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128).
__device__ __forceinline__ uint32_t make_idesc(int n, int fmt) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive columns of this thread's TMEM lane (no wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- splits
__device__ __forceinline__ uint32_t bf16_bits(float x) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint32_t b) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
}
__device__ __forceinline__ uint32_t tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r & 0xffffe000u;   // keep the 10 explicit mantissa bits only
}

// Teardown: wait (at most 1 s each) until the operator copies this thread started have landed,
// so that no copy is still writing into shared memory when the CTA exits, also after an abort.
__device__ __forceinline__ bool wait_bulk_copies(uint64_t *bulk_bar, const int *started, int nstages) {
    bool ok = true;
    for (int s = 0; s < nstages; ++s)
        if (started[s] > 0) ok = mbar_wait(&bulk_bar[s], (uint32_t)(started[s] - 1) & 1u, kWaitNs) && ok;
    return ok;
}

// ---------------------------------------------------------------- work list helpers
struct SegInfo {
    const float *X;
    int ldx, K;
    const unsigned char *Wt;
    int nchunks;
};

// Per-tile tables held in shared memory: the operator index and the transfer vector of every
// class slot of the tile's octant class (stencil mode), so that moving to the next segment
// needs no dependent global loads.
struct TileTables {
    int slot[kClassSlots];
    int delta[kClassSlots];
};

__device__ __forceinline__ long long w_index_fast(const GemmDev &g, const Tile &t, const TileTables &tt, int seg) {
    return g.mode == GM_STENCIL ? (long long)tt.slot[seg] : gemm_w_index(g, t, seg);
}

__device__ __forceinline__ SegInfo seg_info(const TcDev &p, const Tile &t, const TileTables &tt, int seg,
                                            int chunk_elems) {
    SegInfo s;
    const GemmDev &g = p.g;
    const bool second = g.mode == GM_PARENT2 && seg == 1;
    s.X = (const float *)(second ? g.X1 : g.X0);
    s.ldx = second ? g.ldx1 : g.ldx0;
    s.K = second ? g.k1 : g.k0;
    s.Wt = second ? p.Wt1[t.cls] : p.Wt0 + w_index_fast(g, t, tt, seg) * p.wt_stride;
    s.nchunks = (s.K + chunk_elems - 1) / chunk_elems;
    return s;
}

// One tile row: its box and, for the stencil, the box's integer coordinates.
struct RowRef {
    int box, ax, ay, az;
};

__device__ __forceinline__ RowRef row_ref(const GemmDev &g, int box) {
    RowRef r{box, 0, 0, 0};
    if (box >= 0 && g.mode == GM_STENCIL) demorton3(g.keys[box], r.ax, r.ay, r.az);
    return r;
}

// source row of (row, seg), -1 for none (one global load: the dense table or the child/parent table)
__device__ __forceinline__ int src_fast(const GemmDev &g, const Tile &t, const TileTables &tt, const RowRef &r,
                                        int seg) {
    if (r.box < 0) return -1;
    if (g.mode == GM_STENCIL) {
        int dx, dy, dz;
        unpack_delta(tt.delta[seg], dx, dy, dz);
        return dense_find(g.dense, g.level, r.ax + dx, r.ay + dy, r.az + dz);
    }
    return gemm_src_row(g, t, r.box, seg);
}


}  // namespace

// The kernel body.  PL (plane layout, A rows from split planes): 384 threads, warps 0-2
// produce, warp 3 issues, warps 4-11 drain, two per TMEM lane quarter, each holding half of the
// row's columns (80), so that a CTA needs about half the registers of the 256-thread layout and
// near-field CTAs can share its SM.  Otherwise: 256 threads, warps 0-3 gather and split A in
// registers, warps 4-7 drain whole rows (warp 4 also issues).
template <bool TF32, bool PL>
__device__ __forceinline__ void tc_body(const TcDev &p) {
    constexpr int NT = PL ? 384 : kTcThreads;        // threads
    constexpr int DC = PL ? kTcMaxN / 2 : kTcMaxN;   // columns a drain thread holds
    constexpr int NDRAIN = PL ? 8 : 4;               // drain warps
    extern __shared__ unsigned char smem_raw[];
    // full: the producers' A rows of a stage; bulk: its operator copy; empty: the stage's MMAs
    // done; tfull / tempty: an accumulator's MMAs done / drained; fin: every MMA of the CTA done
    __shared__ uint64_t full_bar[4], bulk_bar[4], empty_bar[4], tfull_bar[3], tempty_bar[3], fin_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int box[kTcRows];
    __shared__ int srcs[2][kTcRows];
    __shared__ int plist[2][kTcRows + 1];   // rows with a source row ([kTcRows] = their count)
    __shared__ uint32_t mask[6];
    __shared__ int abort_flag;
    __shared__ TileTables tt;
    __shared__ float pmax[2][(kTcMaxN + 63) / 64][kTcRows];   // PL: the halves' chunk maxima of each row

    const GemmDev &g = p.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Tile t = g.tiles[blockIdx.x];
    const int n_lo = blockIdx.y * p.ncta;                 // this CTA's output columns
    const int N = min(p.ncta, g.n_out - n_lo);            // multiple of 16
    constexpr int esz = TF32 ? 4 : 2;                     // bytes per plane element
    constexpr int chunk_elems = kAtomBytes / esz;         // K values per stage
    const int a_plane_bytes = kTcRows * kAtomBytes;       // 16 KB
    const int b_plane_bytes = N * kAtomBytes;
    const int stage_bytes = p.nplanes * (a_plane_bytes + p.ncta * kAtomBytes);
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    if (tid == 0) {
        for (int s = 0; s < p.nstages; ++s) {
            // register gather: 4 producer warps; plane copies: 96 cp.async arrivals (3 producer warps)
            mbar_init(&full_bar[s], p.a_planes ? kPlaneProducers : 4);
            mbar_init(&bulk_bar[s], 1);       // thread 0's expect_tx arrive, then the copy's bytes
            mbar_init(&empty_bar[s], 1);      // tcgen05.commit
        }
        mbar_init(&fin_bar, 1);               // tcgen05.commit after the last MMA
        for (int b = 0; b < 3; ++b) {
            mbar_init(&tfull_bar[b], 1);      // tcgen05.commit
            mbar_init(&tempty_bar[b], NDRAIN);   // the accumulator warps
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 6) mask[tid] = g.mode == GM_STENCIL ? g.masks[(size_t)t.mask * 6 + tid] : 0xffffffffu;
    if (tid < kTcRows) box[tid] = tid < t.nrows ? gemm_row_box(g, t, tid) : -1;
    if (g.mode == GM_STENCIL)
        for (int k = tid; k < kClassSlots; k += NT) {
            tt.slot[k] = g.class_slots[t.cls * kClassSlots + k];
            tt.delta[k] = g.class_delta[t.cls * kClassSlots + k];
        }
    // Rows and K units that are never copied keep what the stage held before: zero the stages
    // once so that they hold finite values (their products are then multiplied by zero).
    const bool scaled_a = p.a_planes && p.a_scale != nullptr;
    if (scaled_a)
        for (int i = tid; i < p.nstages * stage_bytes / 16; i += NT)
            reinterpret_cast<uint4 *>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tmem_alloc(&tmem_base, p.tmem_cols);
    fence_proxy_async();   // the zeroed stages (generic proxy) before any tensor-core read
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = make_idesc(N, TF32 ? 2 : (p.f16 ? 0 : 1));   // kind::f16: 0 = FP16, 1 = BF16
    const int nseg = gemm_nseg(g);
    auto active = [&](int seg) { return g.mode != GM_STENCIL || ((mask[seg >> 5] >> (seg & 31)) & 1u); };
    // number of stage items (segment chunks) and of active segments of the tile
    int n_items = 0, n_segs = 0;
    for (int seg = 0; seg < nseg; ++seg)
        if (active(seg)) n_items += (gemm_seg_k(g, seg) + chunk_elems - 1) / chunk_elems, ++n_segs;
    // accumulator uses: one per item, or one per segment with segment accumulation
    const int nacc = p.seg_acc ? 3 : 2;
    const int n_units = p.seg_acc ? n_segs : n_items;
    // the split products (plane pairs), held in registers
    int pa[6], pb[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) pa[i] = p.prod_a[i], pb[i] = p.prod_b[i];

    // One stage item's MMAs into accumulator b, issued by one thread: the split products of the
    // chunk, then commits that free the stage and (after the last chunk of the accumulation)
    // mark the accumulator full.  `first` starts the accumulator afresh.
    auto issue_item = [&](int stage, int b, const SegInfo &si, int chunk, bool first, bool last) {
        tc_fence_after();
        fence_proxy_async();   // cp.async / st.shared writes (generic proxy) -> tcgen05.mma
        const uint32_t sa = smem_u32(base + (size_t)stage * stage_bytes);
        const uint32_t sb = sa + p.nplanes * a_plane_bytes;
        const uint32_t dt = tmem + (uint32_t)(b * p.ncta);
        const int kval = min(chunk_elems, si.K - chunk * chunk_elems);
        const int ksteps = min(kAtomBytes / 32, (kval * esz + 31) / 32);
        // descriptors of the stage's planes; a K step of 32 bytes adds 2 to the address field
        const uint64_t a0 = sw128_desc(sa), b0 = sw128_desc(sb);
        uint32_t accum = first ? 0u : 1u;
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            if (pr >= p.nprod) break;
            const uint64_t ap = a0 + (uint64_t)((pa[pr] * a_plane_bytes) >> 4);
            const uint64_t bp = b0 + (uint64_t)((pb[pr] * b_plane_bytes) >> 4);
            for (int ks = 0; ks < ksteps; ++ks) {
                if (TF32) mma_tf32(dt, ap + 2 * ks, bp + 2 * ks, idesc, accum);
                else mma_bf16(dt, ap + 2 * ks, bp + 2 * ks, idesc, accum);
                accum = 1;
            }
        }
        mma_commit(&empty_bar[stage]);
        if (last) mma_commit(&tfull_bar[b]);
    };

    if (warp < 3 && p.a_planes) {
        // ------------------------------------------------------------ producers, split planes
        // The source rows are already split into planes in global memory, so the producers only
        // copy: every thread issues 16-byte cp.async copies straight into the swizzled stage
        // (8 lanes per row, 4 rows per warp instruction, zero fill for missing rows), then
        // arrives on the stage barrier when its copies have landed.
        // Thread 0 adds the operator's bulk copy.  Copies of several stages stay in flight.
        // Every producer thread runs the same segment loop and the same named barrier per active
        // segment whatever happens; after a failed (bounded) wait it only skips its copies.
        // The source row of the next active segment is looked up while the current one is copied.
        // Three warps (96 threads) cover the 128 rows: thread i looks up rows i and i + 96.
        int item = 0, sidx = 0;
        int bulk_started[4] = {0, 0, 0, 0};   // operator copies thread 0 started per stage
        bool ok = true;
        const bool two = tid + kPlaneProducers < kTcRows;
        const RowRef me = row_ref(g, box[tid]);
        const RowRef me2 = row_ref(g, two ? box[tid + kPlaneProducers] : -1);
        int seg = 0;
        while (seg < nseg && !active(seg)) ++seg;
        int src_next = seg < nseg ? src_fast(g, t, tt, me, seg) : -1;
        int src_next2 = seg < nseg ? src_fast(g, t, tt, me2, seg) : -1;
        for (; seg < nseg;) {
            int seg2 = seg + 1;
            while (seg2 < nseg && !active(seg2)) ++seg2;
            const SegInfo si = seg_info(p, t, tt, seg, chunk_elems);
            srcs[sidx][tid] = src_next;
            if (two) srcs[sidx][tid + kPlaneProducers] = src_next2;
            asm volatile("bar.sync 1, 96;" ::: "memory");
            if (scaled_a && warp == 0) {
                // rows that have a source, compacted, so that every copy instruction carries full
                // rows (rows without one are multiplied by zero in the drain and are not copied)
                int cnt = 0;
#pragma unroll
                for (int r0 = 0; r0 < kTcRows; r0 += 32) {
                    const bool has = srcs[sidx][r0 + lane] >= 0;
                    const unsigned m = __ballot_sync(0xffffffffu, has);
                    if (has) plist[sidx][cnt + __popc(m & ((1u << lane) - 1u))] = r0 + lane;
                    cnt += __popc(m);
                }
                if (lane == 0) plist[sidx][kTcRows] = cnt;
            }
            if (scaled_a) asm volatile("bar.sync 1, 96;" ::: "memory");
            src_next = seg2 < nseg ? src_fast(g, t, tt, me, seg2) : -1;
            src_next2 = seg2 < nseg ? src_fast(g, t, tt, me2, seg2) : -1;
            const int *rs = srcs[sidx];
            const int unit = lane & 7;
            const bool seg_second = g.mode == GM_PARENT2 && seg == 1;   // parent rows
            const unsigned char *xpb = seg_second ? p.xp1 : p.xp;
            const long long xpp = seg_second ? p.xp1_plane : p.xp_plane;
            const int xld = seg_second ? p.xp1_ld : p.xp_ld;
            for (int c = 0; c < si.nchunks; ++c, ++item) {
                const int stage = item % p.nstages;
                if (!ok) continue;
                if ((item >= p.nstages && !mbar_wait(&empty_bar[stage], ((item / p.nstages) - 1) & 1, p.wait_ns)) ||
                    *(volatile int *)&abort_flag) {
                    ok = false;
                    continue;
                }
                unsigned char *sa = base + (size_t)stage * stage_bytes;
                unsigned char *sb = sa + p.nplanes * a_plane_bytes;
                if (tid == 0) {
                    mbar_arrive_tx(&bulk_bar[stage], (uint32_t)(p.nplanes * b_plane_bytes));
                    ++bulk_started[stage];
                    const size_t plane_full = (size_t)g.n_out * kAtomBytes;
                    if ((size_t)b_plane_bytes == plane_full)   // the chunk's planes are contiguous: one copy
                        bulk_g2s(sb, si.Wt + (size_t)c * p.nplanes * plane_full,
                                 (uint32_t)(p.nplanes * b_plane_bytes), &bulk_bar[stage]);
                    else
                        for (int pl = 0; pl < p.nplanes; ++pl)
                            bulk_g2s(sb + pl * b_plane_bytes,
                                     si.Wt + ((size_t)c * p.nplanes + pl) * plane_full + (size_t)n_lo * kAtomBytes,
                                     (uint32_t)b_plane_bytes, &bulk_bar[stage]);
                }
                const int k0 = c * chunk_elems;
                const int kval = min(chunk_elems, si.K - k0);
                const int valid_units = (kval * esz + 15) / 16;
                const bool unit_ok = unit < valid_units;
                if (scaled_a) {
                    // (present row, valid 16-byte unit) pairs, consecutive over the producers
                    const int *pl_rows = plist[sidx];
                    const int total = pl_rows[kTcRows] * valid_units;
                    for (int e = tid; e < total; e += kPlaneProducers) {
                        const int r = pl_rows[e / valid_units], u = e % valid_units;
                        const size_t elem = (size_t)rs[r] * xld + k0 + u * (16 / esz);
                        const int dst_off = r * kAtomBytes + ((u ^ (r & 7)) << 4);
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl)
                            if (pl < p.nplanes)
                                cp_async16(sa + pl * a_plane_bytes + dst_off, xpb + pl * xpp + elem * esz, 16);
                    }
                    cp_async_arrive(&full_bar[stage]);
                    continue;
                }
#pragma unroll
                for (int j = 0; j < (kTcRows + 11) / 12; ++j) {   // 12 rows per pass of 3 warps
                    const int r = j * 12 + warp * 4 + (lane >> 3);
                    if (r >= kTcRows) break;
                    const int sr = rs[r];
                    const bool have = unit_ok && sr >= 0;
                    // with per-row factors (scaled planes) a row without a source is multiplied by
                    // zero in the drain, so it needs no copy; K units past the segment are never read
                    if (!have && (scaled_a || !unit_ok)) continue;
                    const size_t elem = (size_t)(have ? sr : 0) * xld + k0 + unit * (16 / esz);
                    const int dst_off = r * kAtomBytes + ((unit ^ (r & 7)) << 4);
#pragma unroll
                    for (int pl = 0; pl < 3; ++pl) {
                        if (pl < p.nplanes)
                            cp_async16(sa + pl * a_plane_bytes + dst_off, xpb + pl * xpp + elem * esz,
                                       have ? 16 : 0);
                    }
                }
                cp_async_arrive(&full_bar[stage]);
            }
            sidx ^= 1;
            seg = seg2;
        }
        if (!ok) {
            atomicExch(p.err, FMM_ETIMEOUT);
            *(volatile int *)&abort_flag = 1;
        }
        // nothing of this thread's may still be in flight when the CTA exits
        cp_async_wait_all();
        if (tid == 0 && !wait_bulk_copies(bulk_bar, bulk_started, p.nstages)) atomicExch(p.err, FMM_ETIMEOUT);
    } else if (warp == 3 && p.a_planes) {
        // ------------------------------------------------------------ MMA issuer (plane mode)
        // A warp of its own issues the MMAs, so the tensor pipe runs while the accumulator
        // warps drain: the issue of an item's MMAs returns only as the tensor pipe takes them.
        if (lane == 0) {
            bool ok = true;
            int seg = 0, chunk = 0, seg_ord = 0;
            while (seg < nseg && !active(seg)) ++seg;
            SegInfo si{};
            if (seg < nseg) si = seg_info(p, t, tt, seg, chunk_elems);
            for (int item = 0; item < n_items; ++item) {
                const int stage = item % p.nstages;
                const bool first = !p.seg_acc || chunk == 0, last = !p.seg_acc || chunk + 1 == si.nchunks;
                const int u = p.seg_acc ? seg_ord : item, b = u % nacc;   // accumulator use
                if (!mbar_wait(&full_bar[stage], (item / p.nstages) & 1, p.wait_ns) ||
                    !mbar_wait(&bulk_bar[stage], (item / p.nstages) & 1, p.wait_ns) ||
                    (first && u >= nacc && !mbar_wait(&tempty_bar[b], ((u / nacc) - 1) & 1, p.wait_ns)) ||
                    *(volatile int *)&abort_flag) {
                    ok = false;
                    break;
                }
                issue_item(stage, b, si, chunk, first, last);
                if (last) ++seg_ord;
                if (++chunk == si.nchunks) {
                    chunk = 0;
                    ++seg;
                    while (seg < nseg && !active(seg)) ++seg;
                    if (seg < nseg) si = seg_info(p, t, tt, seg, chunk_elems);
                }
            }
            if (!ok) {
                atomicExch(p.err, FMM_ETIMEOUT);
                *(volatile int *)&abort_flag = 1;
            }
            // every MMA issued (also before an abort) completes before the tensor memory is freed
            mma_commit(&fin_bar);
            if (!mbar_wait(&fin_bar, 0, kWaitNs)) atomicExch(p.err, FMM_ETIMEOUT);
        }
    } else if (!PL && warp < 4) {
        // ------------------------------------------------------------ producers
        int item = 0;
        int bulk_started[4] = {0, 0, 0, 0};   // operator copies thread 0 started per stage
        bool ok = true;
        const RowRef me = row_ref(g, box[tid]);
        int seg0 = 0;
        while (seg0 < nseg && !active(seg0)) ++seg0;
        int src_next = seg0 < nseg ? src_fast(g, t, tt, me, seg0) : -1;
        for (int seg = seg0; seg < nseg && ok;) {
            int seg2 = seg + 1;
            while (seg2 < nseg && !active(seg2)) ++seg2;
            const SegInfo si = seg_info(p, t, tt, seg, chunk_elems);
            // source row of this warp's rows (row 32 * warp + lane), shared by shuffles; the
            // next segment's is looked up now
            const int my_src = src_next;
            src_next = seg2 < nseg ? src_fast(g, t, tt, me, seg2) : -1;
            for (int c = 0; c < si.nchunks; ++c, ++item) {
                const int stage = item % p.nstages;
                if (item >= p.nstages && !mbar_wait(&empty_bar[stage], ((item / p.nstages) - 1) & 1, p.wait_ns)) {
                    ok = false;
                    break;
                }
                if (*(volatile int *)&abort_flag) { ok = false; break; }
                unsigned char *sa = base + (size_t)stage * stage_bytes;
                unsigned char *sb = sa + p.nplanes * a_plane_bytes;
                if (tid == 0) {
                    // rows [n_lo, n_lo + N) of every plane of chunk c: contiguous per plane, and
                    // all planes contiguous when the CTA covers every row (one copy then)
                    mbar_arrive_tx(&bulk_bar[stage], (uint32_t)(p.nplanes * b_plane_bytes));
                    ++bulk_started[stage];
                    const size_t plane_full = (size_t)g.n_out * kAtomBytes;
                    if ((size_t)b_plane_bytes == plane_full)
                        bulk_g2s(sb, si.Wt + (size_t)c * p.nplanes * plane_full,
                                 (uint32_t)(p.nplanes * b_plane_bytes), &bulk_bar[stage]);
                    else
                        for (int pl = 0; pl < p.nplanes; ++pl)
                            bulk_g2s(sb + pl * b_plane_bytes,
                                     si.Wt + ((size_t)c * p.nplanes + pl) * plane_full + (size_t)n_lo * kAtomBytes,
                                     (uint32_t)b_plane_bytes, &bulk_bar[stage]);
                }
                // gather: each warp covers its 32 rows; lanes split a row into 16-byte pieces.
                // All loads of the warp are issued before any is used (memory-level parallelism).
                const int k0 = c * chunk_elems;
                const int kval = min(chunk_elems, si.K - k0);       // valid K values in this chunk
                constexpr int per_row = chunk_elems / 4;            // float4 loads per row
                constexpr int rows_per_pass = 32 / per_row;
                constexpr int passes = 32 / rows_per_pass;
                const int my_row_in_pass = lane / per_row, my_q = lane % per_row;
                const int k = my_q * 4;                             // first of 4 values
                float4 vbuf[passes];
#pragma unroll
                for (int ps = 0; ps < passes; ++ps) {
                    const int r = warp * 32 + ps * rows_per_pass + my_row_in_pass;
                    const int sr = __shfl_sync(0xffffffffu, my_src, r - warp * 32);
                    vbuf[ps] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (sr >= 0 && k < kval)
                        vbuf[ps] = __ldg(reinterpret_cast<const float4 *>(si.X + (size_t)sr * si.ldx + k0 + k));
                }
#pragma unroll
                for (int ps = 0; ps < passes; ++ps) {
                    const int r = warp * 32 + ps * rows_per_pass + my_row_in_pass;
                    const float x[4] = {vbuf[ps].x, vbuf[ps].y, vbuf[ps].z, vbuf[ps].w};
                    const int rowoff = (r >> 3) * 1024 + (r & 7) * 128;
                    if (!TF32) {
                        // 4 BF16 values = 8 bytes: half of a 16-byte unit
                        const int unit = k >> 3, half = (k >> 2) & 1;
                        const int off = rowoff + ((unit ^ (r & 7)) << 4) + half * 8;
                        uint32_t hb[4], lb[4], mb[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            hb[i] = bf16_bits(x[i]);
                            const float r1 = x[i] - bf16_val(hb[i]);
                            lb[i] = bf16_bits(r1);
                            mb[i] = bf16_bits(r1 - bf16_val(lb[i]));
                        }
                        // plane order: 0 = hi, 1 = lo, 2 = third term
                        *reinterpret_cast<uint2 *>(sa + off) = make_uint2(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16));
                        *reinterpret_cast<uint2 *>(sa + a_plane_bytes + off) =
                            make_uint2(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16));
                        if (p.nplanes == 3)
                            *reinterpret_cast<uint2 *>(sa + 2 * a_plane_bytes + off) =
                                make_uint2(mb[0] | (mb[1] << 16), mb[2] | (mb[3] << 16));
                    } else {
                        // 4 TF32 values = one 16-byte unit
                        const int unit = k >> 2;
                        const int off = rowoff + ((unit ^ (r & 7)) << 4);
                        uint32_t bb[4], ss[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            bb[i] = tf32_round(x[i]);
                            ss[i] = tf32_round(x[i] - __uint_as_float(bb[i]));
                        }
                        *reinterpret_cast<uint4 *>(sa + off) = make_uint4(bb[0], bb[1], bb[2], bb[3]);
                        *reinterpret_cast<uint4 *>(sa + a_plane_bytes + off) = make_uint4(ss[0], ss[1], ss[2], ss[3]);
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_bar[stage]);
            }
            seg = seg2;
        }
        if (!ok) {
            atomicExch(p.err, FMM_ETIMEOUT);
            *(volatile int *)&abort_flag = 1;
        }
        if (tid == 0 && !wait_bulk_copies(bulk_bar, bulk_started, p.nstages)) atomicExch(p.err, FMM_ETIMEOUT);
    } else {
        // ------------------------------------------------------------ accumulators / epilogue
        // Each stage item's products land in one of two TMEM accumulators; these warps add the
        // item's partial sums (32 rows each) into FP32 registers, so that no TMEM accumulator
        // takes more than one stage of tensor-core additions.
        const int q = (warp - 4) & 3;                     // TMEM lane quarter
        const int hf = PL ? (warp - 4) >> 2 : 0;          // column half (PL)
        const int c0 = hf * DC;                           // first column this thread holds
        const bool issuer = !PL && warp == 4;             // PL: warp 3 issues
        float acc[DC];
#pragma unroll
        for (int i = 0; i < DC; ++i) acc[i] = 0.f;
        bool ok = true;
        // Scaled FP16 operands: the factor of every item for this thread's row.  The walk keeps
        // the source row of the current and the next active segment, so that every load behind
        // a factor is issued at least one item before the factor is used.
        const bool scaled = p.a_scale != nullptr;
        const int my_row = q * 32 + lane;
        const int my_box = my_row < t.nrows ? box[my_row] : -1;
        auto next_active = [&](int sg) {
            ++sg;
            while (sg < nseg && !active(sg)) ++sg;
            return sg;
        };
        const RowRef me = row_ref(g, scaled ? my_box : -1);
        auto src_of = [&](int sg) { return sg < nseg ? src_fast(g, t, tt, me, sg) : -1; };
        auto factor = [&](int src, int sg, int ch) -> float {
            if (!scaled || sg >= nseg) return 1.f;
            if (g.mode == GM_PARENT2 && sg == 1) {   // parent rows, operator of the tile's class
                const float fb1 = __ldg(p.b_scale1 + t.cls * p.b_scale1_ld + ch);
                return src >= 0 ? __ldg(p.a_scale1 + (size_t)src * p.a_scale1_ld + ch) * fb1 : 0.f;
            }
            const float fb = __ldg(p.b_scale + w_index_fast(g, t, tt, sg) * p.b_scale_ld + ch);
            return src >= 0 ? __ldg(p.a_scale + (size_t)src * p.a_scale_ld + ch) * fb : 0.f;
        };
        int d_seg = next_active(-1), d_next = next_active(d_seg), d_chunk = 0;
        int d_src = scaled ? src_of(d_seg) : -1, d_src_next = scaled ? src_of(d_next) : -1;
        float f_cur = factor(d_src, d_seg, 0);
        auto advance = [&]() -> float {   // step to the next unit; its factor, loads issued now
            if (d_seg >= nseg) return 1.f;
            if (p.seg_acc || ++d_chunk * chunk_elems >= gemm_seg_k(g, d_seg)) {
                d_chunk = 0;
                d_seg = d_next;
                d_next = next_active(d_seg);
                d_src = d_src_next;
                d_src_next = scaled ? src_of(d_next) : -1;
            }
            return factor(d_src, d_seg, d_chunk);
        };
        auto drain = [&](int unit) -> bool {   // one accumulator use: an item, or a segment
            const float f = f_cur;
            f_cur = advance();
            const int b = unit % nacc;
            if (!mbar_wait(&tfull_bar[b], (unit / nacc) & 1, p.wait_ns)) return false;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * p.ncta);
            if constexpr (PL) {
#pragma unroll
                for (int n0 = 0; n0 < DC; n0 += 16) {
                    if (c0 + n0 < N) {   // N is a multiple of 16
                        float v[16];
                        tmem_ld16(ta + (uint32_t)(c0 + n0), v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) acc[n0 + i] = fmaf(f, v[i], acc[n0 + i]);
                    }
                }
            } else {
#pragma unroll
                for (int n0 = 0; n0 < kTcMaxN; n0 += 32) {
                    if (n0 < N) {
                        uint32_t v[32];
                        tmem_ld32(ta + (uint32_t)n0, v);
                        tmem_wait_ld();
                        // N is a multiple of 16: the upper half of the last load may be past N
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (n0 + i < kTcMaxN && (i < 16 || n0 + 16 < N))
                                acc[n0 + i] = fmaf(f, __uint_as_float(v[i]), acc[n0 + i]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty_bar[b]);
            return true;
        };
        if (!issuer) {
            for (int u = 0; u < n_units && ok; ++u) ok = drain(u);
        } else {
            // lane 0 issues item i; the whole warp then drains item i - 1 while item i runs
            int seg = 0, chunk = 0;
            while (seg < nseg && !active(seg)) ++seg;
            SegInfo si{};
            if (seg < nseg) si = seg_info(p, t, tt, seg, chunk_elems);
            for (int item = 0; item < n_items && ok; ++item) {
                int good = 1;
                if (lane == 0) {
                    const int stage = item % p.nstages, b = item & 1;
                    if (!mbar_wait(&full_bar[stage], (item / p.nstages) & 1, p.wait_ns) ||
                        !mbar_wait(&bulk_bar[stage], (item / p.nstages) & 1, p.wait_ns) ||
                        (item >= 2 && !mbar_wait(&tempty_bar[b], ((item >> 1) - 1) & 1, p.wait_ns)) ||
                        *(volatile int *)&abort_flag) {
                        good = 0;
                    } else {
                        issue_item(stage, b, si, chunk, true, true);
                        if (++chunk == si.nchunks) {
                            chunk = 0;
                            ++seg;
                            while (seg < nseg && !active(seg)) ++seg;
                            if (seg < nseg) si = seg_info(p, t, tt, seg, chunk_elems);
                        }
                    }
                }
                ok = __shfl_sync(0xffffffffu, good, 0) != 0;
                if (ok && item >= 1) ok = drain(item - 1);
            }
            if (ok && n_items >= 1) ok = drain(n_items - 1);
            // every MMA issued (also before an abort) completes before the tensor memory is freed
            if (lane == 0) {
                mma_commit(&fin_bar);
                if (!mbar_wait(&fin_bar, 0, kWaitNs)) atomicExch(p.err, FMM_ETIMEOUT);
            }
            __syncwarp();
        }
        // epilogue: this thread's row (q * 32 + lane) and columns [c0, c0 + DC)
        const int row = q * 32 + lane;
        const int b = row < t.nrows ? box[row] : -1;
        const bool f16p = p.yp && p.yp_f16;            // uniform over the launch
        float pm0 = 0.f, pm1 = 0.f, pm2 = 0.f;         // |value| maxima of the 64-column chunks
        if (!ok) {
            atomicExch(p.err, FMM_ETIMEOUT);
            *(volatile int *)&abort_flag = 1;
        } else {
            if (b >= 0 && g.Y) {   // FP32 rows (alone, or beside split planes for a later gather)
                float *y = (float *)g.Y + (size_t)b * g.ldy + n_lo;
#pragma unroll
                for (int n0 = 0; n0 < DC; n0 += 4) {
                    const int col = c0 + n0;
                    if (col < N) {
                        float4 o = make_float4(g.alpha * acc[n0], g.alpha * acc[n0 + 1], g.alpha * acc[n0 + 2],
                                               g.alpha * acc[n0 + 3]);
                        if (g.accumulate) {
                            const float4 old = *reinterpret_cast<const float4 *>(y + col);
                            o.x += old.x, o.y += old.y, o.z += old.z, o.w += old.w;
                        }
                        *reinterpret_cast<float4 *>(y + col) = o;
                    }
                }
            }
            if (f16p) {
#pragma unroll
                for (int n = 0; n < DC; ++n) {
                    const int col = c0 + n, ch = col >> 6;
                    const float m = col < N ? fabsf(g.alpha * acc[n]) : 0.f;
                    pm0 = ch == 0 ? fmaxf(pm0, m) : pm0;
                    pm1 = ch == 1 ? fmaxf(pm1, m) : pm1;
                    pm2 = ch == 2 ? fmaxf(pm2, m) : pm2;
                }
            }
        }
        if (PL && f16p) {
            // a chunk can straddle the two halves of a row: exchange the maxima.  Every drain warp
            // passes this barrier, also after a failed wait, so none is left waiting.
            pmax[hf][0][row] = pm0, pmax[hf][1][row] = pm1, pmax[hf][2][row] = pm2;
            asm volatile("bar.sync 2, 256;" ::: "memory");
            pm0 = fmaxf(pmax[0][0][row], pmax[1][0][row]);
            pm1 = fmaxf(pmax[0][1][row], pmax[1][1][row]);
            pm2 = fmaxf(pmax[0][2][row], pmax[1][2][row]);
        }
        if (f16p && p.yp_row_scale) {   // one scale for the whole row (the launch covers every column)
            const float m = fmaxf(pm0, fmaxf(pm1, pm2));
            pm0 = pm1 = pm2 = m;
        }
        if (ok && b >= 0 && f16p) {
            // FP16 hi/lo planes of the row scaled by a power of two per 64-column chunk, so that
            // its largest entry is below 2^14 (no overflow, full FP16 precision)
            float sc[3];
            const float mxs[3] = {pm0, pm1, pm2};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int ex = 0;
                frexpf(mxs[c], &ex);                       // mx < 2^ex
                const int e = min(max(14 - ex, -126), 126);
                sc[c] = mxs[c] > 0.f ? ldexpf(1.f, e) : 1.f;
                // the scale entry is written by the thread holding the chunk's first column
                if (c * 64 < N && c * 64 >= c0 && c * 64 < c0 + DC)
                    p.yp_scale[(size_t)b * p.yp_scale_ld + n_lo / 64 + c] = mxs[c] > 0.f ? ldexpf(1.f, -e) : 0.f;
            }
#pragma unroll
            for (int n0 = 0; n0 < DC; n0 += 8) {
                const int col = c0 + n0;   // 8 columns never straddle a 64-column chunk
                if (col < N) {
                    const int ch = col >> 6;
                    const float s8 = ch == 0 ? sc[0] : ch == 1 ? sc[1] : sc[2];
                    const size_t e = (size_t)b * p.yp_ld + n_lo + col;
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        uint32_t h[2], l[2];
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const float x = g.alpha * acc[n0 + i + j] * s8;
                            const __half hh = __float2half_rn(x);
                            h[j] = __half_as_ushort(hh);
                            l[j] = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
                        }
                        hw[i / 2] = h[0] | (h[1] << 16);
                        lw[i / 2] = l[0] | (l[1] << 16);
                    }
                    *reinterpret_cast<uint4 *>(p.yp + e * 2) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(p.yp + p.yp_plane + e * 2) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
        } else if (ok && b >= 0 && p.yp) {
            // split planes for a later tensor-core gather (BF16 hi/lo[/third] or TF32 big/small)
#pragma unroll
            for (int n0 = 0; n0 < DC; n0 += 8) {
                const int col = c0 + n0;
                if (col < N) {
                    const size_t e = (size_t)b * p.yp_ld + n_lo + col;
                    if (!TF32) {
                        uint32_t w[3][4];
#pragma unroll
                        for (int i = 0; i < 8; i += 2) {
                            uint32_t h[2], l[2], m[2];
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                const float x = g.alpha * acc[n0 + i + j];
                                h[j] = bf16_bits(x);
                                const float r1 = x - bf16_val(h[j]);
                                l[j] = bf16_bits(r1);
                                m[j] = bf16_bits(r1 - bf16_val(l[j]));
                            }
                            w[0][i / 2] = h[0] | (h[1] << 16);
                            w[1][i / 2] = l[0] | (l[1] << 16);
                            w[2][i / 2] = m[0] | (m[1] << 16);
                        }
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl)
                            if (pl < p.nplanes)
                                *reinterpret_cast<uint4 *>(p.yp + pl * p.yp_plane + e * 2) =
                                    make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
                    } else {
                        uint32_t bb[8], ss[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float x = g.alpha * acc[n0 + i];
                            bb[i] = tf32_round(x);
                            ss[i] = tf32_round(x - __uint_as_float(bb[i]));
                        }
                        uint4 *d0 = reinterpret_cast<uint4 *>(p.yp + e * 4);
                        uint4 *d1 = reinterpret_cast<uint4 *>(p.yp + p.yp_plane + e * 4);
                        d0[0] = make_uint4(bb[0], bb[1], bb[2], bb[3]);
                        d0[1] = make_uint4(bb[4], bb[5], bb[6], bb[7]);
                        d1[0] = make_uint4(ss[0], ss[1], ss[2], ss[3]);
                        d1[1] = make_uint4(ss[4], ss[5], ss[6], ss[7]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
}

template <bool TF32>
__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc_kernel(const __grid_constant__ TcDev p) {
    tc_body<TF32, false>(p);
}

// Plane layout: capped at 120 registers a thread (46K for the CTA), so that near-field CTAs fit
// beside it on an SM.
template <bool TF32>
__global__ void __maxnreg__(120) gemm_tc_plane_kernel(const __grid_constant__ TcDev p) {
    tc_body<TF32, true>(p);
}

// ---------------------------------------------------------------------------------------
// FP32 rows -> FP16 hi/lo planes, each row scaled by a power of two per 64-column chunk (its
// largest entry below 2^14), 1 / scale per (row, chunk): the form the FP16X3 contractions read.
// One warp per row.
// ---------------------------------------------------------------------------------------
namespace {
__global__ void rows_to_planes_kernel(const float *__restrict__ x, int ldx, int nrows, int ncols,
                                      unsigned char *__restrict__ planes, long long plane_bytes, int ldp,
                                      float *__restrict__ scales, int lds) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= nrows) return;
    const float *xr = x + (size_t)row * ldx;
    uint16_t *hi = reinterpret_cast<uint16_t *>(planes) + (size_t)row * ldp;
    uint16_t *lo = reinterpret_cast<uint16_t *>(planes + plane_bytes) + (size_t)row * ldp;
    for (int c0 = 0; c0 < ncols; c0 += 64) {
        const int i0 = c0 + lane, i1 = c0 + 32 + lane;
        const float v0 = i0 < ncols ? xr[i0] : 0.f, v1 = i1 < ncols ? xr[i1] : 0.f;
        float m = fmaxf(fabsf(v0), fabsf(v1));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        int ex = 0;
        frexpf(m, &ex);
        const int e = min(max(14 - ex, -126), 126);
        const float sc = m > 0.f ? ldexpf(1.f, e) : 1.f;
        if (lane == 0) scales[(size_t)row * lds + c0 / 64] = m > 0.f ? ldexpf(1.f, -e) : 0.f;
        for (int k = 0; k < 2; ++k) {
            const int i = k ? i1 : i0;
            if (i >= ncols) continue;
            const float v = (k ? v1 : v0) * sc;
            const __half h = __float2half_rn(v);
            hi[i] = __half_as_ushort(h);
            lo[i] = __half_as_ushort(__float2half_rn(v - __half2float(h)));
        }
    }
}
}  // namespace

cudaError_t launch_rows_to_planes(const float *x, int ldx, int64_t nrows, int ncols, void *planes,
                                  long long plane_bytes, int ldp, float *scales, int lds, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    rows_to_planes_kernel<<<(unsigned)((nrows + 7) / 8), 256, 0, s>>>(x, ldx, (int)nrows, ncols,
                                                                      (unsigned char *)planes, plane_bytes, ldp,
                                                                      scales, lds);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// host side: operand planes and launch
// ---------------------------------------------------------------------------------------
namespace {

// planes of the operands in a precision mode (FMM_FP16X3: of every GEMM but the stencil's)
int planes_of(int prec) { return (prec == FMM_BF16X6 || prec == FMM_FP16X3) ? 3 : 2; }

uint16_t host_bf16(float x) {   // round to nearest even
    uint32_t u;
    std::memcpy(&u, &x, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}
float host_bf16_val(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
uint32_t host_tf32(float x) {   // round to nearest (ties away), 10 explicit mantissa bits
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x1000u;
    return u & 0xffffe000u;
}
float host_f(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
uint16_t host_f16(float x) {   // IEEE binary16, round to nearest even (|x| < 65520 here)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
    const uint32_t a = u & 0x7fffffffu;
    if (a >= 0x477ff000u) return sign | 0x7c00u;                 // rounds beyond the largest finite
    if (a < 0x38800000u) {                                       // below 2^-14: subnormal steps of 2^-24
        float f;
        std::memcpy(&f, &a, 4);
        return sign | (uint16_t)std::nearbyint((double)f * 16777216.0);
    }
    uint32_t h = ((((a >> 23) - 112u) << 10) | ((a & 0x7fffffu) >> 13));
    const uint32_t rem = a & 0x1fffu;
    if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;     // a carry moves into the exponent
    return sign | (uint16_t)h;
}
double host_f16_val(uint16_t h) {
    const int e = (h >> 10) & 0x1f, m = h & 0x3ff;
    const double v = e == 0 ? std::ldexp((double)m, -24) : std::ldexp(1.0 + m / 1024.0, e - 15);
    return (h & 0x8000u) ? -v : v;
}

}  // namespace

// rows x cols FP64 (row-major) -> the split planes of the padded rows_p x cols_p operand, in
// the stage layout [chunk][plane][rows_p x 128 B, SWIZZLE_128B], appended to `out`.  With
// `f16` the planes are FP16 hi/lo of the operand scaled per chunk by a power of two (largest
// entry below 2^14); 1 / scale of every chunk is appended to `scales`.  With `uniform` every
// chunk gets the scale of the whole operand, so that the chunks of one operator can accumulate
// in one tensor-memory accumulator.
static void tc_pack(int prec, bool f16, const double *w, int rows, int cols, int rows_p, int cols_p,
                    std::vector<unsigned char> &out, std::vector<float> &scales, bool uniform = false) {
    const bool tf32 = prec == FMM_TF32X3;
    const int np = f16 ? 2 : planes_of(prec);
    const int esz = tf32 ? 4 : 2;
    const int ce = kAtomBytes / esz;
    const int nchunks = (cols_p + ce - 1) / ce;
    const size_t plane_bytes = (size_t)rows_p * kAtomBytes;
    const size_t base = out.size();
    out.resize(base + (size_t)nchunks * np * plane_bytes, 0);
    unsigned char *h = out.data() + base;
    std::vector<double> sc(nchunks, 1.0);
    if (f16)
        for (int k = 0; k < nchunks; ++k) {
            double mx = 0;
            const int c_lo = uniform ? 0 : k * ce, c_hi = uniform ? cols : std::min(cols, (k + 1) * ce);
            for (int r = 0; r < rows; ++r)
                for (int c = c_lo; c < c_hi; ++c) mx = std::max(mx, std::fabs(w[(size_t)r * cols + c]));
            int ex = 0;
            std::frexp(mx, &ex);
            sc[k] = mx > 0 ? std::ldexp(1.0, 14 - ex) : 1.0;
            scales.push_back(mx > 0 ? (float)std::ldexp(1.0, ex - 14) : 0.f);
        }
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) {
            const double x = w[(size_t)r * cols + c] * sc[c / ce];
            const int chunk = c / ce, kin = c % ce;
            const int unit = (kin * esz) >> 4, within = (kin * esz) & 15;
            const size_t off = (size_t)(r >> 3) * 1024 + (r & 7) * 128 + ((unit ^ (r & 7)) << 4) + within;
            unsigned char *dst = h + (size_t)chunk * np * plane_bytes + off;
            if (f16) {
                const uint16_t hi = host_f16((float)x);
                const uint16_t lo = host_f16((float)(x - host_f16_val(hi)));
                std::memcpy(dst, &hi, 2);
                std::memcpy(dst + plane_bytes, &lo, 2);
            } else if (tf32) {
                const uint32_t b = host_tf32((float)x);
                const uint32_t sm = host_tf32((float)(x - (double)host_f(b)));
                std::memcpy(dst, &b, 4);
                std::memcpy(dst + plane_bytes, &sm, 4);
            } else {
                const uint16_t b0 = host_bf16((float)x);
                const double r1 = x - (double)host_bf16_val(b0);
                const uint16_t b1 = host_bf16((float)r1);
                const double r2 = r1 - (double)host_bf16_val(b1);
                const uint16_t b2 = host_bf16((float)r2);
                const uint16_t v[3] = {b0, b1, b2};
                for (int pl = 0; pl < np; ++pl) std::memcpy(dst + pl * plane_bytes, &v[pl], 2);
            }
        }
}

// `count` operators of rows x cols (consecutive in w) packed into one allocation
static cudaError_t tc_upload_many(fmm_ctx *ctx, const double *w, int count, int rows, int cols,
                                  int rows_p, int cols_p, TcMat *out, bool f16 = false, bool uniform = false) {
    std::vector<unsigned char> h;
    std::vector<float> scales;
    for (int k = 0; k < count; ++k)
        tc_pack(ctx->opt.precision, f16, w + (size_t)k * rows * cols, rows, cols, rows_p, cols_p, h, scales, uniform);
    void *d = nullptr;
    FMM_CUDA_TRY(dev_malloc(&d, h.size()));
    ctx->op_allocs.push_back(d);
    FMM_CUDA_TRY(cudaMemcpy(d, h.data(), h.size(), cudaMemcpyHostToDevice));
    out->planes[0] = d;
    out->rows = rows_p;
    out->cols = cols_p;
    out->nplanes = f16 ? 2 : planes_of(ctx->opt.precision);
    out->bytes = h.size() / count;   // bytes of one operator (the stride)
    if (f16) {
        void *ds = nullptr;
        FMM_CUDA_TRY(dev_malloc(&ds, scales.size() * sizeof(float)));
        ctx->op_allocs.push_back(ds);
        FMM_CUDA_TRY(cudaMemcpy(ds, scales.data(), scales.size() * sizeof(float), cudaMemcpyHostToDevice));
        out->scale = (float *)ds;
        out->scale_ld = (int)(scales.size() / count);
    }
    return cudaSuccess;
}

// FMM_FP16X3 M2L stencil with segment accumulation: every K chunk of one transfer vector's
// product goes into one tensor-memory accumulator, drained once per segment.  That needs one
// scale per source row (written by the compress epilogue, so its output must fit one CTA) and
// one per operator, in both directions.
static bool stencil_segment_acc(const fmm_ctx *ctx) {
    if (ctx->opt.precision != FMM_FP16X3) return false;
    for (int l = 0; l <= kMaxDepth; ++l) {
        const OpSet &o = ctx->fwd[l];
        if (o.ns && std::max(o.kinp, o.koutp) > kTcMaxN) return false;
    }
    return true;
}

static cudaError_t tc_upload_set(fmm_ctx *ctx, const HostOps &h, bool adjoint, const OpSet &o, TcOpSet &t) {
    const int ns = h.ns, nsp = o.nsp;
    const auto &U = adjoint ? h.a_up : h.up;
    const auto &D = adjoint ? h.a_down : h.down;
    std::vector<double> ups;
    for (int c = 0; c < 8; ++c) ups.insert(ups.end(), U[c].begin(), U[c].end());
    const bool f16ops = ctx->opt.precision == FMM_FP16X3;   // FP16 planes for every contraction
    FMM_CUDA_TRY(tc_upload_many(ctx, ups.data(), 8, ns, ns, nsp, nsp, &t.up, f16ops));
    // the 8 D2D operators in one allocation (contiguous operators and scales), one view each
    {
        const bool f16 = ctx->opt.precision == FMM_FP16X3;
        std::vector<double> downs;
        for (int c = 0; c < 8; ++c) downs.insert(downs.end(), D[c].begin(), D[c].end());
        TcMat all;
        FMM_CUDA_TRY(tc_upload_many(ctx, downs.data(), 8, ns, ns, nsp, nsp, &all, f16));
        for (int c = 0; c < 8; ++c) {
            t.down[c] = all;
            t.down[c].planes[0] = (unsigned char *)all.planes[0] + (size_t)c * all.bytes;
            if (all.scale) t.down[c].scale = all.scale + (size_t)c * all.scale_ld;
        }
    }
    FMM_CUDA_TRY(tc_upload_many(ctx, (adjoint ? h.a_compress : h.compress).data(), 1, o.kin, ns, o.kinp, nsp,
                                &t.compress, f16ops));
    FMM_CUDA_TRY(tc_upload_many(ctx, (adjoint ? h.a_decompress : h.decompress).data(), 1, ns, o.kout, nsp,
                                o.koutp, &t.decompress, f16ops));
    // the stencil operators scaled as a whole (see segment accumulation in tc_body)
    FMM_CUDA_TRY(tc_upload_many(ctx, (adjoint ? h.a_stencil : h.stencil).data(), kNumTransfer, o.kout, o.kin,
                                o.koutp, o.kinp, &t.stencil, ctx->opt.precision == FMM_FP16X3,
                                stencil_segment_acc(ctx)));
    return cudaSuccess;
}

cudaError_t tc_upload_operators(fmm_ctx *ctx) {
    for (int l = 0; l <= kMaxDepth; ++l) {   // each distinct host set once, as the SIMT copies
        int first = -1;
        for (int k = 0; k < l && first < 0; ++k)
            if (ctx->host_ops[k] == ctx->host_ops[l]) first = k;
        if (first >= 0) {
            ctx->tc_fwd[l] = ctx->tc_fwd[first];
            ctx->tc_adj[l] = ctx->tc_adj[first];
            continue;
        }
        ctx->tc_owned.push_back(ctx->tc_fwd[l] = new TcOpSet());
        ctx->tc_owned.push_back(ctx->tc_adj[l] = new TcOpSet());
        FMM_CUDA_TRY(tc_upload_set(ctx, *ctx->host_ops[l], false, ctx->fwd[l], *ctx->tc_fwd[l]));
        FMM_CUDA_TRY(tc_upload_set(ctx, *ctx->host_ops[l], true, ctx->adj[l], *ctx->tc_adj[l]));
    }
    return cudaSuccess;
}

void tc_free(fmm_ctx *ctx) {
    for (TcOpSet *t : ctx->tc_owned) delete t;
    ctx->tc_owned.clear();
    for (int l = 0; l <= kMaxDepth; ++l) ctx->tc_fwd[l] = ctx->tc_adj[l] = nullptr;
}

GemmDev make_gemm_dev(const fmm_ctx *ctx, const GemmCall &c);

cudaError_t gemm_tc(const fmm_ctx *ctx, const GemmCall &c, int op_id, cudaStream_t s) {
    if (c.tiles || c.rows) return cudaErrorNotSupported;   // box subsets: SIMT form only
    const bool adj = op_id >= OP_COUNT;
    const int op = op_id % OP_COUNT;
    // the output level's operators; PARENT2's D2D segment those of the parent level
    const TcOpSet &T = adj ? *ctx->tc_adj[c.level] : *ctx->tc_fwd[c.level];
    const int lp = c.level > 0 ? c.level - 1 : 0;
    const TcOpSet &T1 = adj ? *ctx->tc_adj[lp] : *ctx->tc_fwd[lp];
    TcDev p{};
    p.g = make_gemm_dev(ctx, c);
    const TileSet &ts = (c.mode == GM_STENCIL || c.mode == GM_PARENT2) ? ctx->tiles_cls[c.level]
                                                                       : ctx->tiles_plain[c.level];
    if (ts.ntiles == 0) return cudaSuccess;
    p.g.tiles = ts.tiles;
    p.g.masks = ts.masks;
    if (c.mode == GM_STENCIL && ctx->masks_ev) FMM_CUDA_TRY(cudaStreamWaitEvent(s, ctx->masks_ev, 0));
    switch (op) {
        case OP_UP: p.Wt0 = (const unsigned char *)T.up.planes[0]; p.wt_stride = (long long)T.up.bytes; break;
        case OP_COMPRESS: p.Wt0 = (const unsigned char *)T.compress.planes[0]; break;
        case OP_STENCIL: p.Wt0 = (const unsigned char *)T.stencil.planes[0]; p.wt_stride = (long long)T.stencil.bytes; break;
        case OP_DECOMPRESS:
            p.Wt0 = (const unsigned char *)T.decompress.planes[0];
            for (int k = 0; k < 8; ++k) p.Wt1[k] = (const unsigned char *)T1.down[k].planes[0];
            break;
        default: return cudaErrorInvalidValue;
    }
    const int prec = ctx->opt.precision;
    p.tf32 = prec == FMM_TF32X3;
    p.f16 = prec == FMM_FP16X3;   // FP16 split planes with scales for every contraction
    p.nplanes = p.f16 ? 2 : planes_of(prec);
    if (p.nplanes == 3) {
        const int a[6] = {2, 1, 0, 1, 0, 0}, b[6] = {0, 1, 2, 0, 1, 0};
        p.nprod = 6;
        for (int i = 0; i < 6; ++i) p.prod_a[i] = a[i], p.prod_b[i] = b[i];
    } else {
        const int a[3] = {1, 0, 0}, b[3] = {0, 1, 0};
        p.nprod = 3;
        for (int i = 0; i < 3; ++i) p.prod_a[i] = a[i], p.prod_b[i] = b[i];
    }
    if (p.f16) {
        const TcMat &W = op == OP_UP ? T.up : op == OP_COMPRESS ? T.compress : op == OP_STENCIL ? T.stencil : T.decompress;
        if (!c.Xp || !c.xp_scale || !W.scale) return cudaErrorInvalidValue;
        p.a_scale = c.xp_scale;
        p.a_scale_ld = c.xp_scale_ld;
        p.b_scale = W.scale;
        p.b_scale_ld = W.scale_ld;
        if (c.mode == GM_PARENT2 && c.X1) {
            if (!c.Xp1 || !c.xp1_scale || !T1.down[0].scale || ((uintptr_t)c.Xp1 & 15) || ((c.xp1_ld * 2) & 15) ||
                (c.xp1_plane & 15))
                return cudaErrorInvalidValue;
            p.xp1 = (const unsigned char *)c.Xp1;
            p.xp1_plane = c.xp1_plane;
            p.xp1_ld = c.xp1_ld;
            p.a_scale1 = c.xp1_scale;
            p.a_scale1_ld = c.xp1_scale_ld;
            p.b_scale1 = T1.down[0].scale;   // the 8 class operators' scales, contiguous
            p.b_scale1_ld = T1.down[0].scale_ld;
        }
    }
    if (c.n_out % 16 != 0 || (c.k0 % 16) != 0 || (c.X1 && c.k1 % 16 != 0)) return cudaErrorInvalidValue;
    int nsplit = (c.n_out + kTcMaxN - 1) / kTcMaxN;
    p.ncta = round_up((c.n_out + nsplit - 1) / nsplit, 16);
    if (prec == FMM_FP16X3 && c.Yp && nsplit > 1) {   // FP16 output planes: 64-column aligned CTAs
        p.ncta = 128;
        nsplit = (c.n_out + 127) / 128;
    }
    const int stage_bytes = p.nplanes * (kTcRows + p.ncta) * kAtomBytes;
    // 227 KB per CTA in all: the stages, 1 KB of alignment slack and the static shared memory.
    // The plane layout keeps two stages, which leaves room on the SM for near-field CTAs.
    const bool plane = c.Xp != nullptr;
    auto kern = plane ? (p.tf32 ? gemm_tc_plane_kernel<true> : gemm_tc_plane_kernel<false>)
                      : (p.tf32 ? gemm_tc_kernel<true> : gemm_tc_kernel<false>);
    const int threads = plane ? 384 : kTcThreads;
    cudaFuncAttributes fa{};
    FMM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const int budget = 227 * 1024 - 1024 - (int)fa.sharedSizeBytes;
    p.nstages = std::min(plane ? kPlaneStages : 4, budget / stage_bytes);
    if (p.nstages < 2) return cudaErrorInvalidValue;
    // two accumulators of ncta columns; the drain reads 32 columns at a time, so the last read
    // of the second accumulator may extend 16 columns past it: keep that inside the allocation
    p.seg_acc = c.mode == GM_STENCIL && plane && stencil_segment_acc(ctx);
    p.yp_row_scale = op == OP_COMPRESS && c.Yp && stencil_segment_acc(ctx) && nsplit == 1;
    if (op == OP_COMPRESS && stencil_segment_acc(ctx) && !p.yp_row_scale) return cudaErrorInvalidValue;
    int cols = 32;
    while (cols < (p.seg_acc ? 3 : 2) * p.ncta + 16) cols <<= 1;
    if (cols > 512) return cudaErrorInvalidValue;
    p.tmem_cols = cols;
    p.err = ctx->dev_flag;
    p.wait_ns = ctx->tc_wait_ns;
    if (c.Xp) {
        // A rows from split planes: K of the segment must be the planes' width
        if (c.mode == GM_PARENT2 && c.X1 && !c.Xp1) return cudaErrorInvalidValue;
        if (((uintptr_t)c.Xp & 15) || ((c.xp_ld * (p.tf32 ? 4 : 2)) & 15) || (c.xp_plane & 15))
            return cudaErrorInvalidValue;
        p.a_planes = 1;
        p.xp = (const unsigned char *)c.Xp;
        p.xp_plane = c.xp_plane;
        p.xp_ld = c.xp_ld;
    }
    if (c.Yp) {
        p.yp = (unsigned char *)c.Yp;
        p.yp_plane = c.yp_plane;
        p.yp_ld = c.yp_ld;
        if (prec == FMM_FP16X3) {
            // per-chunk scales need every CTA's columns to start on a 64-column chunk
            if (!c.yp_scale || (nsplit > 1 && p.ncta % 64 != 0)) return cudaErrorInvalidValue;
            p.yp_f16 = 1;
            p.yp_scale = c.yp_scale;
            p.yp_scale_ld = c.yp_scale_ld;
        }
    }
    const size_t smem = (size_t)p.nstages * stage_bytes + 1024;
    FMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3(ts.ntiles, (c.n_out + p.ncta - 1) / p.ncta), threads, smem, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace fmm
