// k_vote_tc.cu -- the vote on the tcgen05 tensor cores (sm_103a).
//
// D[c][i] = sum_k A[c][k] B[i][k] with
//   A row (cell c):  K = 16: [m(q_c) (10), -tau_hi, -tau_lo, m_0..m_3]
//                    K = 32: [m_hi (10), m_hi (10), m_lo (10), -tau_hi, -tau_lo]
//   B row (pair i):  K = 16: [s_i (10), 1, 1, lo(s_0)..lo(s_3)]
//                    K = 32: [s_hi (10), s_lo (10), s_hi (10), 1, 1]
// so D = m.s - tau ~ q_c^T S_i q_c - tau_c, in FP32 in tensor memory.  The
// cell votes for the pair iff D <= 0; the epilogue counts D < 0 and flags
// |D| <= band_c, a rigorous per-cell bound on |D - (v - tau)_exact| (operand
// rounding to 16 bits, the FP32 pair step, FP32 accumulation).  Flagged tests
// are re-evaluated with the FP32 re-check |b - R_c a|^2/4 - c_i, whose error
// is below 7e-7; those within kBand64 = 2e-6 of the threshold go to the FP64
// resolution pass (k_resolve64.cu), so every decision is the FP64 one.
//
// One persistent CTA per SM.  The MMA unit is U = 256 or 128 pairs (N of one
// tcgen05.mma) and TMEM holds 512 / U accumulator stages of U columns:
//   warp 0      lane 0 streams 256-pair B tiles global -> shared with the bulk
//               copy engine (cp.async.bulk + mbarrier complete_tx), kNB stages
//   warp 1      allocates 512 TMEM columns; lane 0 issues tcgen05.mma
//               (M = 128 cells, N = U pairs, K = 16 per instruction), each
//               U-pair unit of a B tile into the next accumulator stage, and
//               commits to mbarriers
//   warps 2-3   build the 128-row A tile of each work item in shared memory
//               (double buffered)
//   warps 4..   G epilogue warpgroups; warpgroup g drains columns
//               [g U/G, (g+1) U/G) of every unit in turn, so each has all
//               stages in flight; each thread owns one TMEM lane = one cell and
//               reads 16 or 32 columns per tcgen05.ld, double-buffered so the
//               next load is in flight while it counts the current one (and
//               releases the stage as soon as its last load has completed): the
//               signs two per packed fma rounding toward -inf on the FMA pipe
//               (sign_fma2) and the minimum of |D| two values per three-input
//               minimum on the ALU pipe.  One warp vote per chunk: when a lane's
//               chunk holds a value within the band (rare), the warp queues
//               those tests from the registers it still holds into a per-warp
//               shared-memory queue that is drained 32 at a time (one lane per
//               test), so no warp waits on one global load per flagged test.
// The autotuner picks U, G and the chunk width per workload.
// Every mbarrier wait is bounded (2 s or 2^24 polls): on expiry the CTA sets
// *err_flag, stops all roles, waits (bounded) for its own copies and MMAs,
// frees its TMEM and returns.
//
// Operand tiles use the canonical no-swizzle K-major layout: 8 rows x 16 B
// core matrices stored contiguously (128 B); SBO = 128 B between 8-row
// groups; LBO = rows x 16 B between the 8-column halves of a K = 16 slice
// (2048 B for the 128-row A tile, 4096 B for the 256-row B tile).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

constexpr int kNB = 5;                         // B stages
constexpr int kMaxAcc = 4;                     // accumulator stages (512 TMEM columns / unit width)
constexpr int kATileBytesMax = 128 * 32 * 2;   // 128 rows x K = 32 x 2 B
constexpr int kBTileBytesMax = kPairTile * 32 * 2; // 256 rows x K = 32 x 2 B
constexpr int kALbo = 128 * 16, kBLbo = kPairTile * 16;
// Deferred re-check state, per epilogue warp / warpgroup (after the barriers):
//   queue   kQCap entries {pair offset in the item, lane | (D < 0) << 5} per warp
//   defer   kDCap entries {pair offset in the item, cell row} per warp: tests
//           whose re-check lies within kBand64 of tau, staged for the FP64 pass
//   rows    R (9), tau, table position, pad per cell row, per warpgroup
//   corr    count correction per cell row, per warpgroup
constexpr int kQCap = 64;
constexpr int kMaxG = 4;
constexpr size_t kQueueBytes = (size_t)4 * kMaxG * kQCap * 8;
constexpr size_t kRowBytes = (size_t)kMaxG * 128 * 12 * 4;
constexpr size_t kCorrBytes = (size_t)kMaxG * 128 * 4;
constexpr int kDCap = 64;
constexpr size_t kDeferBytes = (size_t)4 * kMaxG * (kDCap * 8 + 16);  // entries + count + queue-full flag
constexpr size_t kBarBytes = 1024;
// 1024 B alignment slack + A (2 stages) + B (kNB stages) + barriers/flags + re-check state.
// Over 116 KB, so one CTA per SM (each holds all 512 TMEM columns).
constexpr size_t kSmemBytes =
    1024 + 2 * kATileBytesMax + kNB * kBTileBytesMax + kBarBytes + kQueueBytes + kRowBytes + kCorrBytes +
    kDeferBytes;
static_assert(kSmemBytes > 116 * 1024 && kSmemBytes <= 227 * 1024, "shared memory budget");
static_assert((2 * kNB + 2 * kMaxAcc + 5) * 8 + 8 + 16 <= (int)kBarBytes, "barrier area");
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kWaitPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// One poll of a phase.  The thread may stay suspended in it for up to 1 us (the
// suspend-time hint) while the phase is pending; with the hint the coarse vote
// ran 1.5% faster than with the default limit.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Control block of the bounded waits: `abort` is set by any role that gives up;
// `limit_ns` bounds one wait (kWaitNs, or 1 ms in the wait-expiry test mode).
struct WaitCtl {
    volatile int abort;
    int pad;
    uint64_t limit_ns;
};

// Bounded wait for the phase of parity `parity` to complete.  Returns false
// when the CTA was aborted or the wait expired.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity, WaitCtl *w) {
    const uint64_t t0 = gtimer(), lim = w->limit_ns;
    for (uint32_t it = 1; it < kWaitPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 0) {
            if (w->abort) return false;
            if (gtimer() - t0 > lim) return false;
        }
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, WaitCtl *w) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity, w);
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc512(uint32_t *slot) {  // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc512(uint32_t taddr) {  // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(taddr) : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// N (16 or 32) consecutive 32-bit TMEM columns of this thread's lane; the
// wait (for all of the thread's outstanding loads) binds the registers, so no
// use is scheduled before the data has arrived.
#define RV_R4(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3])
#define RV_W4(b) "+r"(r[b]), "+r"(r[b + 1]), "+r"(r[b + 2]), "+r"(r[b + 3])
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];\n"
                 : RV_R4(0), RV_R4(4), RV_R4(8), RV_R4(12)
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : RV_R4(0), RV_R4(4), RV_R4(8), RV_R4(12), RV_R4(16), RV_R4(20), RV_R4(24), RV_R4(28)
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" : RV_W4(0), RV_W4(4), RV_W4(8), RV_W4(12) : : "memory");
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : RV_W4(0), RV_W4(4), RV_W4(8), RV_W4(12), RV_W4(16), RV_W4(20), RV_W4(24), RV_W4(28)
                 :
                 : "memory");
}
#undef RV_R4
#undef RV_W4

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO = 128 B >> 4 (32-45), version 1 (46).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(128u >> 4) << 32) |
           (1ull << 46);
}
// Instruction descriptor of kind::f16: D = F32 (bit 4), A = B = F16 (0) or
// BF16 (1) at bits 7 and 10, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <bool BF16, int N>
__host__ __device__ constexpr uint32_t idesc_f16() {
    return (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((128u >> 4) << 24);
}

__device__ __forceinline__ int a_off(int r, int k) { return (k >> 3) * kALbo + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

template <bool BF16>
__device__ __forceinline__ uint16_t h16(float x) {
    if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}
template <bool BF16>
__device__ __forceinline__ float f16(uint16_t x) {
    if (BF16) return __bfloat162float(__ushort_as_bfloat16(x));
    return __half2float(__ushort_as_half(x));
}

// Sign counting on the FMA pipe.  A counter starts at 1.5; fma rounding toward
// -inf of counter + d 2^-30 returns the counter lowered by exactly one ulp
// (2^-23) when d < 0 (|d 2^-30| < 2^-23 for |d| < 2^7) and the counter itself
// when d >= 0, -0 included.  Two counters per 64-bit register, two tests per
// packed fma; while a counter stays in [1, 2) its decrement count is
// bits(1.5f) - bits(counter).
constexpr uint64_t kCnt0 = 0x3FC000003FC00000ull;  // (1.5f, 1.5f)
constexpr uint64_t kTiny2 = 0x3080000030800000ull; // (2^-30, 2^-30)
__device__ __forceinline__ uint64_t sign_fma2(uint32_t a, uint32_t b, uint64_t acc) {
    uint64_t d;
    asm("{\n .reg .b64 t;\n mov.b64 t, {%1, %2};\n fma.rm.f32x2 %0, t, %3, %4;\n}\n"
        : "=l"(d)
        : "r"(a), "r"(b), "l"(kTiny2), "l"(acc));
    return d;
}
__device__ __forceinline__ int sign_fma2_count(uint64_t acc) {
    return (int)(2u * 0x3FC00000u - (uint32_t)acc - (uint32_t)(acc >> 32));
}
// min(m, |x|, |y|) (three-input minimum).
__device__ __forceinline__ float min3_abs(float m, float x, float y) {
    float r;
    asm("min.abs.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(x), "f"(y));
    return r;
}

// Rigorous per-cell bound on |D - (v - tau)| (see the file comment).  smax_k
// bounds |s_k| for unit a, b: 1 for the diagonal entries S00..S33, 1/2 for the
// six others (each is half a cross-product component, or half of a0 b1 + a1 b0
// and the like, and |a0 b1 + a1 b0| <= |a| |b| by Cauchy-Schwarz); the final
// factor 1.25 covers inputs whose squared norms are within 1e-5 of 1.
template <int KSTEPS, bool BF16>
__device__ __forceinline__ float cell_band(const float m[10]) {
    const float u32 = 5.9604645e-8f;
    const float u16 = BF16 ? 3.90625e-3f : 4.8828125e-4f;
    const float sub = BF16 ? 0.f : 2.9802322e-8f;  // half the FP16 subnormal spacing
    const float smax[10] = {1.f, 1.f, 1.f, 1.f, 0.5f, 0.5f, 0.5f, 0.5f, 0.5f, 0.5f};
    const int K = 16 * KSTEPS;
    const float accum = (14.f + 12.f * K) * u32 + 1e-6f;
    float msum = 0.f, mabs = 0.f;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        msum = fmaf(fabsf(m[k]), smax[k], msum);
        mabs += fabsf(m[k]);
    }
    float b;
    if (KSTEPS == 1) {
        // A holds m~ = m rounded to 16 bits, whose error is known exactly; B holds s
        // rounded to 16 bits plus, in the padding columns, the low halves of the four
        // diagonal entries.  D - (v - tau) = sum (m - m~) s + sum m~ (s - s_B) + ...:
        // dm below, u16 |m~| smax for the six off-diagonal entries, u16^2 for the
        // diagonal ones and for tau's hi/lo split; 2 u32 for the FP32 m, s and tau.
        float dm = 0.f, mt_off = 0.f, mt_diag = 0.f;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const float mt = f16<BF16>(h16<BF16>(m[k]));
            dm = fmaf(fabsf(m[k] - mt), smax[k], dm);
            if (k < 4)
                mt_diag += fabsf(mt);
            else
                mt_off = fmaf(fabsf(mt), smax[k], mt_off);
        }
        b = dm + u16 * mt_off + u16 * u16 * (mt_diag + 1.f) + 2.f * u32 * (msum + 1.f) +
            2.f * sub * (mabs + 1.f) + accum;
    } else {
        b = (3.f * u16 * u16 + u16 * u16 * u16 + 2.f * u32) * msum + 2.f * sub * (mabs + 7.f) + accum;
    }
    return b * 1.25f;
}

struct ItemView {
    VoteItem W;
    ProbRef P;
    LevelRef L;
    int ncell;
    int ntiles;
};

__device__ __forceinline__ bool load_item(const VoteItem *items, int it, const ProbRef *probs, const LevelRef *lref,
                                          int level_stride, int level, ItemView &v) {
    v.W = items[it];
    v.P = probs[v.W.prob];
    if (level > v.P.levels) return false;
    v.L = lref[v.W.prob * level_stride + level];
    v.ncell = *v.L.ncells;
    if (v.W.cell_begin >= v.ncell) return false;
    v.ntiles = (v.W.pair_end - v.W.pair_begin) / kPairTile;
    return v.ntiles > 0;
}

// Warps 2-3: the A tile (128 cells x K, 16-bit) of every work item, double
// buffered; a cold role kept out of line so the epilogue keeps its registers.
template <int KSTEPS, bool BF16>
__device__ __noinline__ void build_a_tiles(const VoteItem *__restrict__ items, int n_items,
                                           const ProbRef *__restrict__ probs, const LevelRef *__restrict__ lref,
                                           int level_stride, int level, uint8_t *sA, uint64_t *a_full,
                                           uint64_t *a_empty, WaitCtl *wctl, int *err_flag, int warp,
                                           int lane) {
    constexpr int K = 16 * KSTEPS;
    const int r0 = (warp - 2) * 64 + lane;
    int i = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        ItemView v;
        if (!load_item(items, it, probs, lref, level_stride, level, v)) continue;
        const int ab = i & 1;
        const uint32_t ua = (uint32_t)(i >> 1);
        // warp-uniform outcome of the bounded wait
        if (!__all_sync(0xffffffffu, mbar_wait(&a_empty[ab], (ua & 1u) ^ 1u, wctl))) {
            wctl->abort = 1;
            atomicExch(err_flag, 1);
            break;
        }
        uint8_t *tile = sA + ab * kATileBytesMax;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + 32 * h;
            const int pos = v.W.cell_begin + r;
            uint16_t row[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) row[k] = 0;
            if (pos < v.ncell) {
                const float4 m0 = v.L.cells.m32[3 * pos], m1 = v.L.cells.m32[3 * pos + 1],
                             m2 = v.L.cells.m32[3 * pos + 2];
                const float m[10] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y};
                const float tau = (float)tau_cs(v.P.sin_d, v.P.cos_d, v.L.cells.trig[pos]);
                const uint16_t th = h16<BF16>(tau);
                const uint16_t tl = h16<BF16>(tau - f16<BF16>(th));
                if (KSTEPS == 1) {
#pragma unroll
                    for (int k = 0; k < 10; ++k) row[k] = h16<BF16>(m[k]);
                    row[10] = th ^ 0x8000u;  // -tau_hi
                    row[11] = tl ^ 0x8000u;  // -tau_lo
#pragma unroll
                    for (int k = 0; k < 4; ++k) row[12 + k] = row[k];  // times the low halves of S00..S33
                } else {
#pragma unroll
                    for (int k = 0; k < 10; ++k) {
                        const uint16_t hi = h16<BF16>(m[k]);
                        const uint16_t lo = h16<BF16>(m[k] - f16<BF16>(hi));
                        row[k] = hi;
                        row[10 + k] = hi;
                        row[20 + k] = lo;
                    }
                    row[30] = th ^ 0x8000u;
                    row[31] = tl ^ 0x8000u;
                }
            } else {  // absent cell: D = 1 for every pair
                row[KSTEPS == 1 ? 10 : 30] = h16<BF16>(1.f);
            }
#pragma unroll
            for (int c = 0; c < K / 8; ++c) {
                uint4 w;
                w.x = (uint32_t)row[8 * c + 0] | ((uint32_t)row[8 * c + 1] << 16);
                w.y = (uint32_t)row[8 * c + 2] | ((uint32_t)row[8 * c + 3] << 16);
                w.z = (uint32_t)row[8 * c + 4] | ((uint32_t)row[8 * c + 5] << 16);
                w.w = (uint32_t)row[8 * c + 6] | ((uint32_t)row[8 * c + 7] << 16);
                *reinterpret_cast<uint4 *>(tile + a_off(r, 8 * c)) = w;
            }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[ab]);
        ++i;
    }
}

template <int G, int KSTEPS, bool BF16, int CH, int U>
__global__ void __launch_bounds__(128 + 128 * G, 1)
    vote_tc_kernel(const VoteItem *__restrict__ items, int n_items, const ProbRef *__restrict__ probs,
                   const LevelRef *__restrict__ lref, int level_stride, int level, PairPool pool, ProbStats *stats,
                   float band_req, int *err_flag, uint64_t wait_ns, int test_stall, AmbQueue amb) {
    // Every warpgroup drains every stage, in unit order, so no wait ever runs
    // more than one phase ahead of its stage (an mbarrier parity wait could not
    // tell phase k+1 from a pending phase k).
    constexpr int kNAcc = 512 / U;     // accumulator stages of U columns
    constexpr int kUPT = kPairTile / U;  // units (MMAs of N = U) per B tile
    static_assert((U == 128 || U == 256) && kNAcc <= kMaxAcc, "unit width");
    static_assert(G >= 1 && G <= kMaxG && U % (32 * G) == 0, "epilogue warpgroups");
    constexpr int kCols = U / G;  // columns of each unit per warpgroup
    static_assert((CH == 16 || CH == 32) && (kCols == CH || kCols % (2 * CH) == 0), "TMEM chunks");
    constexpr int kTileBytes = kPairTile * 16 * KSTEPS * 2;  // 256 rows x K x 2 B
    constexpr uint32_t IDESC = idesc_f16<BF16, U>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                          // 2 x kATileBytesMax
    uint8_t *sB = smem + 2 * kATileBytesMax;     // kNB x kBTileBytesMax
    uint64_t *bars = (uint64_t *)(sB + kNB * kBTileBytesMax);
    uint64_t *b_full = bars, *b_empty = bars + kNB, *acc_full = bars + 2 * kNB, *acc_empty = acc_full + kNAcc;
    uint64_t *a_full = acc_empty + kNAcc, *a_empty = a_full + 2, *mma_done = a_empty + 2;
    uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
    WaitCtl *wctl = (WaitCtl *)(tmem_slot + 2);  // 8-byte aligned
    uint8_t *rq = (uint8_t *)bars + kBarBytes;  // deferred re-check state
    uint2 *q_all = (uint2 *)rq;
    float *rows_all = (float *)(rq + kQueueBytes);
    int *corr_all = (int *)(rq + kQueueBytes + kRowBytes);
    uint2 *d_all = (uint2 *)(rq + kQueueBytes + kRowBytes + kCorrBytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNB; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int s = 0; s < kNAcc; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4 * G);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_full[s], 2);
            mbar_init(&a_empty[s], 1);
        }
        mbar_init(mma_done, 1);
        wctl->abort = 0;
        wctl->limit_ns = wait_ns;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) tmem_alloc512(tmem_slot);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto fail = [&]() {
        wctl->abort = 1;
        atomicExch(err_flag, 1);
    };

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            int64_t j = 0;
            int pbs = 0;
            uint32_t pph = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                ItemView v;
                if (!load_item(items, it, probs, lref, level_stride, level, v)) continue;
                const uint8_t *src = (const uint8_t *)pool.tcb +
                                     ((v.P.pool_off + v.W.pair_begin) / kPairTile) * (int64_t)kTileBytes;
                for (int t = 0; t < v.ntiles; ++t, ++j) {
                    const int bs = pbs;  // B stage of tile j and its phase parity, carried incrementally
                    const uint32_t ph = pph;
                    if (++pbs == kNB) {
                        pbs = 0;
                        pph ^= 1u;
                    }
                    if (!mbar_wait(&b_empty[bs], ph ^ 1u, wctl)) {
                        fail();
                        ok = false;
                        break;
                    }
                    if (test_stall) continue;  // wait-expiry test: the copy never arrives
                    mbar_arrive_expect_tx(&b_full[bs], kTileBytes);
                    bulk_g2s(sB + bs * kBTileBytesMax, src + (int64_t)t * kTileBytes, kTileBytes, &b_full[bs]);
                }
            }
            // drain: the last issued copy of each stage has completed before exit
            WaitCtl drain{0, 0, kWaitNs};
            for (int64_t jj = j - 1; !test_stall && jj >= 0 && jj >= j - kNB; --jj) {
                const int bs = (int)(jj % kNB);
                const uint32_t u = (uint32_t)(jj / kNB);
                if (!mbar_wait(&b_full[bs], u & 1u, &drain)) atomicExch(err_flag, 1);
            }
        }
    } else if (warp == 1) {
        // --------------------------------- MMA --------------------------------
        if (lane == 0) {
            int64_t j = 0;
            int i = 0;
            bool ok = true;
            // B stage and accumulator stage of the next tile / unit with their phase parities,
            // and the shared-memory descriptors (start address in bits 0-13: offsets add there)
            int bs = 0, as = 0;
            uint32_t bph = 0, aph = 0;
            const uint64_t b_desc0 = sdesc(smem_u32(sB), kBLbo);
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                ItemView v;
                if (!load_item(items, it, probs, lref, level_stride, level, v)) continue;
                const int ab = i & 1;
                const uint32_t ua = (uint32_t)(i >> 1);
                if (!mbar_wait(&a_full[ab], ua & 1u, wctl)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint64_t a_desc = sdesc(smem_u32(sA + ab * kATileBytesMax), kALbo);
                for (int t = 0; t < v.ntiles && ok; ++t, ++j) {
                    if (!mbar_wait(&b_full[bs], bph, wctl)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint64_t b_desc = b_desc0 + (uint64_t)(bs * (kBTileBytesMax >> 4));
#pragma unroll
                    for (int h = 0; h < kUPT; ++h) {  // rows [h U, (h+1) U) of the B tile: U / 8 groups of 128 B
                        if (!mbar_wait(&acc_empty[as], aph ^ 1u, wctl)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)(as * U);
#pragma unroll
                        for (int k = 0; k < KSTEPS; ++k)
                            mma_f16(d_tmem, a_desc + (uint64_t)(k * (2 * kALbo >> 4)),
                                    b_desc + (uint64_t)(h * (U / 8) * (128 >> 4) + k * (2 * kBLbo >> 4)), IDESC,
                                    k > 0 ? 1u : 0u);
                        mma_commit(&acc_full[as]);
                        if (++as == kNAcc) {
                            as = 0;
                            aph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(&b_empty[bs]);
                    if (++bs == kNB) {
                        bs = 0;
                        bph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(&a_empty[ab]);
                ++i;
            }
            mma_commit(mma_done);  // arrives once every MMA issued above has completed
        }
    } else if (warp < 4) {
        // ---------------------------- A-tile builder ---------------------------
        build_a_tiles<KSTEPS, BF16>(items, n_items, probs, lref, level_stride, level, sA, a_full, a_empty, wctl,
                                    err_flag, warp, lane);
    } else {
        // ------------------------------- epilogue ------------------------------
        const int g = (warp - 4) >> 2;        // warpgroup (0 .. G-1)
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const int row = 32 * q + lane;        // cell row of this thread
        uint2 *qw = q_all + (size_t)(warp - 4) * kQCap;  // this warp's re-check queue
        // this warp's FP64 staging: kDCap entries, then its count and queue-full flag (in shared
        // memory, so the cold path holds no register across the drain loop)
        uint2 *const dw = d_all + (size_t)(warp - 4) * (kDCap + 2);
        int *const dstate = reinterpret_cast<int *>(dw + kDCap);
        if (lane == 0) dstate[0] = dstate[1] = 0;
        __syncwarp();
        float *rows = rows_all + (size_t)g * 128 * 12;   // this warpgroup's row table
        int *corr = corr_all + g * 128;
        // accumulator stage of the next unit and the parity of its phase, carried across items
        int stage = 0;
        uint32_t parity = 0;
        const uint32_t tbase = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * kCols);
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            ItemView v;
            if (!load_item(items, it, probs, lref, level_stride, level, v)) continue;
            const int nunits = kUPT * v.ntiles;
            const int pos = v.W.cell_begin + row;
            const bool valid = pos < v.ncell;
            float tau = 0.f, band = -1.f;
            if (valid) {
                const float4 m0 = v.L.cells.m32[3 * pos], m1 = v.L.cells.m32[3 * pos + 1],
                             m2 = v.L.cells.m32[3 * pos + 2];
                const float m[10] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y};
                tau = (float)tau_cs(v.P.sin_d, v.P.cos_d, v.L.cells.trig[pos]);
                band = fmaxf(cell_band<KSTEPS, BF16>(m), band_req);
            }
            int cnt = 0;
            unsigned rechecked = 0;
            {  // the cell's rotation and threshold, for re-checks of this row by any lane of the warp
                float4 R0 = make_float4(0, 0, 0, 0), R1 = R0, R2 = R0;
                if (valid) {
                    R0 = v.L.cells.R32[3 * pos];
                    R1 = v.L.cells.R32[3 * pos + 1];
                    R2 = v.L.cells.R32[3 * pos + 2];
                }
                float4 *rr = reinterpret_cast<float4 *>(rows + row * 12);
                rr[0] = R0;
                rr[1] = R1;
                rr[2] = make_float4(R2.x, tau, __int_as_float(valid ? pos : 0), 0.f);
                corr[row] = 0;
            }
            __syncwarp();
            int qn = 0;  // entries in this warp's queue (warp-uniform)
            const int64_t gbase = v.P.pool_off + v.W.pair_begin;
            // hands the staged tests to the FP64 pass with one atomic for the warp; when the
            // queue is full, flags their cells for the pass's recount instead
            auto defer_flush = [&]() {
                const int dn = dstate[0];
                int base = 0;
                if (lane == 0) base = (dstate[1] || __ldcg(amb.ovf)) ? amb.cap : atomicAdd(amb.count, dn);
                base = __shfl_sync(0xffffffffu, base, 0);
                const bool room = base <= amb.cap - dn;
                __syncwarp();
                if (lane == 0) {
                    dstate[0] = 0;
                    dstate[1] = room ? 0 : 1;
                }
                for (int k = lane; k < dn; k += 32) {
                    const uint2 e = dw[k];
                    const int cpos = __float_as_int(rows[e.y * 12 + 10]);
                    if (room) {
                        amb.q[base + k] = Amb64{v.W.prob, cpos, gbase + (int64_t)e.x};
                    } else {
                        atomicOr(&v.L.counts[cpos], kOvfBit);
                        *amb.ovf = 1;
                    }
                }
                __syncwarp();
            };
            // drains the re-check queue: one entry per lane, loads issued in parallel; the
            // tests within kBand64 of tau are staged for the FP64 pass (their fast-path count
            // removed here, their vote added there)
            auto flush = [&]() {
                for (int k0 = 0; k0 < qn; k0 += 32) {
                    const int k = k0 + lane;
                    bool in_band = false;
                    uint32_t poff = 0, rrow = 0;
                    if (k < qn) {
                        const uint2 en = qw[k];
                        rrow = 32 * q + (en.y & 31u);
                        poff = en.x;
                        const float4 *rr = reinterpret_cast<const float4 *>(rows + rrow * 12);
                        const float4 R0 = rr[0], R1 = rr[1], R2x = rr[2];
                        const float rtau = R2x.y;
                        const int64_t gp = gbase + (int64_t)en.x;
                        const float4 p0 = pool.pr[2 * gp], p1 = pool.pr[2 * gp + 1];
                        const float vv = recheck_v(R0, R1, make_float4(R2x.x, 0.f, 0.f, 0.f), p0, p1);
                        in_band = fabsf(vv - rtau) <= kBand64;
                        atomicAdd(&corr[rrow], (in_band ? 0 : (int)(vv <= rtau)) - (int)(en.y >> 5));
                        ++rechecked;
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, in_band);
                    if (bal != 0) {
                        const int dn = dstate[0];
                        if (in_band) dw[dn + __popc(bal & ((1u << lane) - 1u))] = make_uint2(poff, rrow);
                        __syncwarp();
                        if (lane == 0) dstate[0] = dn + __popc(bal);
                        __syncwarp();
                        if (dn + __popc(bal) > kDCap - 32) defer_flush();
                    }
                }
                __syncwarp();
                qn = 0;
            };
            // counts the CH values of one chunk: the tests with D < 0 into the two
            // FMA-pipe counters of tsum (sign_fma2), decoded once per two chunks;
            // returns whether the chunk holds a value within the band (one chain
            // of three-input minima of |D|, two values each).
            uint64_t tsum = kCnt0;
            auto chunk_count = [&](const uint32_t(&r)[CH]) -> uint32_t {
                float m = 4.f;  // min |D| (|D| <= 4)
#pragma unroll
                for (int e = 0; e < CH; e += 4) {
                    tsum = sign_fma2(r[e], r[e + 1], tsum);
                    tsum = sign_fma2(r[e + 2], r[e + 3], tsum);
                    m = min3_abs(m, __uint_as_float(r[e]), __uint_as_float(r[e + 1]));
                    m = min3_abs(m, __uint_as_float(r[e + 2]), __uint_as_float(r[e + 3]));
                }
                return m <= band ? 1u : 0u;
            };
            auto decode = [&]() {
                cnt += sign_fma2_count(tsum);
                tsum = kCnt0;
            };
            // queues the tests within the band of one chunk (pair offset poff in
            // the item) for the FP32 re-check; hit: this lane's chunk holds one
            auto chunk_queue = [&](const uint32_t(&r)[CH], int poff, bool hit) {
                uint32_t fm = 0, sm = 0;  // flag and D < 0 masks, constant register indices only
                if (hit) {
#pragma unroll
                    for (int e = 0; e < CH; ++e) {
                        fm |= (uint32_t)(fabsf(__uint_as_float(r[e])) <= band) << e;
                        sm |= (uint32_t)(__uint_as_float(r[e]) < 0.f) << e;
                    }
                }
                for (;;) {
                    const bool has = fm != 0;
                    const uint32_t bal = __ballot_sync(0xffffffffu, has);
                    if (bal == 0) break;
                    if (has) {
                        const int e = __ffs((int)fm) - 1;
                        fm &= fm - 1;
                        qw[qn + __popc(bal & ((1u << lane) - 1u))] =
                            make_uint2((uint32_t)(poff + e), (uint32_t)lane | (((sm >> e) & 1u) << 5));
                    }
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn > kQCap - 32) flush();
                }
            };
            int pbase = g * kCols;  // pair offset of this warpgroup's columns of the unit in the item
            for (int t = 0; t < nunits; ++t, pbase += U) {
                // warp-uniform outcome: every lane must reach the .sync.aligned tcgen05.ld below
                if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[stage], parity, wctl))) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tbase + (uint32_t)(stage * U);
                uint64_t *const empty_bar = &acc_empty[stage];
                if (++stage == kNAcc) {
                    stage = 0;
                    parity ^= 1u;
                }
                // CH-column chunks, double-buffered: the load of the next chunk is in
                // flight while this one is counted (fully unrolled, so the chunk offsets
                // are immediates and no loop bookkeeping runs per chunk)
                uint32_t ra[CH], rb[CH];
                tmem_ld(taddr, ra);
                tmem_ld_wait(ra);
                // the stage is released once this warp's last load of it has completed
                auto release = [&]() {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty_bar);
                };
                if constexpr (kCols == CH) {
                    release();
                    const uint32_t h = chunk_count(ra);
                    decode();
                    if (__any_sync(0xffffffffu, h)) chunk_queue(ra, pbase, h);
                } else {
#pragma unroll
                    for (int c = 0; c < kCols / CH; c += 2) {
                        tmem_ld(taddr + (c + 1) * CH, rb);
                        const uint32_t ha = chunk_count(ra);
                        if (__any_sync(0xffffffffu, ha)) chunk_queue(ra, pbase + c * CH, ha);
                        tmem_ld_wait(rb);
                        const bool more = c + 2 < kCols / CH;
                        if (more)
                            tmem_ld(taddr + (c + 2) * CH, ra);
                        else
                            release();
                        const uint32_t hb = chunk_count(rb);
                        decode();
                        if (__any_sync(0xffffffffu, hb)) chunk_queue(rb, pbase + (c + 1) * CH, hb);
                        if (more) tmem_ld_wait(ra);
                    }
                }
            }
            if (qn > 0) flush();
            if (dstate[0] > 0) defer_flush();
            cnt += corr[row];
            if (valid && cnt != 0) atomicAdd(&v.L.counts[pos], cnt);
            const unsigned rc = __reduce_add_sync(0xffffffffu, rechecked);
            if (lane == 0 && rc) atomicAdd(&stats[v.W.prob].rechecked, (unsigned long long)rc);
        }
    }

    // ------------------------------- teardown -------------------------------
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        if (lane == 0) {
            WaitCtl done_ctl{0, 0, kWaitNs};
            if (!mbar_wait(mma_done, 0, &done_ctl)) atomicExch(err_flag, 1);
        }
        __syncwarp();
        tc_fence_after();
        tmem_dealloc512(tmem_base);
    }
}

template <int G, int KSTEPS, bool BF16, int CH, int U>
cudaError_t prepare_t() {
    return cudaFuncSetAttribute(vote_tc_kernel<G, KSTEPS, BF16, CH, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes);
}

// The tile shapes the autotuner chooses from: variant = G (epilogue warpgroups)
// + 10 if the TMEM chunks are 16 columns wide (else 32) + 100 if the MMA unit
// is 128 pairs wide (four accumulator stages; else 256 pairs and two stages).
#define RV_TC_VARIANTS(X) X(2, 32, 256, 2) X(4, 32, 256, 4) X(2, 16, 256, 12) X(4, 16, 256, 14) \
    X(2, 32, 128, 102) X(4, 32, 128, 104) X(2, 16, 128, 112) X(4, 16, 128, 114)

template <int KSTEPS, bool BF16>
cudaError_t prepare_all() {
    cudaError_t e = cudaSuccess, x;
#define RV_PREP(G_, CH_, U_, V_) \
    if ((x = prepare_t<G_, KSTEPS, BF16, CH_, U_>()) != cudaSuccess) e = x;
    RV_TC_VARIANTS(RV_PREP)
#undef RV_PREP
    return e;
}

template <int KSTEPS, bool BF16>
cudaError_t launch_v(int variant, const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                     int level_stride, int level, PairPool pool, ProbStats *stats, float band_req, int grid,
                     int *err_flag, int test_stall, AmbQueue amb, cudaStream_t s) {
    switch (variant) {
#define RV_CASE(G_, CH_, U_, V_)                                                                             \
    case V_:                                                                                                 \
        vote_tc_kernel<G_, KSTEPS, BF16, CH_, U_><<<grid, 128 + 128 * G_, kSmemBytes, s>>>(                  \
            items, n_items, probs, lref, level_stride, level, pool, stats, band_req, err_flag,               \
            test_stall ? 1000000ull : kWaitNs, test_stall, amb);                                              \
        return cudaGetLastError();
        RV_TC_VARIANTS(RV_CASE)
#undef RV_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Sets the dynamic shared-memory limit of every variant (once, outside any
// stream capture).
cudaError_t prepare_vote_tc() {
    const cudaError_t r[4] = {prepare_all<1, false>(), prepare_all<1, true>(), prepare_all<2, false>(),
                              prepare_all<2, true>()};
    for (cudaError_t x : r)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

cudaError_t launch_vote_tc(const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                           int level_stride, int level, PairPool pool, ProbStats *stats, int prec, float band_req,
                           int variant, int grid_blocks, int *err_flag, int test_stall, AmbQueue amb,
                           cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int grid = grid_blocks < n_items ? grid_blocks : n_items;
#define RV_TC_G(KS_, BF_) \
    launch_v<KS_, BF_>(variant, items, n_items, probs, lref, level_stride, level, pool, stats, band_req, grid, \
                       err_flag, test_stall, amb, s)
    switch (prec) {
    case ROT_PREC_FP16: return RV_TC_G(1, false);
    case ROT_PREC_BF16: return RV_TC_G(1, true);
    case ROT_PREC_FP16X2: return RV_TC_G(2, false);
    case ROT_PREC_BF16X2: return RV_TC_G(2, true);
    default: return cudaErrorInvalidValue;
    }
#undef RV_TC_G
}

}  // namespace rv
