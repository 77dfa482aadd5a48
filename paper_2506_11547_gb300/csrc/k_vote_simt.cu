// k_vote_simt.cu -- the vote on CUDA cores in FP32 (the plain form).
//
// Two kernels compute the same FP32 values in the same order:
//   vote_simt_kernel   scalar: each thread owns CPT cells and runs one fmaf
//                      chain per (cell, pair);
//   vote_simt2_kernel  packed: one fma.rn.f32x2 advances the chains of the
//                      same cell for two consecutive pairs (pair-interleaved
//                      S entries from pool.s2x, monomials duplicated in both
//                      halves), halving the issue slots spent on FMAs.  Each
//                      packed FMA rounds exactly like fmaf, so every value and
//                      decision equals the scalar kernel's.
//
// For cell c and pair i the test is v = m(q_c) . s_i <= tau_c (q^T S_i q as a
// 10-term dot product of the cell's monomials and the pair's S entries).  Each
// thread owns CPT cells (their monomials and thresholds live in registers);
// the block streams the item's pairs through shared memory with cp.async
// double buffering, and every thread tests its cells against each pair:
// d = fma-chain(m, s, -tau), count += signbit(d).
//
// Exactness: |d - (v - tau)_exact| <= kBandFP32 (input rounding of m, s, tau
// plus ten FMA roundings, with |m|_1 <= 4 and sum |m_k s_k| <= 1.9).  Tests
// with |d| <= kBandFP32 are re-evaluated with the FP32 re-check
// |b - R_c a|^2 / 4 - c_i (error < 7e-7), so every decision with
// |v - tau| > 1e-6 equals the FP64 decision.
#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kTP = 128;     // pairs per shared-memory tile

// Next work item of this CTA: from the atomic counter if there is one (CTAs
// take items as they finish, so no CTA is left with a long tail), else in
// grid-stride order.  Block-uniform; every thread must call it.
__device__ __forceinline__ int next_item(int *counter, int &stride_it, int *s_item) {
    if (!counter) {
        const int it = stride_it;
        stride_it += gridDim.x;
        return it;
    }
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();  // every thread has read the slot before it is reused
    return it;
}
constexpr int kThreads = 128;

template <int CPT>
__global__ void __launch_bounds__(kThreads, 4) vote_simt_kernel(const VoteItem *__restrict__ items, int n_items,
                                                             const ProbRef *__restrict__ probs,
                                                             const LevelRef *__restrict__ lref, int level_stride,
                                                             int level, PairPool pool, ProbStats *stats,
                                                             int *item_counter) {
    __shared__ __align__(16) float4 sh[2][kTP * 3];
    __shared__ int s_item;
    int stride_it = blockIdx.x;
    for (int it = next_item(item_counter, stride_it, &s_item); it < n_items;
         it = next_item(item_counter, stride_it, &s_item)) {
        const VoteItem W = items[it];
        const ProbRef P = probs[W.prob];
        if (level > P.levels) continue;  // uniform across the block
        const LevelRef L = lref[W.prob * level_stride + level];
        const int ncell = *L.ncells;
        if (W.cell_begin >= ncell) continue;
        // the item's kSimtItemCells cells, CPT x kThreads at a time
        const int cell_end = min(ncell, W.cell_begin + kSimtItemCells);
      for (int sub = W.cell_begin; sub < cell_end; sub += CPT * kThreads) {
        float m[CPT][10], tau[CPT];
        int cnt[CPT];
        int pos[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            pos[k] = sub + (int)threadIdx.x + k * kThreads;
            cnt[k] = 0;
            if (pos[k] < cell_end) {
                const float4 m0 = L.cells.m32[3 * pos[k]], m1 = L.cells.m32[3 * pos[k] + 1],
                             m2 = L.cells.m32[3 * pos[k] + 2];
                m[k][0] = m0.x; m[k][1] = m0.y; m[k][2] = m0.z; m[k][3] = m0.w;
                m[k][4] = m1.x; m[k][5] = m1.y; m[k][6] = m1.z; m[k][7] = m1.w;
                m[k][8] = m2.x; m[k][9] = m2.y;
                tau[k] = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[pos[k]]);
            } else {  // absent cell: d = 1 for every pair, never counted, never in the band
#pragma unroll
                for (int e = 0; e < 10; ++e) m[k][e] = 0.f;
                tau[k] = -1.f;
            }
        }
        const int64_t g0 = P.pool_off + W.pair_begin;
        const int npairs = W.pair_end - W.pair_begin;        // multiple of kTP (pool padding)
        const int ntiles = (npairs + kTP - 1) / kTP;
        const float4 *src = pool.s32 + 3 * g0;
        unsigned rechecked = 0, ambiguous = 0;

        auto load_tile = [&](int buf, int t) {
            const float4 *gsrc = src + (int64_t)t * kTP * 3;
            for (int e = threadIdx.x; e < kTP * 3; e += kThreads) cp_async16(&sh[buf][e], gsrc + e);
        };
        load_tile(0, 0);
        cp_async_commit();
        for (int t = 0; t < ntiles; ++t) {
            if (t + 1 < ntiles) load_tile((t + 1) & 1, t + 1);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            const float4 *S = sh[t & 1];
#pragma unroll 2
            for (int j = 0; j < kTP; ++j) {
                const float4 s0 = S[3 * j], s1 = S[3 * j + 1], s2 = S[3 * j + 2];
                float d[CPT];
                bool flag = false;
#pragma unroll
                for (int k = 0; k < CPT; ++k) {
                    float x = fmaf(m[k][0], s0.x, -tau[k]);
                    x = fmaf(m[k][1], s0.y, x);
                    x = fmaf(m[k][2], s0.z, x);
                    x = fmaf(m[k][3], s0.w, x);
                    x = fmaf(m[k][4], s1.x, x);
                    x = fmaf(m[k][5], s1.y, x);
                    x = fmaf(m[k][6], s1.z, x);
                    x = fmaf(m[k][7], s1.w, x);
                    x = fmaf(m[k][8], s2.x, x);
                    x = fmaf(m[k][9], s2.y, x);
                    d[k] = x;
                    cnt[k] += (int)(__float_as_uint(x) >> 31);
                    flag |= fabsf(x) <= kBandFP32;
                }
                if (flag) {  // rare: re-check the flagged tests of this pair
                    const int64_t gp = g0 + (int64_t)t * kTP + j;
                    const float4 p0 = pool.pr[2 * gp], p1 = pool.pr[2 * gp + 1];
#pragma unroll
                    for (int k = 0; k < CPT; ++k) {
                        if (fabsf(d[k]) <= kBandFP32) {
                            const float4 R0 = L.cells.R32[3 * pos[k]], R1 = L.cells.R32[3 * pos[k] + 1],
                                         R2 = L.cells.R32[3 * pos[k] + 2];
                            const float v = recheck_v(R0, R1, R2, p0, p1);
                            const int vote = v <= tau[k];
                            cnt[k] += vote - (int)(__float_as_uint(d[k]) >> 31);
                            ++rechecked;
                            ambiguous += fabsf(v - tau[k]) <= kAmbig;
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < CPT; ++k)
            if (pos[k] < cell_end && cnt[k] != 0) atomicAdd(&L.counts[pos[k]], cnt[k]);
        const unsigned rc = __reduce_add_sync(0xffffffffu, rechecked);
        const unsigned am = __reduce_add_sync(0xffffffffu, ambiguous);
        if ((threadIdx.x & 31) == 0) {
            if (rc) atomicAdd(&stats[W.prob].rechecked, (unsigned long long)rc);
            if (am) atomicAdd(&stats[W.prob].ambiguous, (unsigned long long)am);
        }
      }
    }
}

__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
// Sign bytes of two FP32 values, each twice: [s(a), s(b), s(a), s(b)], s(x) = 0xFF if x's sign bit is set.
__device__ __forceinline__ uint32_t sign_bytes2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, 0xFBFB;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
// Number of set sign bits among the 2k values whose sign_bytes2 words sum (mod 2^32) to t, k <= 63:
// t = 255 X, X = sum_i n_i 256^i; 255 is odd, so X = t 255^-1 mod 2^32, and 2 (n_0 + n_1) is the
// top byte of X 0x01010101 (0xFBFCFDFF = 255^-1 0x01010101 mod 2^32).
__device__ __forceinline__ int sign_count(uint32_t t) { return (int)((t * 0xFBFCFDFFu) >> 25); }
// min(m, |x|, |y|).
__device__ __forceinline__ float min3_abs(float m, float x, float y) {
    float r;
    asm("min.abs.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(x), "f"(y));
    return r;
}

constexpr int kPP = kTP / 2;  // pair-pairs per shared-memory tile

template <int CPT>
__global__ void __launch_bounds__(kThreads, 4) vote_simt2_kernel(const VoteItem *__restrict__ items, int n_items,
                                                              const ProbRef *__restrict__ probs,
                                                              const LevelRef *__restrict__ lref, int level_stride,
                                                              int level, PairPool pool, ProbStats *stats,
                                                              int *item_counter) {
    __shared__ __align__(16) float4 sh[2][kPP * 5];
    __shared__ int s_item;
    int stride_it = blockIdx.x;
    for (int it = next_item(item_counter, stride_it, &s_item); it < n_items;
         it = next_item(item_counter, stride_it, &s_item)) {
        const VoteItem W = items[it];
        const ProbRef P = probs[W.prob];
        if (level > P.levels) continue;  // uniform across the block
        const LevelRef L = lref[W.prob * level_stride + level];
        const int ncell = *L.ncells;
        if (W.cell_begin >= ncell) continue;
        const int cell_end = min(ncell, W.cell_begin + kSimtItemCells);
        for (int sub = W.cell_begin; sub < cell_end; sub += CPT * kThreads) {
            uint64_t mm[CPT][10], nt[CPT];  // (m_k, m_k) and (-tau, -tau)
            float m[CPT][10], tau[CPT];
            int cnt[CPT], pos[CPT];
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                pos[k] = sub + (int)threadIdx.x + k * kThreads;
                cnt[k] = 0;
                if (pos[k] < cell_end) {
                    const float4 m0 = L.cells.m32[3 * pos[k]], m1 = L.cells.m32[3 * pos[k] + 1],
                                 m2 = L.cells.m32[3 * pos[k] + 2];
                    m[k][0] = m0.x; m[k][1] = m0.y; m[k][2] = m0.z; m[k][3] = m0.w;
                    m[k][4] = m1.x; m[k][5] = m1.y; m[k][6] = m1.z; m[k][7] = m1.w;
                    m[k][8] = m2.x; m[k][9] = m2.y;
                    tau[k] = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[pos[k]]);
                } else {  // absent cell: d = 1 for every pair, never counted, never in the band
#pragma unroll
                    for (int e = 0; e < 10; ++e) m[k][e] = 0.f;
                    tau[k] = -1.f;
                }
#pragma unroll
                for (int e = 0; e < 10; ++e) mm[k][e] = pack2(m[k][e], m[k][e]);
                nt[k] = pack2(-tau[k], -tau[k]);
            }
            const int64_t g0 = P.pool_off + W.pair_begin;  // even: pool offsets and item bounds are multiples of kTP
            const int ntiles = (W.pair_end - W.pair_begin) / kTP;
            const float4 *src = pool.s2x + (g0 >> 1) * 5;
            unsigned rechecked = 0, ambiguous = 0;
            auto load_tile = [&](int buf, int t) {
                const float4 *gsrc = src + (int64_t)t * kPP * 5;
                for (int e = threadIdx.x; e < kPP * 5; e += kThreads) cp_async16(&sh[buf][e], gsrc + e);
            };
            load_tile(0, 0);
            cp_async_commit();
            for (int t = 0; t < ntiles; ++t) {
                if (t + 1 < ntiles) load_tile((t + 1) & 1, t + 1);
                cp_async_commit();
                cp_async_wait<1>();
                __syncthreads();
                const ulonglong2 *S2 = reinterpret_cast<const ulonglong2 *>(sh[t & 1]);
                float mn[CPT];
#pragma unroll
                for (int k = 0; k < CPT; ++k) mn[k] = 4.f;
#pragma unroll 1
                for (int half = 0; half < 2; ++half) {  // 32 pair-pairs per count decode
                    uint32_t T[CPT];
#pragma unroll
                    for (int k = 0; k < CPT; ++k) T[k] = 0;
#pragma unroll 2
                    for (int j = half * (kPP / 2); j < (half + 1) * (kPP / 2); ++j) {
                        const ulonglong2 v0 = S2[5 * j], v1 = S2[5 * j + 1], v2 = S2[5 * j + 2], v3 = S2[5 * j + 3],
                                         v4 = S2[5 * j + 4];
                        // term-major: consecutive packed FMAs share the pair operand; each
                        // cell's chain keeps the order m_0 s_0 - tau, + m_1 s_1, ..., + m_9 s_9
                        const uint64_t sv[10] = {v0.x, v0.y, v1.x, v1.y, v2.x, v2.y, v3.x, v3.y, v4.x, v4.y};
                        uint64_t d[CPT];
#pragma unroll
                        for (int k = 0; k < CPT; ++k) d[k] = ffma2(mm[k][0], sv[0], nt[k]);
#pragma unroll
                        for (int e = 1; e < 10; ++e)
#pragma unroll
                            for (int k = 0; k < CPT; ++k) d[k] = ffma2(mm[k][e], sv[e], d[k]);
#pragma unroll
                        for (int k = 0; k < CPT; ++k) {
                            const uint32_t lo = (uint32_t)d[k], hi = (uint32_t)(d[k] >> 32);
                            T[k] += sign_bytes2(lo, hi);
                            mn[k] = min3_abs(mn[k], __uint_as_float(lo), __uint_as_float(hi));
                        }
                    }
#pragma unroll
                    for (int k = 0; k < CPT; ++k) cnt[k] += sign_count(T[k]);
                }
                // rare: a cell of this warp has a test of this tile within the band.  The
                // whole warp recomputes that cell's 128 values (same order, 4 pairs per
                // lane), re-checks those within the band and returns the count correction
                // to the owning lane, so no thread rescans the tile alone.
                uint32_t flag = 0;
#pragma unroll
                for (int k = 0; k < CPT; ++k) flag |= (uint32_t)(mn[k] <= kBandFP32) << k;
                if (__any_sync(0xffffffffu, flag != 0)) {
                    const float *Sf = reinterpret_cast<const float *>(sh[t & 1]);
                    const int lane = threadIdx.x & 31;
#pragma unroll
                    for (int k = 0; k < CPT; ++k) {
                        for (uint32_t who = __ballot_sync(0xffffffffu, (flag >> k) & 1u); who != 0; who &= who - 1) {
                            const int src = __ffs((int)who) - 1;
                            float mb[10];
#pragma unroll
                            for (int e = 0; e < 10; ++e) mb[e] = __shfl_sync(0xffffffffu, m[k][e], src);
                            const float tb = __shfl_sync(0xffffffffu, tau[k], src);
                            const int pb = __shfl_sync(0xffffffffu, pos[k], src);
                            int corr = 0;
                            for (int i = lane; i < kTP; i += 32) {
                                const float *q = Sf + 20 * (i >> 1) + (i & 1);  // s_2k at q[4k], s_2k+1 at q[4k + 2]
                                float x = fmaf(mb[0], q[0], -tb);
                                x = fmaf(mb[1], q[2], x);
                                x = fmaf(mb[2], q[4], x);
                                x = fmaf(mb[3], q[6], x);
                                x = fmaf(mb[4], q[8], x);
                                x = fmaf(mb[5], q[10], x);
                                x = fmaf(mb[6], q[12], x);
                                x = fmaf(mb[7], q[14], x);
                                x = fmaf(mb[8], q[16], x);
                                x = fmaf(mb[9], q[18], x);
                                if (fabsf(x) <= kBandFP32) {
                                    const int64_t gp = g0 + (int64_t)t * kTP + i;
                                    const float4 p0 = pool.pr[2 * gp], p1 = pool.pr[2 * gp + 1];
                                    const float4 R0 = L.cells.R32[3 * pb], R1 = L.cells.R32[3 * pb + 1],
                                                 R2 = L.cells.R32[3 * pb + 2];
                                    const float v = recheck_v(R0, R1, R2, p0, p1);
                                    corr += (int)(v <= tb) - (int)(__float_as_uint(x) >> 31);
                                    ++rechecked;
                                    ambiguous += fabsf(v - tb) <= kAmbig;
                                }
                            }
                            corr = __reduce_add_sync(0xffffffffu, corr);
                            if (lane == src) cnt[k] += corr;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < CPT; ++k)
                if (pos[k] < cell_end && cnt[k] != 0) atomicAdd(&L.counts[pos[k]], cnt[k]);
            const unsigned rc = __reduce_add_sync(0xffffffffu, rechecked);
            const unsigned am = __reduce_add_sync(0xffffffffu, ambiguous);
            if ((threadIdx.x & 31) == 0) {
                if (rc) atomicAdd(&stats[W.prob].rechecked, (unsigned long long)rc);
                if (am) atomicAdd(&stats[W.prob].ambiguous, (unsigned long long)am);
            }
        }
    }
}

}  // namespace

cudaError_t launch_vote_simt(const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                             int level_stride, int level, PairPool pool, ProbStats *stats, int variant,
                             int grid_blocks, int *item_counter, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int grid = grid_blocks < n_items ? grid_blocks : n_items;
    if (variant > 100 && !pool.s2x) return cudaErrorInvalidValue;
    switch (variant) {
    case 102: vote_simt2_kernel<2><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats, item_counter); break;
    case 104: vote_simt2_kernel<4><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats, item_counter); break;
    case 2: vote_simt_kernel<2><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats, item_counter); break;
    case 4: vote_simt_kernel<4><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats, item_counter); break;
    case 8: vote_simt_kernel<8><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats, item_counter); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rv
