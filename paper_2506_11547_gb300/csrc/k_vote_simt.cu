// k_vote_simt.cu -- the vote on CUDA cores in FP32 (the plain form).
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
constexpr int kThreads = 128;

template <int CPT>
__global__ void __launch_bounds__(kThreads, 4) vote_simt_kernel(const VoteItem *__restrict__ items, int n_items,
                                                             const ProbRef *__restrict__ probs,
                                                             const LevelRef *__restrict__ lref, int level_stride,
                                                             int level, PairPool pool, ProbStats *stats) {
    __shared__ __align__(16) float4 sh[2][kTP * 3];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
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

}  // namespace

cudaError_t launch_vote_simt(const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                             int level_stride, int level, PairPool pool, ProbStats *stats, int cells_per_thread,
                             int grid_blocks, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int grid = grid_blocks < n_items ? grid_blocks : n_items;
    switch (cells_per_thread) {
    case 2: vote_simt_kernel<2><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats); break;
    case 4: vote_simt_kernel<4><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats); break;
    case 8: vote_simt_kernel<8><<<grid, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rv
