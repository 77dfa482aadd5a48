// k_resolve64.cu -- the FP64 resolution pass of one level's vote.
//
// The vote kernels decide every (cell, pair) test whose FP32 re-check value
// lies more than kBand64 = 2e-6 from the threshold; the others (about 4e-6 of
// all tests for uniform outliers: the band on both sides of tau) they leave
// uncounted in a queue.  This pass decides them by the FP64 evaluation of the
// definition (quad_fp64: App. A's M = L(a)^T L'(b), Lemma 1's S = (I - M)/2,
// v = q^T S q, in the definition's order of IEEE double operations) against
// the cell's FP64 threshold, one test per thread, so the FP64 pipe serves full
// warps rather than the one divergent lane a vote kernel would give it.
//   1. Each queued test adds its vote to the cell's count, and to the
//      problem's resolved count (and ambiguous count when |v - tau| <= 1e-6).
//   2. If the queue overflowed, the cells the vote flagged (kOvfBit in the
//      count) are recounted from all of their pairs, one block per cell, with
//      the same decision (FP32 re-check outside kBand64, FP64 inside); their
//      queued tests, if any, are skipped in step 1.
// Step 2 clears each recounted cell's flag, so it runs as a second launch after
// step 1 has finished: in one launch a block done with step 2 could clear a flag
// that a slower block's step 1 still has to see.
#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

constexpr int kResolveThreads = 256;

// Adds this thread's (ambiguous, resolved) of problem `cur` to its statistics,
// one atomic per problem per warp; called by the whole warp.
__device__ __forceinline__ void flush_stats(int cur, unsigned am, unsigned rs, ProbStats *stats) {
    const int lane = threadIdx.x & 31;
    for (unsigned pending = __ballot_sync(0xffffffffu, cur >= 0); pending != 0;) {
        const int leader = __ffs((int)pending) - 1;
        const int key = __shfl_sync(0xffffffffu, cur, leader);
        const bool mine = ((pending >> lane) & 1u) && cur == key;
        const unsigned a = __reduce_add_sync(0xffffffffu, mine ? am : 0u);
        const unsigned r = __reduce_add_sync(0xffffffffu, mine ? rs : 0u);
        if (lane == leader) {
            if (a) atomicAdd(&stats[key].ambiguous, (unsigned long long)a);
            atomicAdd(&stats[key].resolved, (unsigned long long)r);
        }
        pending &= ~__ballot_sync(0xffffffffu, mine);
    }
}

__global__ void __launch_bounds__(kResolveThreads) resolve64_kernel(AmbQueue Q, const ProbRef *__restrict__ probs,
                                                                    int nprob, const LevelRef *__restrict__ lref,
                                                                    int level_stride, int level, PairPool pool,
                                                                    ProbStats *stats) {
    // ---- 1. the queued tests (cells flagged in step 2's sense are left to it) ----
    const int n = min(*(volatile int *)Q.count, Q.cap);
    int cur = -1;  // the problem this thread's statistics belong to
    unsigned am = 0, rs = 0;
    for (int i = blockIdx.x * kResolveThreads + threadIdx.x; i < n; i += gridDim.x * kResolveThreads) {
        const Amb64 e = Q.q[i];
        const LevelRef &L = lref[e.prob * level_stride + level];
        if (L.counts[e.pos] & kOvfBit) continue;  // recounted whole in step 2
        if (e.prob != cur) {
            if (cur >= 0) {
                if (am) atomicAdd(&stats[cur].ambiguous, (unsigned long long)am);
                atomicAdd(&stats[cur].resolved, (unsigned long long)rs);
            }
            cur = e.prob;
            am = rs = 0;
        }
        const ProbRef &P = probs[e.prob];
        const int dec = decide_fp64(L.cells.q[e.pos], tau_cs(P.sin_d, P.cos_d, L.cells.trig[e.pos]),
                                    pool.pr[2 * e.gp], pool.pr[2 * e.gp + 1]);
        if (dec & 1) atomicAdd(&L.counts[e.pos], 1);
        am += (dec >> 1) & 1;
        ++rs;
    }
    flush_stats(cur, am, rs, stats);
}

__global__ void __launch_bounds__(kResolveThreads) recount64_kernel(AmbQueue Q, const ProbRef *__restrict__ probs,
                                                                    int nprob, const LevelRef *__restrict__ lref,
                                                                    int level_stride, int level, PairPool pool,
                                                                    ProbStats *stats) {
    // ---- 2. cells flagged when the queue was full: recount from all pairs ----
    if (!*(volatile int *)Q.ovf) return;
    __shared__ unsigned red[3][kResolveThreads / 32];
    for (int p = 0; p < nprob; ++p) {
        const ProbRef P = probs[p];
        if (level > P.levels) continue;
        const LevelRef L = lref[p * level_stride + level];
        const int nc = *L.ncells;
        for (int c = blockIdx.x; c < nc; c += gridDim.x) {
            if (!(L.counts[c] & kOvfBit)) continue;  // uniform across the block
            const float4 R0 = L.cells.R32[3 * c], R1 = L.cells.R32[3 * c + 1], R2 = L.cells.R32[3 * c + 2];
            const double tau64 = tau_cs(P.sin_d, P.cos_d, L.cells.trig[c]);
            const float tau32 = (float)tau64;
            unsigned cnt = 0, amb = 0, res = 0;
            for (int64_t i = threadIdx.x; i < P.n; i += kResolveThreads) {
                const float4 p0 = pool.pr[2 * (P.pool_off + i)], p1 = pool.pr[2 * (P.pool_off + i) + 1];
                const float v = recheck_v(R0, R1, R2, p0, p1);
                if (!(fabsf(v - tau32) <= kBand64)) {
                    cnt += v <= tau32;
                } else {
                    const int dec = decide_fp64(L.cells.q[c], tau64, p0, p1);
                    cnt += dec & 1;
                    amb += (dec >> 1) & 1;
                    ++res;
                }
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            amb = __reduce_add_sync(0xffffffffu, amb);
            res = __reduce_add_sync(0xffffffffu, res);
            if ((threadIdx.x & 31) == 0) {
                red[0][threadIdx.x >> 5] = cnt;
                red[1][threadIdx.x >> 5] = amb;
                red[2][threadIdx.x >> 5] = res;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned tc = 0, ta = 0, tr = 0;
                for (int w = 0; w < kResolveThreads / 32; ++w) {
                    tc += red[0][w];
                    ta += red[1][w];
                    tr += red[2][w];
                }
                L.counts[c] = (int32_t)tc;  // replaces the partial count and its flag
                if (ta) atomicAdd(&stats[p].ambiguous, (unsigned long long)ta);
                if (tr) atomicAdd(&stats[p].resolved, (unsigned long long)tr);
                atomicAdd(&stats[p].rechecked, (unsigned long long)P.n);
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_resolve64(AmbQueue amb, const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride,
                             int level, PairPool pool, ProbStats *stats, int grid_blocks, cudaStream_t s) {
    if (!amb.count || !amb.ovf) return cudaErrorInvalidValue;
    const int grid = grid_blocks < 1 ? 1 : grid_blocks;
    resolve64_kernel<<<grid, kResolveThreads, 0, s>>>(amb, probs, nprob, lref, level_stride, level, pool, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // step 2 after step 1 on the same stream (returns at once when the queue never filled)
    recount64_kernel<<<grid, kResolveThreads, 0, s>>>(amb, probs, nprob, lref, level_stride, level, pool, stats);
    return cudaGetLastError();
}

}  // namespace rv
