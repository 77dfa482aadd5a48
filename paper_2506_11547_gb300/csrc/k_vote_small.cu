// k_vote_small.cu -- the vote of a refinement level (a few hundred cells per
// problem against all of its pairs), pair-major.
//
// A refinement level holds at most 8 top_k cells per problem, far too few for
// the cell-major kernels to fill the GPU.  Here each thread owns one pair (the
// pair step's 256-pair tiles are the blocks), stages the level's monomials and
// thresholds in shared memory once, and tests its pair against every cell with
// the FP32 chain d = fma-chain(m, s, -tau) of the plain form.  Tests with
// |d| <= kBandFP32 take the FP32 re-check |b - R_c a|^2/4 - c, so the counts
// are the exact counts of every precision form.  Per cell, a warp's 32 votes
// are summed by a ballot and a population count into a shared-memory counter,
// added to the level's counts once per block.
#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

constexpr int kSmallThreads = kPairTile;   // one pair per thread, one pair tile per block
constexpr int kSmallMaxCells = 8 * kMaxTopK;  // refinement levels hold at most 8 top_k cells

__global__ void __launch_bounds__(kSmallThreads) vote_small_kernel(const ProbRef *__restrict__ probs,
                                                                   const int2 *__restrict__ tiles, int ntiles,
                                                                   const LevelRef *__restrict__ lref,
                                                                   int level_stride, int level, PairPool pool,
                                                                   ProbStats *stats) {
    __shared__ float4 sm[kSmallMaxCells * 3];  // monomials (3 float4 per cell)
    __shared__ float stau[kSmallMaxCells];
    __shared__ int scnt[kSmallMaxCells];
    const int b = blockIdx.x;
    if (b >= ntiles) return;
    const int2 tl = tiles[b];
    const ProbRef P = probs[tl.x];
    if (level > P.levels) return;  // uniform across the block
    const LevelRef L = lref[tl.x * level_stride + level];
    const int nc = min(*L.ncells, kSmallMaxCells);
    for (int e = threadIdx.x; e < 3 * nc; e += kSmallThreads) sm[e] = L.cells.m32[e];
    for (int c = threadIdx.x; c < nc; c += kSmallThreads) {
        stau[c] = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[c]);
        scnt[c] = 0;
    }
    __syncthreads();
    const int64_t g = P.pool_off + (int64_t)tl.y * kPairTile + threadIdx.x;  // padding pairs (S = 4I) never vote
    const float4 s0 = pool.s32[3 * g], s1 = pool.s32[3 * g + 1], s2 = pool.s32[3 * g + 2];
    const int lane = threadIdx.x & 31;
    unsigned rechecked = 0, ambiguous = 0;
    for (int c = 0; c < nc; ++c) {
        const float4 m0 = sm[3 * c], m1 = sm[3 * c + 1], m2 = sm[3 * c + 2];
        const float tau = stau[c];
        float x = fmaf(m0.x, s0.x, -tau);
        x = fmaf(m0.y, s0.y, x);
        x = fmaf(m0.z, s0.z, x);
        x = fmaf(m0.w, s0.w, x);
        x = fmaf(m1.x, s1.x, x);
        x = fmaf(m1.y, s1.y, x);
        x = fmaf(m1.z, s1.z, x);
        x = fmaf(m1.w, s1.w, x);
        x = fmaf(m2.x, s2.x, x);
        x = fmaf(m2.y, s2.y, x);
        bool vote = __float_as_uint(x) >> 31;
        if (fabsf(x) <= kBandFP32) {  // rare: the FP32 re-check decides
            const float4 R0 = L.cells.R32[3 * c], R1 = L.cells.R32[3 * c + 1], R2 = L.cells.R32[3 * c + 2];
            const float v = recheck_v(R0, R1, R2, pool.pr[2 * g], pool.pr[2 * g + 1]);
            vote = v <= tau;
            ++rechecked;
            ambiguous += fabsf(v - tau) <= kAmbig;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, vote);
        if (lane == 0 && bal) atomicAdd(&scnt[c], __popc(bal));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += kSmallThreads)
        if (scnt[c]) atomicAdd(&L.counts[c], scnt[c]);
    const unsigned rc = __reduce_add_sync(0xffffffffu, rechecked);
    const unsigned am = __reduce_add_sync(0xffffffffu, ambiguous);
    if (lane == 0) {
        if (rc) atomicAdd(&stats[tl.x].rechecked, (unsigned long long)rc);
        if (am) atomicAdd(&stats[tl.x].ambiguous, (unsigned long long)am);
    }
}

}  // namespace

cudaError_t launch_vote_small(const ProbRef *probs, const int2 *tiles, int ntiles, const LevelRef *lref,
                              int level_stride, int level, PairPool pool, ProbStats *stats, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    vote_small_kernel<<<ntiles, kSmallThreads, 0, s>>>(probs, tiles, ntiles, lref, level_stride, level, pool, stats);
    return cudaGetLastError();
}

}  // namespace rv
