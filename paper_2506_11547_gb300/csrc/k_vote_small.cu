// k_vote_small.cu -- the vote of a refinement level (a few hundred cells per
// problem against all of its pairs), pair-major.
//
// A refinement level holds at most 8 top_k cells per problem, far too few for
// the cell-major kernels to fill the GPU.  Here each thread owns one pair (the
// pair step's 256-pair tiles are the blocks), stages the level's -R_c and
// 1 - 2 tau_c in shared memory once, and tests its pair against every cell
// with the FP32 chain d = fma-chain(-R_c, b a^T, 1 - 2 tau_c) of the plain
// form (k_vote_simt.cu).  Tests with |d| <= kBandR take the FP32 re-check
// |b - R_c a|^2/4 - c, and those within kBand64 of the threshold the FP64
// resolution pass, so the counts are the exact counts of every precision
// form.  Per cell, a warp's 32 votes are summed by a ballot and a population
// count into a shared-memory counter, added to the level's counts once per
// block.  Padding pairs do not vote.
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
                                                                   ProbStats *stats, AmbQueue amb) {
    __shared__ float4 sm[kSmallMaxCells * 3];  // -R (9), c0 = 1 - 2 tau, tau (3 float4 per cell)
    __shared__ int scnt[kSmallMaxCells];
    static_assert(sizeof(float4) * kSmallMaxCells * 3 + sizeof(int) * kSmallMaxCells <= 48 * 1024, "static smem");
    const int b = blockIdx.x;
    if (b >= ntiles) return;
    const int2 tl = tiles[b];
    const ProbRef P = probs[tl.x];
    if (level > P.levels) return;  // uniform across the block
    const LevelRef L = lref[tl.x * level_stride + level];
    const int nc = min(*L.ncells, kSmallMaxCells);
    for (int c = threadIdx.x; c < nc; c += kSmallThreads) {
        const float4 R0 = L.cells.R32[3 * c], R1 = L.cells.R32[3 * c + 1], R2 = L.cells.R32[3 * c + 2];
        const float tau = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[c]);
        sm[3 * c] = make_float4(-R0.x, -R0.y, -R0.z, -R0.w);
        sm[3 * c + 1] = make_float4(-R1.x, -R1.y, -R1.z, -R1.w);
        sm[3 * c + 2] = make_float4(-R2.x, fmaf(-2.f, tau, 1.f), tau, 0.f);
        scnt[c] = 0;
    }
    __syncthreads();
    const int64_t i = (int64_t)tl.y * kPairTile + threadIdx.x;
    const bool real = i < P.n;  // padding pairs do not vote
    const int64_t g = P.pool_off + i;
    const float4 s0 = pool.p32[3 * g], s1 = pool.p32[3 * g + 1], s2 = pool.p32[3 * g + 2];
    const int lane = threadIdx.x & 31;
    unsigned rechecked = 0;
    for (int c = 0; c < nc; ++c) {
        const float4 m0 = sm[3 * c], m1 = sm[3 * c + 1], m2 = sm[3 * c + 2];
        const float tau = m2.z;
        float x = fmaf(m0.x, s0.x, m2.y);
        x = fmaf(m0.y, s0.y, x);
        x = fmaf(m0.z, s0.z, x);
        x = fmaf(m0.w, s0.w, x);
        x = fmaf(m1.x, s1.x, x);
        x = fmaf(m1.y, s1.y, x);
        x = fmaf(m1.z, s1.z, x);
        x = fmaf(m1.w, s1.w, x);
        x = fmaf(m2.x, s2.x, x);
        bool vote = real && (__float_as_uint(x) >> 31);
        if (real && fabsf(x) <= kBandR) {  // rare: the FP32 re-check decides
            const float4 R0 = L.cells.R32[3 * c], R1 = L.cells.R32[3 * c + 1], R2 = L.cells.R32[3 * c + 2];
            const float4 p0 = pool.pr[2 * g], p1 = pool.pr[2 * g + 1];
            const float v = recheck_v(R0, R1, R2, p0, p1);
            const int dec = decide_or_defer(v, tau, L, c, tl.x, g, amb);
            vote = dec & 1;
            ++rechecked;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, vote);
        if (lane == 0 && bal) atomicAdd(&scnt[c], __popc(bal));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += kSmallThreads)
        if (scnt[c]) atomicAdd(&L.counts[c], scnt[c]);
    const unsigned rc = __reduce_add_sync(0xffffffffu, rechecked);
    if (lane == 0 && rc) atomicAdd(&stats[tl.x].rechecked, (unsigned long long)rc);
}

}  // namespace

cudaError_t launch_vote_small(const ProbRef *probs, const int2 *tiles, int ntiles, const LevelRef *lref,
                              int level_stride, int level, PairPool pool, ProbStats *stats, AmbQueue amb,
                              cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    vote_small_kernel<<<ntiles, kSmallThreads, 0, s>>>(probs, tiles, ntiles, lref, level_stride, level, pool, stats,
                                                       amb);
    return cudaGetLastError();
}

}  // namespace rv
