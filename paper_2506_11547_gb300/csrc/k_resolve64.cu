// k_resolve64.cu -- the FP64 resolution pass of one level's vote.
//
// The vote kernels decide every (cell, pair) test whose FP32 re-check value
// lies more than kBand64 = 2e-6 from the threshold; the others (about 4e-6 of
// all tests for uniform outliers: the band on both sides of tau) they leave
// uncounted in a queue.  Here each queued test is decided by the FP64
// evaluation of the definition (quad_fp64: App. A's M = L(a)^T L'(b), Lemma
// 1's S = (I - M)/2, v = q^T S q, in the definition's order of IEEE double
// operations) against the cell's FP64 threshold, one test per thread, so the
// FP64 pipe serves full warps rather than the one divergent lane a vote
// kernel would give it.  A vote adds one to the cell's count; each test adds
// to the problem's resolved count, and to its ambiguous count when
// |v - tau| <= 1e-6.
#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

constexpr int kResolveThreads = 256;

__global__ void __launch_bounds__(kResolveThreads) resolve64_kernel(AmbQueue Q, const ProbRef *__restrict__ probs,
                                                                    const LevelRef *__restrict__ lref,
                                                                    int level_stride, int level, PairPool pool,
                                                                    ProbStats *stats) {
    const int n = min(*(volatile int *)Q.count, Q.cap);
    int cur = -1;  // the problem this thread's statistics belong to
    unsigned am = 0, rs = 0;
    for (int i = blockIdx.x * kResolveThreads + threadIdx.x; i < n; i += gridDim.x * kResolveThreads) {
        const Amb64 e = Q.q[i];
        if (e.prob != cur) {
            if (cur >= 0) {
                if (am) atomicAdd(&stats[cur].ambiguous, (unsigned long long)am);
                atomicAdd(&stats[cur].resolved, (unsigned long long)rs);
            }
            cur = e.prob;
            am = rs = 0;
        }
        const ProbRef &P = probs[e.prob];
        const LevelRef &L = lref[e.prob * level_stride + level];
        const int dec = decide_fp64(L.cells.q[e.pos], tau_cs(P.sin_d, P.cos_d, L.cells.trig[e.pos]),
                                    pool.pr[2 * e.gp], pool.pr[2 * e.gp + 1]);
        if (dec & 1) atomicAdd(&L.counts[e.pos], 1);
        am += (dec >> 1) & 1;
        ++rs;
    }
    // the last problem's statistics, one atomic per problem per warp
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

}  // namespace

cudaError_t launch_resolve64(AmbQueue amb, const ProbRef *probs, const LevelRef *lref, int level_stride, int level,
                             PairPool pool, ProbStats *stats, int grid_blocks, cudaStream_t s) {
    if (!amb.q || amb.cap <= 0) return cudaSuccess;
    const int need = (amb.cap + kResolveThreads - 1) / kResolveThreads;
    const int grid = grid_blocks < need ? grid_blocks : need;
    resolve64_kernel<<<grid < 1 ? 1 : grid, kResolveThreads, 0, s>>>(amb, probs, lref, level_stride, level, pool,
                                                                      stats);
    return cudaGetLastError();
}

}  // namespace rv
