// k_select_fit.cu -- ranking of the voted cells, top-K selection, and the
// final fit (Eq. stack, Sec. 4.2) with its refit loop.
#include <cooperative_groups.h>
#include <float.h>

#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

// Total order of candidates: score descending, then linear index ascending.
// The score is compared through an order-preserving 64-bit integer image of
// the double (integer compares run on the ALU; GB300's FP64 pipe is narrow).
struct Key {
    uint64_t key;
    int64_t idx;
    int32_t pos;
};

__device__ __forceinline__ uint64_t order_key(double s) {
    if (s == 0.0) s = 0.0;  // -0 and +0 compare equal as scores
    const uint64_t b = (uint64_t)__double_as_longlong(s);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_score(uint64_t k) {
    const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ bool better(const Key &a, const Key &b) {
    return a.key > b.key || (a.key == b.key && a.idx < b.idx);
}

__device__ __forceinline__ Key shfl_key(const Key &k, int src_lane_delta) {
    Key o;
    o.key = __shfl_down_sync(0xffffffffu, k.key, src_lane_delta);
    o.idx = __shfl_down_sync(0xffffffffu, k.idx, src_lane_delta);
    o.pos = __shfl_down_sync(0xffffffffu, k.pos, src_lane_delta);
    return o;
}

constexpr int kSelThreads = 256;
constexpr int kPerThread = kSelChunk / kSelThreads;  // 16

// Selects, in order, the best `k` of the keys held by the block (each thread
// holds up to kPerThread in registers) by k rounds of "best key strictly worse
// than the previous winner".  out[r] gets rank r; pos = -1 marks exhaustion.
__device__ void block_select(const Key (&mine)[kPerThread], int k, Cand *out) {
    __shared__ Key wbest[kSelThreads / 32];
    __shared__ Key prev_s;
    Key prev;
    prev.key = ~0ull;  // above every score
    prev.idx = -1;
    prev.pos = -1;
    const Key none = {0ull, INT64_MAX, -1};
    for (int r = 0; r < k; ++r) {
        Key best = none;
#pragma unroll
        for (int e = 0; e < kPerThread; ++e)
            if (mine[e].pos >= 0 && better(prev, mine[e]) && better(mine[e], best)) best = mine[e];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Key o = shfl_key(best, off);
            if (better(o, best)) best = o;
        }
        if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            Key b = wbest[0];
            for (int w = 1; w < kSelThreads / 32; ++w)
                if (better(wbest[w], b)) b = wbest[w];
            prev_s = b;
            Cand c;
            c.score = key_score(b.key);
            c.idx = b.idx;
            c.pos = b.pos;
            c.pad = 0;
            out[r] = c;
        }
        __syncthreads();
        prev = prev_s;
        if (prev.pos < 0) {  // exhausted: the remaining ranks stay empty
            if (threadIdx.x == 0)
                for (int rr = r + 1; rr < k; ++rr) out[rr] = Cand{0.0, -1, -1, 0};
            break;
        }
    }
}

// Phase 1: block (chunk, problem) ranks kSelChunk cells of one level.
__global__ void __launch_bounds__(kSelThreads) topk_phase1(const ProbRef *__restrict__ probs,
                                                           const LevelRef *__restrict__ lref, int level_stride,
                                                           int level, int top_k, int rank_mode, Cand *cand,
                                                           int chunks_per_prob) {
    const int chunk = blockIdx.x, p = blockIdx.y;
    const ProbRef P = probs[p];
    Cand *out = cand + ((int64_t)p * chunks_per_prob + chunk) * top_k;
    if (level > P.levels) return;
    const LevelRef L = lref[p * level_stride + level];
    const int ncell = *L.ncells;
    const int c0 = chunk * kSelChunk;
    Key mine[kPerThread];
    const double nd = (double)P.n;
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
        const int c = c0 + (int)threadIdx.x + e * kSelThreads;
        if (c < ncell) {
            const int32_t cnt = L.counts[c];
            const double t = rank_mode == ROT_RANK_RAW ? 0.0 : tau_cs(P.sin_d, P.cos_d, L.cells.trig[c]);
            mine[e].key = order_key(rank_mode == ROT_RANK_RAW ? (double)cnt : dsub((double)cnt, dmul(nd, t)));
            mine[e].idx = L.cells.idx[c];
            mine[e].pos = c;
        } else {
            mine[e].key = 0ull;
            mine[e].idx = INT64_MAX;
            mine[e].pos = -1;
        }
    }
    if (c0 >= ncell) {
        if (threadIdx.x == 0)
            for (int r = 0; r < top_k; ++r) out[r] = Cand{0.0, -1, -1, 0};
        return;
    }
    block_select(mine, top_k, out);
}

// Phase 2: block p merges its problem's chunk candidates into the kept list.
__global__ void __launch_bounds__(kSelThreads) topk_phase2(const ProbRef *__restrict__ probs,
                                                           const LevelRef *__restrict__ lref, int level_stride,
                                                           int level, int top_k, const Cand *__restrict__ cand,
                                                           int chunks_per_prob, int32_t *kept_pos, int32_t *nkept,
                                                           ProbStats *stats, Cand *scratch) {
    const int p = blockIdx.x;
    const ProbRef P = probs[p];
    if (level > P.levels) return;
    const LevelRef L = lref[p * level_stride + level];
    const int ncell = *L.ncells;
    const int nchunks = (ncell + kSelChunk - 1) / kSelChunk;
    const int ncand = nchunks * top_k;
    const Cand *src = cand + (int64_t)p * chunks_per_prob * top_k;
    Cand *tmp = scratch + (int64_t)p * top_k;
    // Candidates beyond kSelChunk per round are folded in blocks of kSelChunk:
    // select from [kept so far + next block] until all are seen.
    __shared__ Cand keep[kMaxTopK];
    __shared__ int nkeep;
    if (threadIdx.x == 0) nkeep = 0;
    __syncthreads();
    const int per_round = kSelChunk - kMaxTopK;
    for (int base = 0; base < ncand || base == 0; base += per_round) {
        Key mine[kPerThread];
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
            const int j = (int)threadIdx.x + e * kSelThreads;  // 0 .. kSelChunk-1
            Cand c;
            if (j < kMaxTopK) {
                c = j < nkeep ? keep[j] : Cand{0.0, -1, -1, 0};
            } else {
                const int ci = base + (j - kMaxTopK);
                c = ci < ncand ? src[ci] : Cand{0.0, -1, -1, 0};
            }
            mine[e].key = c.pos >= 0 ? order_key(c.score) : 0ull;
            mine[e].idx = c.pos >= 0 ? c.idx : INT64_MAX;
            mine[e].pos = c.pos;
        }
        __syncthreads();
        block_select(mine, top_k, tmp);
        __syncthreads();
        if (threadIdx.x == 0) {
            int nk = 0;
            for (int r = 0; r < top_k; ++r) {
                keep[r] = tmp[r];
                if (tmp[r].pos >= 0) ++nk;
            }
            nkeep = nk;
        }
        __syncthreads();
        if (base + per_round >= ncand) break;
    }
    if (threadIdx.x == 0) {
        for (int r = 0; r < top_k; ++r) kept_pos[(p * level_stride + level) * top_k + r] = r < nkeep ? keep[r].pos : -1;
        nkept[p * level_stride + level] = nkeep;
        atomicAdd(&stats[p].tests, (unsigned long long)ncell * (unsigned long long)P.n);
    }
}

// ---------------------------------------------------------------------------
// Fit.
// ---------------------------------------------------------------------------
constexpr int kFitThreads = 512;

__device__ __forceinline__ void canonical(double q[4]) {
    for (int k = 0; k < 4; ++k) {
        if (q[k] > 0.0) return;
        if (q[k] < 0.0) {
            for (int j = 0; j < 4; ++j) q[j] = -q[j];
            return;
        }
    }
}

// Sum of S_i over a set of m pairs from the attitude-profile matrix
// B = sum_i b_i a_i^T (App. A: S_i = (I - M_i)/2 with
// M_i = [[tr B_i, z_i^T], [z_i, B_i + B_i^T - tr(B_i) I]], B_i = b_i a_i^T,
// z_i = a_i x b_i), so only 9 FP64 multiply-adds per member are needed.
// u = [S00 S11 S22 S33 S01 S02 S03 S12 S13 S23] of the sum.
__device__ __forceinline__ void sumS_from_B(const double B[9], double m, double u[10]) {
    const double tr = B[0] + B[4] + B[8];
    u[0] = 0.5 * (m - tr);
    u[1] = 0.5 * (m - (2.0 * B[0] - tr));
    u[2] = 0.5 * (m - (2.0 * B[4] - tr));
    u[3] = 0.5 * (m - (2.0 * B[8] - tr));
    u[4] = -0.5 * (B[7] - B[5]);  // z0 = B21 - B12 = (a x b)_x summed
    u[5] = -0.5 * (B[2] - B[6]);  // z1 = B02 - B20
    u[6] = -0.5 * (B[3] - B[1]);  // z2 = B10 - B01
    u[7] = -0.5 * (B[1] + B[3]);
    u[8] = -0.5 * (B[2] + B[6]);
    u[9] = -0.5 * (B[5] + B[7]);
}

constexpr int kFitPer = 8;                     // pairs per thread per slice
constexpr int kFitSlice = kFitThreads * kFitPer;  // 4096 pairs: the unit of the fixed reduction order
constexpr int kFitMaxCluster = 8;

// Deterministic block-wide exclusive scan of a small per-thread count.
__device__ __forceinline__ int block_excl_scan(int v, int *total) {
    __shared__ int wsum[kFitThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int base = 0, tot = 0;
    for (int k = 0; k < kFitThreads / 32; ++k) {
        if (k < w) base += wsum[k];
        tot += wsum[k];
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

// One slice of a fit pass: membership by the FP32 re-check
// (|b - R a|^2/4 - c <= thr) for pairs [base, base + kFitSlice), stored in
// mem[]; members compacted in index order and their b a^T summed in FP64 by
// warp 0 in a fixed order.  Writes the slice's 9 sums, member count and
// changed count to part[0..10] (thread 0).  Depends only on the slice.
__device__ void fit_slice(const float4 *__restrict__ pr, uint8_t *mem, int64_t n, int64_t base, const float4 &R0,
                          const float4 &R1, const float4 &R2, float thr, bool first, int *list, double *part) {
    int mine[kFitPer];
    int cnt = 0, chg = 0;
#pragma unroll
    for (int e = 0; e < kFitPer; ++e) {
        const int64_t i = base + (int64_t)e * kFitThreads + threadIdx.x;
        mine[e] = -1;
        if (i < n) {
            const bool in = recheck_v(R0, R1, R2, pr[2 * i], pr[2 * i + 1]) <= thr;
            if (!first) chg += in != (mem[i] != 0);
            mem[i] = in;
            if (in) mine[cnt++] = (int)(i - base);
        }
    }
    __shared__ int wchg[kFitThreads / 32];
    for (int o = 16; o > 0; o >>= 1) chg += __shfl_down_sync(0xffffffffu, chg, o);
    if ((threadIdx.x & 31) == 0) wchg[threadIdx.x >> 5] = chg;
    int tot;
    const int off = block_excl_scan(cnt, &tot);
#pragma unroll
    for (int e = 0; e < kFitPer; ++e)
        if (e < cnt) list[off + e] = mine[e];
    __syncthreads();
    if (threadIdx.x < 32) {
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = threadIdx.x; k < tot; k += 32) {
            const int64_t i = base + list[k];
            const float4 p0 = pr[2 * i], p1 = pr[2 * i + 1];
            const double a0 = p0.x, a1 = p0.y, a2 = p0.z, b0 = p0.w, b1 = p1.x, b2 = p1.y;
            acc[0] = fma(b0, a0, acc[0]);
            acc[1] = fma(b0, a1, acc[1]);
            acc[2] = fma(b0, a2, acc[2]);
            acc[3] = fma(b1, a0, acc[3]);
            acc[4] = fma(b1, a1, acc[4]);
            acc[5] = fma(b1, a2, acc[5]);
            acc[6] = fma(b2, a0, acc[6]);
            acc[7] = fma(b2, a1, acc[7]);
            acc[8] = fma(b2, a2, acc[8]);
        }
        if (tot > 0) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        }
        if (threadIdx.x == 0) {
            for (int k = 0; k < 9; ++k) part[k] = tot > 0 ? acc[k] : 0.0;
            part[9] = (double)tot;
            int c = 0;
            for (int j = 0; j < kFitThreads / 32; ++j) c += wchg[j];
            part[10] = (double)c;
        }
    }
    __syncthreads();
}

// Warp-cooperative cyclic Jacobi on a symmetric 4x4 held in shared memory
// (FP64), accumulating rotations into V (which may start from a previous
// eigenbasis).  Each rotation's tan(phi) is estimated in FP32; (c, s) are then
// made orthogonal to FP64 precision (c = 1/sqrt(1 + t^2) by Newton steps), so
// V stays orthogonal and every sweep shrinks the off-diagonal mass by ~1e-7.
// Lanes 0..3 update row/column k = lane.  Called by one whole warp.
__device__ void jacobi4_warp(double (*A)[4], double (*V)[4]) {
    const int lane = threadIdx.x & 31, k = lane & 3;
    for (int sweep = 0; sweep < 12; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int r = 0; r < 4; ++r) {
            dia = fma(A[r][r], A[r][r], dia);
            for (int c = r + 1; c < 4; ++c) off = fma(A[r][c], A[r][c], off);
        }
        if (off <= 1e-40 * dia || off < 1e-300) break;
        for (int p = 0; p < 3; ++p) {
            for (int q = p + 1; q < 4; ++q) {
                const double apq = A[p][q];
                if (apq == 0.0) continue;
                const float th = ((float)A[q][q] - (float)A[p][p]) / (2.f * (float)apq);
                float tf = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                if (!(fabsf(tf) <= 1.f)) tf = 0.f;  // non-finite estimate: skip the rotation
                const double t = (double)tf;
                const double x = fma(t, t, 1.0);
                double r = (double)rsqrtf((float)x);
                r = r * fma(-0.5 * x, r * r, 1.5);
                r = r * fma(-0.5 * x, r * r, 1.5);
                const double c = r, s = t * r;
                __syncwarp();
                if (lane < 4) {  // A <- A J : columns p, q of row k
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
                __syncwarp();
                if (lane < 4) {  // A <- J^T A : rows p, q of column k
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                __syncwarp();
            }
        }
    }
}

__device__ __forceinline__ void R32_of(const double q[4], float4 &R0, float4 &R1, float4 &R2) {
    double R[9];
    quat_to_R(q, R);
    R0 = make_float4((float)R[0], (float)R[1], (float)R[2], (float)R[3]);
    R1 = make_float4((float)R[4], (float)R[5], (float)R[6], (float)R[7]);
    R2 = make_float4((float)R[8], 0.f, 0.f, 0.f);
}

// Shared state of the fit, owned by the cluster's rank-0 CTA.
struct FitShared {
    double q[4];
    int done, status, nin, refits;
};

// Fit of one problem per thread-block cluster (gridDim.x = problems x C):
// the C CTAs split the problem's slices round-robin and write per-slice
// partial sums to global memory; after a cluster barrier, rank 0 sums the
// slices in index order, solves the 4x4 eigenproblem and publishes q in its
// shared memory, which the other CTAs read through distributed shared memory.
// The result is independent of C and of the other problems in the batch.
__global__ void __launch_bounds__(kFitThreads) fit_kernel(const ProbRef *__restrict__ probs,
                                                          const LevelRef *__restrict__ lref, int level_stride,
                                                          const int32_t *__restrict__ kept_pos, int top_k,
                                                          int refit_iters, PairPool pool, uint8_t *member,
                                                          double *slice_part, const int64_t *slice_off,
                                                          const ProbStats *__restrict__ stats,
                                                          rot_vote_result *results) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int p = blockIdx.x / C;
    const ProbRef P = probs[p];
    const int last = P.levels;
    const LevelRef L = lref[p * level_stride + last];
    const int wpos = kept_pos[(p * level_stride + last) * top_k];
    __shared__ FitShared sh;
    __shared__ double As[4][4], Vs[4][4];
    __shared__ double Btot[11];
    __shared__ int list[kFitSlice];
    FitShared *root = cluster.map_shared_rank(&sh, 0);
    if (wpos < 0) {  // no cell at the last level (cannot happen for valid inputs)
        if (rank == 0 && threadIdx.x == 0) {
            rot_vote_result r = {};
            r.status = ROT_VOTE_EDEGENERATE;
            results[p] = r;
        }
        return;  // uniform across the cluster
    }
    const int64_t n = P.n;
    const float4 *pr = pool.pr + 2 * P.pool_off;
    uint8_t *mem = member + P.pool_off;
    double *part = slice_part + 11 * slice_off[p];
    const int64_t nslices = (n + kFitSlice - 1) / kFitSlice;
    double qc[4];
    {
        const double4_32a q4 = L.cells.q[wpos];
        qc[0] = q4.x; qc[1] = q4.y; qc[2] = q4.z; qc[3] = q4.w;
    }
    if (threadIdx.x < 16) Vs[threadIdx.x >> 2][threadIdx.x & 3] = (threadIdx.x >> 2) == (threadIdx.x & 3) ? 1.0 : 0.0;

    // iteration 0: the voters of the winning cell (FP32 re-check decisions);
    // iterations t >= 1: q_{t-1}^T S_i q_{t-1} <= sin^2(delta)
    const float thr_refit = (float)(P.sin_d * P.sin_d);
    float4 R0 = L.cells.R32[3 * wpos], R1 = L.cells.R32[3 * wpos + 1], R2 = L.cells.R32[3 * wpos + 2];
    float thr = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[wpos]);
    for (int t = 0; t <= refit_iters; ++t) {
        for (int64_t sl = rank; sl < nslices; sl += C)
            fit_slice(pr, mem, n, sl * kFitSlice, R0, R1, R2, thr, t == 0, list, part + 11 * sl);
        cluster.sync();  // every slice partial is written
        if (rank == 0) {
            if (threadIdx.x < 11) {  // slices summed in index order
                double acc = 0.0;
                for (int64_t sl = 0; sl < nslices; ++sl) acc += part[11 * sl + threadIdx.x];
                Btot[threadIdx.x] = acc;
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                const int m = (int)Btot[9], chg = (int)Btot[10];
                double u[10];
                sumS_from_B(Btot, (double)m, u);
                const double tr = u[0] + u[1] + u[2] + u[3];
                bool stop = false, degenerate = false;
                if (t == 0) {
                    degenerate = m < 2;
                } else {
                    stop = m < 2 || chg == 0;
                }
                if (!stop && !degenerate) {
                    // the sum in the current eigenbasis (warm start): A' = V^T A V, two 16-lane steps
                    const double Ain[4][4] = {{u[0], u[4], u[5], u[6]}, {u[4], u[1], u[7], u[8]},
                                              {u[5], u[7], u[2], u[9]}, {u[6], u[8], u[9], u[3]}};
                    const int er = (threadIdx.x >> 2) & 3, ec = threadIdx.x & 3;
                    double w = 0.0;
                    if (threadIdx.x < 16)
                        for (int a = 0; a < 4; ++a) w = fma(Ain[er][a], Vs[a][ec], w);  // W = A V
                    __syncwarp();
                    if (threadIdx.x < 16) As[er][ec] = w;
                    __syncwarp();
                    double x = 0.0;
                    if (threadIdx.x < 16)
                        for (int a = 0; a < 4; ++a) x = fma(Vs[a][er], As[a][ec], x);  // V^T W
                    const double vsave = threadIdx.x < 16 ? Vs[er][ec] : 0.0;
                    __syncwarp();
                    if (threadIdx.x < 16) As[er][ec] = x;
                    __syncwarp();
                    jacobi4_warp(As, Vs);
                    __syncwarp();
                    // smallest and second-smallest eigenvalue
                    int i0 = 0;
                    for (int k = 1; k < 4; ++k)
                        if (As[k][k] < As[i0][i0]) i0 = k;
                    double l1 = DBL_MAX;
                    for (int k = 0; k < 4; ++k)
                        if (k != i0 && As[k][k] < l1) l1 = As[k][k];
                    const bool gap_ok = (l1 - As[i0][i0]) > 1e-12 * tr;
                    if (threadIdx.x == 0) {
                        if (!gap_ok) {
                            if (t == 0) degenerate = true;
                            else stop = true;
                        }
                        if (!degenerate && !stop) {
                            for (int r = 0; r < 4; ++r) sh.q[r] = Vs[r][i0];
                            sh.nin = m;
                            sh.refits = t;
                        }
                    }
                    __syncwarp();
                    if (!gap_ok && threadIdx.x < 16) Vs[er][ec] = vsave;  // keep the previous basis
                }
                if (threadIdx.x == 0) {
                    if (t == 0) {
                        sh.status = degenerate ? ROT_VOTE_EDEGENERATE : ROT_VOTE_OK;
                        if (degenerate) {
                            for (int r = 0; r < 4; ++r) sh.q[r] = qc[r];
                            sh.nin = m;
                            sh.refits = 0;
                        }
                        sh.done = degenerate || refit_iters == 0;
                    } else {
                        sh.done = stop || t == refit_iters;
                    }
                }
            }
        }
        cluster.sync();  // rank 0 has published q / done
        if (root->done) break;  // uniform: every CTA reads rank 0's flag
        double q[4] = {root->q[0], root->q[1], root->q[2], root->q[3]};
        R32_of(q, R0, R1, R2);
        thr = thr_refit;
        cluster.sync();  // rank 0's state is not rewritten before everyone has read it
    }
    if (rank == 0 && threadIdx.x == 0) {
        double q[4] = {sh.q[0], sh.q[1], sh.q[2], sh.q[3]};
        canonical(q);
        double R[9];
        quat_to_R(q, R);
        rot_vote_result r;
        for (int k = 0; k < 4; ++k) r.q[k] = q[k];
        for (int k = 0; k < 9; ++k) r.R[k] = R[k];
        r.best_count = L.counts[wpos];
        r.inliers = sh.nin;
        r.best_cell = L.cells.idx[wpos];
        r.best_level = last;
        r.refits = sh.refits;
        r.tests = (int64_t)stats[p].tests;
        r.rechecked = (int64_t)stats[p].rechecked;
        r.ambiguous = (int64_t)stats[p].ambiguous;
        r.status = stats[p].invalid ? ROT_VOTE_EINVAL : sh.status;
        r.ms_gpu = 0.f;
        r.latency_ms = 0.f;
        results[p] = r;
    }
    cluster.sync();  // rank 0's shared memory stays alive until every CTA is done reading it
}

}  // namespace

cudaError_t launch_topk(const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride, int level,
                        int top_k, int rank_mode, int max_cells, Cand *cand, int chunks_per_prob,
                        int32_t *kept_pos, int32_t *nkept, ProbStats *stats, cudaStream_t s) {
    (void)max_cells;
    if (nprob <= 0) return cudaSuccess;
    dim3 g1(chunks_per_prob, nprob);
    topk_phase1<<<g1, kSelThreads, 0, s>>>(probs, lref, level_stride, level, top_k, rank_mode, cand,
                                           chunks_per_prob);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // phase-2 scratch: the tail of the candidate buffer (one top_k row per problem)
    Cand *scratch = cand + (int64_t)nprob * chunks_per_prob * top_k;
    topk_phase2<<<nprob, kSelThreads, 0, s>>>(probs, lref, level_stride, level, top_k, cand, chunks_per_prob,
                                              kept_pos, nkept, stats, scratch);
    return cudaGetLastError();
}

int fit_slices(int64_t n) { return (int)((n + kFitSlice - 1) / kFitSlice); }

cudaError_t launch_fit(const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride,
                       const int32_t *kept_pos, int top_k, int refit_iters, PairPool pool, uint8_t *member,
                       double *slice_part, const int64_t *slice_off, int cluster, const ProbStats *stats,
                       rot_vote_result *results, cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    if (cluster < 1 || cluster > kFitMaxCluster) return cudaErrorInvalidValue;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(nprob * cluster));
    lc.blockDim = dim3(kFitThreads);
    lc.dynamicSmemBytes = 0;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, fit_kernel, probs, lref, level_stride, kept_pos, top_k, refit_iters, pool, member,
                              slice_part, slice_off, stats, results);
}

}  // namespace rv
