// k_select_fit.cu -- ranking of the voted cells, top-K selection, and the
// final fit (Eq. stack, Sec. 4.2) with its refit loop.
#include <float.h>

#include <algorithm>

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

// The same selection as block_select, by ranks: the valid keys go to shared
// memory (in any order), and each key's rank is the number of keys better than
// it -- `better` is a strict total order, the indices being distinct -- so the
// keys of ranks 0 .. k-1 land in out[] in order, with no rounds.  Exhausted
// ranks are filled as block_select fills them.  Up to kRankMax valid keys (one
// per thread: the refinement levels' at most 8 K children); above that -- the
// coarse level's merge of the chunk candidates -- it runs block_select, which
// measured faster there than n^2 comparisons on one SM.
constexpr int kRankMax = kSelThreads;
__device__ void block_select_ranked(const Key (&mine)[kPerThread], int k, Cand *out) {
    __shared__ Key all[kRankMax];
    __shared__ int nall;
    if (threadIdx.x == 0) nall = 0;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kPerThread; ++e)
        if (mine[e].pos >= 0) {
            const int j = atomicAdd(&nall, 1);
            if (j < kRankMax) all[j] = mine[e];
        }
    __syncthreads();
    const int n = nall;
    __syncthreads();  // every thread has read nall before a later call resets it
    if (n > kRankMax) {  // uniform
        block_select(mine, k, out);
        return;
    }
    if ((int)threadIdx.x < n) {
        const Key me = all[threadIdx.x];
        int rank = 0;
#pragma unroll 8
        for (int j = 0; j < n; ++j) rank += better(all[j], me);
        if (rank < k) out[rank] = Cand{key_score(me.key), me.idx, me.pos, 0};
    }
    const int r = (int)threadIdx.x;
    if (r >= n && r < k)  // exhausted: the first empty rank holds the "none" key, the rest are blank
        out[r] = r == n ? Cand{key_score(0ull), INT64_MAX, -1, 0} : Cand{0.0, -1, -1, 0};
    __syncthreads();
}

// Children of one problem's kept cells: the octants of each kept cell at the
// next level that meet the ball, written to the next level's table in (rank,
// octant) order (an ordered block-wide compaction, 8 candidates per kept cell).
// Called by the whole block; keep[0..nk) are the kept cells in rank order.
__device__ void block_children(const LevelRef &L, const LevelRef &C, const Cand *keep, int nk) {
    __shared__ int warp_tot[32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5), lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = L.n_side;
    for (int t0 = 0; t0 < 8 * nk; t0 += blockDim.x) {
        const int t = t0 + (int)threadIdx.x, r = t >> 3, o = t & 7;
        bool ex = false;
        int64_t cx = 0, cy = 0, cz = 0;
        if (r < nk) {
            const int64_t pidx = L.cells.idx[keep[r].pos];
            const int64_t ix = pidx % n, iy = (pidx / n) % n, iz = pidx / (n * n);
            cx = 2 * ix + (o & 1);
            cy = 2 * iy + ((o >> 1) & 1);
            cz = 2 * iz + (o >> 2);
            ex = cell_exists(2 * L.n_side, cx, cy, cz);
        }
        const unsigned ball = __ballot_sync(0xffffffffu, ex);
        if (lane == 0) warp_tot[w] = __popc(ball);
        __syncthreads();
        int base = s_base, tot = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) base += warp_tot[k];
            tot += warp_tot[k];
        }
        if (ex) write_cell(C.cells, base + __popc(ball & ((1u << lane) - 1u)), 2 * L.n_side, C.chart, cx, cy, cz);
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *const_cast<int32_t *>(C.ncells) = s_base;
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
        block_select_ranked(mine, top_k, tmp);
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
    if (level < P.levels) block_children(L, lref[p * level_stride + level + 1], keep, nkeep);  // uniform
}

// Ranking of a level of at most kSelChunk cells (the refinement levels): one
// block per problem selects the top K and writes the next level's children.
__global__ void __launch_bounds__(kSelThreads) select_small_kernel(const ProbRef *__restrict__ probs,
                                                                   const LevelRef *__restrict__ lref,
                                                                   int level_stride, int level, int top_k,
                                                                   int rank_mode, int32_t *kept_pos, int32_t *nkept,
                                                                   ProbStats *stats) {
    const int p = blockIdx.x;
    const ProbRef P = probs[p];
    if (level > P.levels) return;
    const LevelRef L = lref[p * level_stride + level];
    const int ncell = min(*L.ncells, kSelChunk);
    Key mine[kPerThread];
    const double nd = (double)P.n;
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
        const int c = (int)threadIdx.x + e * kSelThreads;
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
    __shared__ Cand sel[kMaxTopK];
    __shared__ int nsel;
    block_select_ranked(mine, top_k, sel);
    __syncthreads();
    if (threadIdx.x == 0) {
        int nk = 0;
        for (int r = 0; r < top_k; ++r) {
            kept_pos[(p * level_stride + level) * top_k + r] = sel[r].pos;
            nk += sel[r].pos >= 0;
        }
        nkept[p * level_stride + level] = nk;
        nsel = nk;
        atomicAdd(&stats[p].tests, (unsigned long long)ncell * (unsigned long long)P.n);
    }
    __syncthreads();
    if (level < P.levels) block_children(L, lref[p * level_stride + level + 1], sel, nsel);
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

// Membership of one pair in a fit pass: q^T S_i q <= thr for the pass's q
// (the winning cell's centre and threshold, or the previous iterate and
// sin^2(delta)), by the FP32 re-check (|b - R a|^2/4 - c against fl32(thr))
// and, within kBand64 of the threshold, by the FP64 evaluation with q and the
// FP64 threshold -- so the winner's voters are exactly the pairs its vote
// counted.
__device__ __forceinline__ bool member_test(const float4 &R0, const float4 &R1, const float4 &R2, float thr,
                                            const double4_32a &qm, double thr64, const float4 &p0,
                                            const float4 &p1) {
    const float v = recheck_v(R0, R1, R2, p0, p1);
    if (!(fabsf(v - thr) <= kBand64)) return v <= thr;
    return (decide_fp64(qm, thr64, p0, p1) & 1) != 0;
}

// One slice of a fit pass: membership (member_test) for pairs
// [base, base + kFitSlice), stored in
// mem[]; members compacted in index order, thread t summing the b a^T of
// members t, t + kFitThreads, ... in FP64, and the thread sums reduced by a
// fixed pairwise tree in shared memory.  The tree skips a partner whose whole
// subtree lies at or beyond the member count: such a subtree holds only
// zeros, and adding 0.0 changes nothing, so the result is that of the full
// tree.  Writes the slice's 9 sums, member count and changed count to
// part[0..10] (thread 0).  Depends only on the slice.
__device__ void fit_slice(const float4 *__restrict__ pr, uint8_t *mem, int64_t n, int64_t base, const float4 &R0,
                          const float4 &R1, const float4 &R2, float thr, const double4_32a &qm, double thr64,
                          bool first, int *list, double (*red)[kFitThreads / 2], double *part) {
    int mine[kFitPer];
    int cnt = 0, chg = 0;
#pragma unroll
    for (int e = 0; e < kFitPer; ++e) {
        const int64_t i = base + (int64_t)e * kFitThreads + threadIdx.x;
        mine[e] = -1;
        if (i < n) {
            const bool in = member_test(R0, R1, R2, thr, qm, thr64, pr[2 * i], pr[2 * i + 1]);
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
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < tot; k += kFitThreads) {
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
    const int active = tot < kFitThreads ? tot : kFitThreads;  // threads holding a member
    constexpr int kHalf = kFitThreads / 2;
    const int t = threadIdx.x;
    // first level (stride kHalf) through shared memory into the lower half's registers
    if (t >= kHalf && t < active)
#pragma unroll
        for (int v = 0; v < 9; ++v) red[v][t - kHalf] = acc[v];
    __syncthreads();
    if (t < kHalf && t + kHalf < active)
#pragma unroll
        for (int v = 0; v < 9; ++v) acc[v] += red[v][t];
    __syncthreads();
    if (t < kHalf && t < active)
#pragma unroll
        for (int v = 0; v < 9; ++v) red[v][t] = acc[v];
    __syncthreads();
#pragma unroll 1
    for (int st = kHalf / 2; st > 0; st >>= 1) {
        if (t < st && t + st < active)
#pragma unroll
            for (int v = 0; v < 9; ++v) red[v][t] += red[v][t + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int v = 0; v < 9; ++v) part[v] = active > 0 ? red[v][0] : 0.0;
        part[9] = (double)tot;
        int c = 0;
        for (int j = 0; j < kFitThreads / 32; ++j) c += wchg[j];
        part[10] = (double)c;
    }
    __syncthreads();
}

// Cyclic Jacobi in FP32 on a symmetric 4x4 (one thread, registers): returns
// an orthogonal basis V (columns = eigenvectors) accurate to ~1e-7 relative.
__device__ void jacobi4_f32(float A[4][4], float V[4][4]) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) V[r][c] = r == c ? 1.f : 0.f;
    for (int sweep = 0; sweep < 10; ++sweep) {
        float off = 0.f, dia = 0.f;
        for (int r = 0; r < 4; ++r) {
            dia = fmaf(A[r][r], A[r][r], dia);
            for (int c = r + 1; c < 4; ++c) off = fmaf(A[r][c], A[r][c], off);
        }
        if (!(off > 1e-14f * dia) || off < 1e-37f) break;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int q = p + 1; q < 4; ++q) {
                const float apq = A[p][q];
                if (apq == 0.f) continue;
                const float th = (A[q][q] - A[p][p]) / (2.f * apq);
                float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                if (!(fabsf(t) <= 1.f)) t = 0.f;
                const float c = rsqrtf(fmaf(t, t, 1.f)), sn = t * c;
#pragma unroll
                for (int k = 0; k < 4; ++k) {  // A <- A J, V <- V J
                    const float akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                    const float vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {  // A <- J^T A
                    const float apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
            }
        }
    }
}

// Cyclic Jacobi in FP64 on a symmetric 4x4 (one thread): the textbook
// rotation zeroing A_pq with t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
// theta = (A_qq - A_pp) / (2 A_pq), c = 1 / sqrt(t^2 + 1), s = t c, applied to
// A from both sides and to V, sweeping (p, q) in row order until the
// off-diagonal sum of squares is at most 1e-40 of the diagonal's (or 50
// sweeps).  Writes the unit eigenvector of the smallest eigenvalue to q and
// returns whether the two smallest eigenvalues differ by more than 1e-12 tr.
__device__ __noinline__ bool jacobi4_f64_smallest(const double (*Ain)[4], double tr, double q[4]) {
    double A[4][4], V[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            A[r][c] = Ain[r][c];
            V[r][c] = r == c ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int r = 0; r < 4; ++r) {
            dia += A[r][r] * A[r][r];
            for (int c = r + 1; c < 4; ++c) off += A[r][c] * A[r][c];
        }
        if (!(off > 1e-40 * dia) || off < 1e-300) break;
        for (int p = 0; p < 3; ++p)
            for (int qq = p + 1; qq < 4; ++qq) {
                const double apq = A[p][qq];
                if (apq == 0.0) continue;
                const double th = (A[qq][qq] - A[p][p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 4; ++k) {  // A <- A J, V <- V J
                    const double akp = A[k][p], akq = A[k][qq];
                    A[k][p] = c * akp - sn * akq;
                    A[k][qq] = sn * akp + c * akq;
                    const double vkp = V[k][p], vkq = V[k][qq];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][qq] = sn * vkp + c * vkq;
                }
                for (int k = 0; k < 4; ++k) {  // A <- J^T A
                    const double apk = A[p][k], aqk = A[qq][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[qq][k] = sn * apk + c * aqk;
                }
            }
    }
    int i0 = 0;
    for (int k = 1; k < 4; ++k)
        if (A[k][k] < A[i0][i0]) i0 = k;
    double l1 = DBL_MAX;
    for (int k = 0; k < 4; ++k)
        if (k != i0 && A[k][k] < l1) l1 = A[k][k];
    double n2 = 0.0;
    for (int r = 0; r < 4; ++r) n2 += V[r][i0] * V[r][i0];
    const double inv = 1.0 / sqrt(n2);
    for (int r = 0; r < 4; ++r) q[r] = V[r][i0] * inv;
    return (l1 - A[i0][i0]) > 1e-12 * tr;
}

// Smallest eigenpair of the symmetric 4x4 A (FP64, in shared memory), called
// by one whole warp.  An FP32 Jacobi gives the basis u_0..u_3 (~1e-7); lane
// j < 4 then takes the FP64 Rayleigh quotient lam_j = u_j^T A u_j / u_j^T u_j
// (second-order accurate, ~1e-14 relative).
//   - Gap lam_1 - lam_0 above 1e-6 tr(A): the smallest vector v gets two FP64
//     first-order corrections v += sum_{j != i0} u_j (u_j^T r) / ((lam_i0 -
//     lam_j) u_j^T u_j), r = A v - (v^T A v / v^T v) v, which bring it to
//     ~1e-14.
//   - Smaller gap: the FP32 basis may mix the two eigenvectors and the
//     corrections need not converge, so the full FP64 Jacobi above decides:
//     its eigenvector, and its eigenvalues for the degeneracy test.
// Writes q (unit, on every lane) and returns whether the gap between the two
// smallest eigenvalues exceeds 1e-12 tr(A).
__device__ bool eig4_smallest(const double (*A)[4], float (*Vs)[4], double q[4]) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        float A32[4][4], V[4][4];
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) A32[r][c] = (float)A[r][c];
        jacobi4_f32(A32, V);
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) Vs[r][c] = V[r][c];
    }
    __syncwarp();
    const int j = lane & 3;
    double u[4], Au[4];
    for (int r = 0; r < 4; ++r) u[r] = (double)Vs[r][j];
    for (int r = 0; r < 4; ++r) Au[r] = fma(A[r][0], u[0], fma(A[r][1], u[1], fma(A[r][2], u[2], A[r][3] * u[3])));
    const double uu = fma(u[0], u[0], fma(u[1], u[1], fma(u[2], u[2], u[3] * u[3])));
    const double uAu = fma(u[0], Au[0], fma(u[1], Au[1], fma(u[2], Au[2], u[3] * Au[3])));
    const double lam = uAu / uu;
    double lams[4];
    for (int k = 0; k < 4; ++k) lams[k] = __shfl_sync(0xffffffffu, lam, k);
    int i0 = 0;
    for (int k = 1; k < 4; ++k)
        if (lams[k] < lams[i0]) i0 = k;
    double l1 = DBL_MAX;
    for (int k = 0; k < 4; ++k)
        if (k != i0 && lams[k] < l1) l1 = lams[k];
    const double tr = A[0][0] + A[1][1] + A[2][2] + A[3][3];
    if (!((l1 - lams[i0]) > 1e-6 * tr)) {  // warp-uniform: lams, i0, l1 and tr agree on every lane
        double qv[4] = {0.0, 0.0, 0.0, 0.0};
        int ok = 0;
        if (lane == 0) ok = jacobi4_f64_smallest(A, tr, qv) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        for (int r = 0; r < 4; ++r) q[r] = __shfl_sync(0xffffffffu, qv[r], 0);
        return ok != 0;
    }
    const bool gap_ok = true;
    double v[4];
    for (int r = 0; r < 4; ++r) v[r] = __shfl_sync(0xffffffffu, u[r], i0);
    if (gap_ok) {
        const double inv_uu = 1.0 / uu;  // lane j: 1 / u_j^T u_j
        for (int round = 0; round < 2; ++round) {
            double Av[4];
            for (int r = 0; r < 4; ++r) Av[r] = fma(A[r][0], v[0], fma(A[r][1], v[1], fma(A[r][2], v[2], A[r][3] * v[3])));
            const double vv = fma(v[0], v[0], fma(v[1], v[1], fma(v[2], v[2], v[3] * v[3])));
            const double vAv = fma(v[0], Av[0], fma(v[1], Av[1], fma(v[2], Av[2], v[3] * Av[3])));
            const double mu = vAv / vv;
            double res[4];
            for (int r = 0; r < 4; ++r) res[r] = fma(-mu, v[r], Av[r]);
            // lane j != i0: coefficient of u_j (the gap keeps the denominator away from 0)
            double coef = 0.0;
            if (j != i0) {
                const double ur = fma(u[0], res[0], fma(u[1], res[1], fma(u[2], res[2], u[3] * res[3])));
                coef = ur * inv_uu / (mu - lams[j]);
            }
            double cf[4];
            for (int k = 0; k < 4; ++k) cf[k] = __shfl_sync(0xffffffffu, coef, k);
            for (int r = 0; r < 4; ++r) {
                double d = 0.0;
                for (int k = 0; k < 4; ++k) d = fma(cf[k], (double)Vs[r][k], d);
                v[r] += d;
            }
        }
    }
    const double n2 = fma(v[0], v[0], fma(v[1], v[1], fma(v[2], v[2], v[3] * v[3])));
    const double inv = 1.0 / sqrt(n2);
    for (int r = 0; r < 4; ++r) q[r] = v[r] * inv;
    return gap_ok;
}

__device__ __forceinline__ void R32_of(const double q[4], float4 &R0, float4 &R1, float4 &R2) {
    double R[9];
    quat_to_R(q, R);
    R0 = make_float4((float)R[0], (float)R[1], (float)R[2], (float)R[3]);
    R1 = make_float4((float)R[4], (float)R[5], (float)R[6], (float)R[7]);
    R2 = make_float4((float)R[8], 0.f, 0.f, 0.f);
}

// The fit state of one problem in shared memory.
struct FitShared {
    double q[4];
    int done, status, nin, refits;
};

// One fit iteration's decision, by warp 0, from the member sums Btot (9 sums
// of b a^T, member count, changed count): iteration 0 fits the winner's
// voters (degenerate below 2 members or without an eigenvalue gap);
// iteration t >= 1 refits unless the set is small or unchanged.  Publishes q,
// the member count and the iteration in sh, and sh.done when the loop ends.
__device__ void fit_step_warp0(int t, int refit_iters, const double *Btot, double (*As)[4], float (*Vf)[4],
                               const double qc[4], FitShared &sh) {
    const int m = (int)Btot[9], chg = (int)Btot[10];
    double u[10];
    sumS_from_B(Btot, (double)m, u);
    bool stop = false, degenerate = false;
    if (t == 0) {
        degenerate = m < 2;
    } else {
        stop = m < 2 || chg == 0;
    }
    if (!stop && !degenerate) {
        const double Ain[4][4] = {{u[0], u[4], u[5], u[6]}, {u[4], u[1], u[7], u[8]},
                                  {u[5], u[7], u[2], u[9]}, {u[6], u[8], u[9], u[3]}};
        if (threadIdx.x < 16) As[threadIdx.x >> 2][threadIdx.x & 3] = Ain[threadIdx.x >> 2][threadIdx.x & 3];
        __syncwarp();
        double qn[4];
        const bool gap_ok = eig4_smallest(As, Vf, qn);
        if (threadIdx.x == 0) {
            if (!gap_ok) {
                if (t == 0) degenerate = true;
                else stop = true;
            }
            if (!degenerate && !stop) {
                for (int r = 0; r < 4; ++r) sh.q[r] = qn[r];
                sh.nin = m;
                sh.refits = t;
            }
        }
        __syncwarp();
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

// Writes problem p's result from the fit state.
__device__ void fit_result(int p, const LevelRef &L, int wpos, int last, const FitShared &sh,
                           const ProbStats *__restrict__ stats, rot_vote_result *results) {
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
    r.resolved = (int64_t)stats[p].resolved;
    r.status = stats[p].invalid ? ROT_VOTE_EINVAL : sh.status;
    r.ms_gpu = 0.f;
    r.latency_ms = 0.f;
    results[p] = r;
}

// One fit step of large problem k (big_list[k] = p) by one warp, once all its
// slices of iteration t are written: the slices summed in index order (read
// past L1: other SMs wrote them), the 4x4 eigen-solve, and q and the stop
// state kept in state[k]; the result is written when the fit stops.
__device__ void fit_solve_warp(int k, int p, int t, int refit_iters, const ProbRef &P, const LevelRef &L, int wpos,
                               int last, const double *slice_part, const int64_t *__restrict__ slice_off,
                               FitState *state, const ProbStats *__restrict__ stats, rot_vote_result *results,
                               FitShared &sh, double (*As)[4], float (*Vf)[4], double *Btot) {
    const int lane = threadIdx.x;
    if (lane == 0 && t > 0) {
        for (int r = 0; r < 4; ++r) sh.q[r] = state[k].q[r];
        sh.done = 0;
        sh.status = state[k].status;
        sh.nin = state[k].nin;
        sh.refits = state[k].refits;
    }
    const double *part = slice_part + 11 * slice_off[p];
    const int64_t nslices = (P.n + kFitSlice - 1) / kFitSlice;
    if (lane < 11) {  // slices summed in index order, eight loads in flight at a time
        double acc = 0.0;
        int64_t sl = 0;
        for (; sl + 8 <= nslices; sl += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + 11 * (sl + u) + lane);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u];
        }
        for (; sl < nslices; ++sl) acc += __ldcg(part + 11 * sl + lane);
        Btot[lane] = acc;
    }
    __syncwarp();
    double qc[4];
    {
        const double4_32a q4 = L.cells.q[wpos];
        qc[0] = q4.x; qc[1] = q4.y; qc[2] = q4.z; qc[3] = q4.w;
    }
    fit_step_warp0(t, refit_iters, Btot, As, Vf, qc, sh);
    __syncwarp();
    if (lane == 0) {
        FitState &st = state[k];
        for (int r = 0; r < 4; ++r) st.q[r] = sh.q[r];
        st.status = sh.status;
        st.nin = sh.nin;
        st.refits = sh.refits;
        st.done = sh.done;
        if (sh.done) fit_result(p, L, wpos, last, sh, stats, results);
    }
}

// Iteration t of the fit of the large problems (n > kFitSmallMax), all of
// them on the whole GPU, one launch per iteration: a grid-stride pass over the
// flat list of their slices (big_soff[k] is the first slice of the k-th large
// problem), skipping problems whose fit has stopped.  The block that writes a
// problem's last slice (counted in done_cnt[k], reset for the next iteration)
// then runs that problem's fit step with its first warp.  Iteration 0 takes
// the winning cell's voters (its rotation and threshold), iteration t >= 1 the
// pairs with q_{t-1}^T S_i q_{t-1} <= sin^2(delta).  The result depends only
// on the problem.
__global__ void __launch_bounds__(kFitThreads, 2) fit_iter_kernel(
    const ProbRef *__restrict__ probs, const LevelRef *__restrict__ lref, int level_stride,
    const int32_t *__restrict__ kept_pos, int top_k, int t, int refit_iters, PairPool pool, uint8_t *member,
    double *slice_part, const int64_t *__restrict__ slice_off, const int32_t *__restrict__ big_list,
    const int64_t *__restrict__ big_soff, int nbig, FitState *state, int *done_cnt,
    const ProbStats *__restrict__ stats, rot_vote_result *results) {
    __shared__ int list[kFitSlice];
    __shared__ double red[9][kFitThreads / 2];
    __shared__ FitShared sh;
    __shared__ double As[4][4];
    __shared__ float Vf[4][4];
    __shared__ double Btot[11];
    __shared__ bool last_block;
    const int64_t total = big_soff[nbig];
    for (int64_t f = blockIdx.x; f < total; f += gridDim.x) {
        int k = 0, hi = nbig - 1;  // the large problem holding slice f: largest k with big_soff[k] <= f
        while (k < hi) {
            const int mid = (k + hi + 1) >> 1;
            if (big_soff[mid] <= f) k = mid;
            else hi = mid - 1;
        }
        if (t > 0 && state[k].done) continue;  // uniform across the block
        const int p = big_list[k];
        const ProbRef P = probs[p];
        const int last = P.levels;
        const LevelRef L = lref[p * level_stride + last];
        const int wpos = kept_pos[(p * level_stride + last) * top_k];
        if (wpos < 0) {  // no cell at the last level (cannot happen for valid inputs)
            if (f == big_soff[k] && threadIdx.x == 0) {
                rot_vote_result r = {};
                r.status = ROT_VOTE_EDEGENERATE;
                results[p] = r;
                state[k].done = 1;
            }
            continue;
        }
        float4 R0, R1, R2;
        float thr;
        double4_32a qm;
        double thr64;
        if (t == 0) {
            R0 = L.cells.R32[3 * wpos];
            R1 = L.cells.R32[3 * wpos + 1];
            R2 = L.cells.R32[3 * wpos + 2];
            qm = L.cells.q[wpos];
            thr64 = tau_cs(P.sin_d, P.cos_d, L.cells.trig[wpos]);
        } else {
            const double q[4] = {state[k].q[0], state[k].q[1], state[k].q[2], state[k].q[3]};
            R32_of(q, R0, R1, R2);
            qm = make_double4_32a(q[0], q[1], q[2], q[3]);
            thr64 = dmul(P.sin_d, P.sin_d);
        }
        thr = (float)thr64;
        const int64_t sl = f - big_soff[k];
        fit_slice(pool.pr + 2 * P.pool_off, member + P.pool_off, P.n, sl * kFitSlice, R0, R1, R2, thr, qm, thr64,
                  t == 0, list, red, slice_part + 11 * (slice_off[p] + sl));
        if (threadIdx.x == 0) {
            __threadfence();  // this slice's sums are visible before it is counted
            last_block = atomicAdd(&done_cnt[k], 1) == (int)(big_soff[k + 1] - big_soff[k]) - 1;
        }
        __syncthreads();
        if (last_block) {
            if (threadIdx.x < 32) {
                __threadfence();
                fit_solve_warp(k, p, t, refit_iters, P, L, wpos, last, slice_part, slice_off, state, stats, results,
                               sh, As, Vf, Btot);
            }
            if (threadIdx.x == 0) done_cnt[k] = 0;  // every slice of iteration t is counted
        }
        __syncthreads();
    }
}


// Fit of one small problem (n <= kFitSmallMax) per CTA: the same membership
// rule, stop rule and eigen-solve as the large problems' passes.  Thread t takes the
// pairs t, t + kFitSmallThreads, ... and sums its members' b a^T in FP64 in
// that order; the sums are then reduced in a fixed tree, so the result depends
// only on the problem (not on the batch).
constexpr int kFitSmallThreads = 128;

__global__ void __launch_bounds__(kFitSmallThreads) fit_small_kernel(
    const ProbRef *__restrict__ probs, const LevelRef *__restrict__ lref, int level_stride,
    const int32_t *__restrict__ kept_pos, int top_k, int refit_iters, PairPool pool, uint8_t *member,
    const int32_t *__restrict__ plist, const ProbStats *__restrict__ stats, rot_vote_result *results) {
    const int p = plist[blockIdx.x];
    const ProbRef P = probs[p];
    const int last = P.levels;
    const LevelRef L = lref[p * level_stride + last];
    const int wpos = kept_pos[(p * level_stride + last) * top_k];
    __shared__ FitShared sh;
    __shared__ double As[4][4];
    __shared__ float Vf[4][4];
    __shared__ double Btot[11];
    __shared__ double red[kFitSmallThreads / 32][11];
    if (wpos < 0) {  // no cell at the last level (cannot happen for valid inputs)
        if (threadIdx.x == 0) {
            rot_vote_result r = {};
            r.status = ROT_VOTE_EDEGENERATE;
            results[p] = r;
        }
        return;
    }
    const int64_t n = P.n;
    const float4 *pr = pool.pr + 2 * P.pool_off;
    uint8_t *mem = member + P.pool_off;
    double qc[4];
    {
        const double4_32a q4 = L.cells.q[wpos];
        qc[0] = q4.x; qc[1] = q4.y; qc[2] = q4.z; qc[3] = q4.w;
    }
    const double thr_refit = dmul(P.sin_d, P.sin_d);
    float4 R0 = L.cells.R32[3 * wpos], R1 = L.cells.R32[3 * wpos + 1], R2 = L.cells.R32[3 * wpos + 2];
    double4_32a qm = L.cells.q[wpos];
    double thr64 = tau_cs(P.sin_d, P.cos_d, L.cells.trig[wpos]);
    float thr = (float)thr64;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = 0; t <= refit_iters; ++t) {
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        int cnt = 0, chg = 0;
        // pairs i, i + kFitSmallThreads, ... in that order; the records (and the
        // previous membership bytes) of four consecutive ones are loaded first, so
        // their loads are in flight together
        for (int64_t i0 = threadIdx.x; i0 < n; i0 += 4 * kFitSmallThreads) {
            float4 q0[4], q1[4];
            uint8_t was[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + (int64_t)u * kFitSmallThreads;
                if (i < n) {
                    q0[u] = pr[2 * i];
                    q1[u] = pr[2 * i + 1];
                    was[u] = mem[i];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + (int64_t)u * kFitSmallThreads;
                if (i >= n) break;
                const float4 p0 = q0[u], p1 = q1[u];
                const bool in = member_test(R0, R1, R2, thr, qm, thr64, p0, p1);
                if (t > 0) chg += in != (was[u] != 0);
                mem[i] = in;
                if (in) {
                    ++cnt;
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
            }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k)
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
            chg += __shfl_down_sync(0xffffffffu, chg, o);
        }
        if (lane == 0) {
            for (int k = 0; k < 9; ++k) red[w][k] = acc[k];
            red[w][9] = (double)cnt;
            red[w][10] = (double)chg;
        }
        __syncthreads();
        if (w == 0) {
            if (lane < 11) {  // warps summed in order
                double s = 0.0;
                for (int k = 0; k < kFitSmallThreads / 32; ++k) s += red[k][lane];
                Btot[lane] = s;
            }
            __syncwarp();
            fit_step_warp0(t, refit_iters, Btot, As, Vf, qc, sh);
        }
        __syncthreads();  // sh is published
        if (sh.done) break;
        const double q[4] = {sh.q[0], sh.q[1], sh.q[2], sh.q[3]};
        R32_of(q, R0, R1, R2);
        qm = make_double4_32a(q[0], q[1], q[2], q[3]);
        thr64 = thr_refit;
        thr = (float)thr64;
        __syncthreads();  // sh is read before warp 0 rewrites it
    }
    if (threadIdx.x == 0) fit_result(p, L, wpos, last, sh, stats, results);
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

cudaError_t launch_select_small(const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride, int level,
                                int top_k, int rank_mode, int32_t *kept_pos, int32_t *nkept, ProbStats *stats,
                                cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    select_small_kernel<<<nprob, kSelThreads, 0, s>>>(probs, lref, level_stride, level, top_k, rank_mode, kept_pos,
                                                      nkept, stats);
    return cudaGetLastError();
}

int fit_slices(int64_t n) { return (int)((n + kFitSlice - 1) / kFitSlice); }

cudaError_t launch_fit(const ProbRef *probs, const LevelRef *lref, int level_stride, const int32_t *kept_pos,
                       int top_k, int refit_iters, PairPool pool, uint8_t *member, double *slice_part,
                       const int64_t *slice_off, const int32_t *small_list, int nsmall, const int32_t *big_list,
                       int nbig, const int64_t *big_soff, int64_t big_slices, FitState *state, int *done_cnt,
                       int sms, const ProbStats *stats, rot_vote_result *results, cudaStream_t s) {
    if (nsmall > 0) {
        fit_small_kernel<<<nsmall, kFitSmallThreads, 0, s>>>(probs, lref, level_stride, kept_pos, top_k, refit_iters,
                                                             pool, member, small_list, stats, results);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nbig <= 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fit_iter_kernel, kFitThreads, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(done_cnt, 0, sizeof(int) * nbig, s);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(big_slices, (int64_t)sms * std::max(per_sm, 1)));
    for (int t = 0; t <= refit_iters && e == cudaSuccess; ++t) {
        fit_iter_kernel<<<grid, kFitThreads, 0, s>>>(probs, lref, level_stride, kept_pos, top_k, t, refit_iters, pool,
                                                     member, slice_part, slice_off, big_list, big_soff, nbig, state,
                                                     done_cnt, stats, results);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace rv
