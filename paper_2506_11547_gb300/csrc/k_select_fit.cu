// k_select_fit.cu -- ranking of the voted cells, top-K selection, and the
// final fit (Eq. stack, Sec. 4.2) with its refit loop.
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

// Cyclic Jacobi on a symmetric 4x4 (row-major, in place); eigenvectors in the
// columns of V; returns eigenvalues unsorted on the diagonal of A.
__device__ void jacobi4(double A[4][4], double V[4][4]) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
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
                const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = copysign(1.0, th) / (fabs(th) + sqrt(fma(th, th, 1.0)));
                const double c = rsqrt(fma(t, t, 1.0));
                const double s = t * c;
                for (int k = 0; k < 4; ++k) {
                    const double x = A[k][p], y = A[k][q];
                    A[k][p] = c * x - s * y;
                    A[k][q] = s * x + c * y;
                }
                for (int k = 0; k < 4; ++k) {
                    const double x = A[p][k], y = A[q][k];
                    A[p][k] = c * x - s * y;
                    A[q][k] = s * x + c * y;
                }
                for (int k = 0; k < 4; ++k) {
                    const double x = V[k][p], y = V[k][q];
                    V[k][p] = c * x - s * y;
                    V[k][q] = s * x + c * y;
                }
            }
        }
    }
}

// Smallest eigenvector of the symmetric matrix with unique entries
// u = [S00 S11 S22 S33 S01 S02 S03 S12 S13 S23]; returns false if the two
// smallest eigenvalues are within 1e-12 * trace (no unique minimiser).
__device__ bool smallest_eigvec(const double u[10], double q[4]) {
    double A[4][4] = {{u[0], u[4], u[5], u[6]}, {u[4], u[1], u[7], u[8]}, {u[5], u[7], u[2], u[9]},
                      {u[6], u[8], u[9], u[3]}};
    const double tr = u[0] + u[1] + u[2] + u[3];
    double V[4][4];
    jacobi4(A, V);
    int i0 = 0;
    for (int k = 1; k < 4; ++k)
        if (A[k][k] < A[i0][i0]) i0 = k;
    double l1 = DBL_MAX;
    for (int k = 0; k < 4; ++k)
        if (k != i0 && A[k][k] < l1) l1 = A[k][k];
    for (int r = 0; r < 4; ++r) q[r] = V[r][i0];
    return (l1 - A[i0][i0]) > 1e-12 * tr;
}

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

constexpr int kFitPer = 8;                     // pairs per thread per chunk
constexpr int kFitChunk = kFitThreads * kFitPer;

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

// One pass over the problem's pairs: membership by the FP32 re-check
// (|b - R a|^2/4 - c <= thr), stored in mem[]; members compacted in a fixed
// order and their b a^T summed in FP64.  Returns (in *m, *changed) block totals
// and the 9 sums in B (thread 0).
__device__ void fit_pass(const float4 *__restrict__ pr, uint8_t *mem, int64_t n, const float4 &R0, const float4 &R1,
                         const float4 &R2, float thr, bool first, int *list, double B[9], int *m_out,
                         int *chg_out) {
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int m = 0, chg = 0;
    for (int64_t base = 0; base < n; base += kFitChunk) {
        int mine[kFitPer];
        int cnt = 0;
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
        int tot;
        const int off = block_excl_scan(cnt, &tot);
#pragma unroll
        for (int e = 0; e < kFitPer; ++e)
            if (e < cnt) list[off + e] = mine[e];
        __syncthreads();
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
        m += tot;
        __syncthreads();
    }
    // fixed-order reduction of the 9 sums and the change count
    __shared__ double wsum[kFitThreads / 32][9];
    __shared__ int wchg[kFitThreads / 32];
#pragma unroll
    for (int k = 0; k < 9; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    for (int o = 16; o > 0; o >>= 1) chg += __shfl_down_sync(0xffffffffu, chg, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 9; ++k) wsum[w][k] = acc[k];
        wchg[w] = chg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int k = 0; k < 9; ++k) {
            double t = 0.0;
            for (int j = 0; j < kFitThreads / 32; ++j) t += wsum[j][k];
            B[k] = t;
        }
        for (int j = 0; j < kFitThreads / 32; ++j) c += wchg[j];
        *m_out = m;
        *chg_out = c;
    }
    __syncthreads();
}

__device__ __forceinline__ void R32_of(const double q[4], float4 &R0, float4 &R1, float4 &R2) {
    double R[9];
    quat_to_R(q, R);
    R0 = make_float4((float)R[0], (float)R[1], (float)R[2], (float)R[3]);
    R1 = make_float4((float)R[4], (float)R[5], (float)R[6], (float)R[7]);
    R2 = make_float4((float)R[8], 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(kFitThreads) fit_kernel(const ProbRef *__restrict__ probs,
                                                          const LevelRef *__restrict__ lref, int level_stride,
                                                          const int32_t *__restrict__ kept_pos, int top_k,
                                                          int refit_iters, PairPool pool, uint8_t *member,
                                                          const ProbStats *__restrict__ stats,
                                                          rot_vote_result *results) {
    const int p = blockIdx.x;
    const ProbRef P = probs[p];
    const int last = P.levels;
    const LevelRef L = lref[p * level_stride + last];
    const int wpos = kept_pos[(p * level_stride + last) * top_k];
    __shared__ double qs[4];
    __shared__ double Bs[9];
    __shared__ int s_m, s_chg, s_done, s_status, s_nin, s_refits;
    __shared__ int list[kFitChunk];
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
    // inliers of the winner: the voters of its cell (FP32 re-check decisions)
    const float tau32 = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[wpos]);
    const float4 C0 = L.cells.R32[3 * wpos], C1 = L.cells.R32[3 * wpos + 1], C2 = L.cells.R32[3 * wpos + 2];
    fit_pass(pr, mem, n, C0, C1, C2, tau32, true, list, Bs, &s_m, &s_chg);
    if (threadIdx.x == 0) {
        s_status = ROT_VOTE_OK;
        s_done = 0;
        s_refits = 0;
        s_nin = s_m;
        double u[10], q[4];
        sumS_from_B(Bs, (double)s_m, u);
        if (s_m < 2 || !smallest_eigvec(u, q)) {
            for (int k = 0; k < 4; ++k) q[k] = qc[k];
            s_status = ROT_VOTE_EDEGENERATE;
            s_done = 1;
        }
        for (int k = 0; k < 4; ++k) qs[k] = q[k];
    }
    __syncthreads();
    const float thr = (float)(P.sin_d * P.sin_d);  // refit rule: q^T S_i q <= sin^2(delta)
    for (int t = 1; t <= refit_iters && !s_done; ++t) {
        double q[4] = {qs[0], qs[1], qs[2], qs[3]};
        float4 R0, R1, R2;
        R32_of(q, R0, R1, R2);
        fit_pass(pr, mem, n, R0, R1, R2, thr, false, list, Bs, &s_m, &s_chg);
        if (threadIdx.x == 0) {
            double u[10], qn[4];
            sumS_from_B(Bs, (double)s_m, u);
            if (s_m < 2 || s_chg == 0 || !smallest_eigvec(u, qn)) {
                s_done = 1;
            } else {
                for (int k = 0; k < 4; ++k) qs[k] = qn[k];
                s_nin = s_m;
                s_refits = t;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double q[4] = {qs[0], qs[1], qs[2], qs[3]};
        canonical(q);
        double R[9];
        quat_to_R(q, R);
        rot_vote_result r;
        for (int k = 0; k < 4; ++k) r.q[k] = q[k];
        for (int k = 0; k < 9; ++k) r.R[k] = R[k];
        r.best_count = L.counts[wpos];
        r.inliers = s_nin;
        r.best_cell = L.cells.idx[wpos];
        r.best_level = last;
        r.refits = s_refits;
        r.tests = (int64_t)stats[p].tests;
        r.rechecked = (int64_t)stats[p].rechecked;
        r.ambiguous = (int64_t)stats[p].ambiguous;
        r.status = stats[p].invalid ? ROT_VOTE_EINVAL : s_status;
        r.ms_gpu = 0.f;
        r.latency_ms = 0.f;
        results[p] = r;
    }
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

cudaError_t launch_fit(const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride,
                       const int32_t *kept_pos, int top_k, int refit_iters, PairPool pool, uint8_t *member,
                       const ProbStats *stats, rot_vote_result *results, cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    fit_kernel<<<nprob, kFitThreads, 0, s>>>(probs, lref, level_stride, kept_pos, top_k, refit_iters, pool, member,
                                            stats, results);
    return cudaGetLastError();
}

}  // namespace rv
