// k_vote_simt.cu -- the vote on CUDA cores in FP32 (the plain form).
//
// For cell c and pair i the vote is v = q_c^T S_i q_c <= tau_c.  With
// M_i = L(a_i)^T L'(b_i) (App. A), q^T M_i q = b_i^T R(q) a_i, so for the unit
// cell centre 2 (v - tau) = (1 - 2 tau) - sum_jk R_jk(q_c) P_jk(i) with
// P(i) = b_i a_i^T: a 9-term dot product of the cell's rotation with the pair's
// outer product.  Each test evaluates, in FP32,
//     d = fma-chain(-R_c, P_i, c0),   c0 = fl(1 - 2 fl(tau_c)),
// in the fixed order (j, k) = (0,0), (0,1), ..., (2,2), and the cell votes iff
// d <= 0 (the sign bit of d is counted).
//
// Exactness: with unit inputs (to 1e-5) every partial sum is at most 4 in
// magnitude, so |d - 2 (v - tau)_exact| <= 45 u = 2.7e-6 (u = 2^-24): 3u for
// c0, 6u for the rounding of R and P, 36u for nine FMA roundings.  Tests with
// |d| <= kBandR = 5e-6 are re-evaluated with the FP32 re-check
// |b - R_c a|^2 / 4 - c_i (error < 7e-7); those whose re-check lies within
// kBand64 = 2e-6 of the threshold go to the FP64 resolution pass
// (k_resolve64.cu), so every decision is the FP64 one.
//
// Two kernels compute the same FP32 values in the same order:
//   vote_simt_kernel   scalar: each thread owns CPT cells and runs one fmaf
//                      chain per (cell, pair);
//   vote_simt2_kernel  packed: one fma.rn.f32x2 advances the chains of the
//                      same cell for two consecutive pairs (pair-interleaved
//                      P from pool.p2x, -R duplicated in both halves), halving
//                      the issue slots spent on FMAs.  Each packed FMA rounds
//                      exactly like fmaf, so every value and decision equals
//                      the scalar kernel's.
// Padding pairs (P = 0) are never counted: the loops stop at the problem's
// last pair, and the packed kernel removes the one padding element an odd
// final pair-pair carries (its d is exactly c0).
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

constexpr int kTP = 128;      // pairs per shared-memory tile
constexpr int kThreads = 128;

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

// -R_c and c0 of a cell (an absent cell gets R = 0, c0 = 1: d = 1 for every
// pair, never counted, never in the band).
__device__ __forceinline__ void load_cell(const LevelRef &L, const ProbRef &P, int pos, bool present, float nr[9],
                                          float &tau, float &c0) {
    if (present) {
        const float4 R0 = L.cells.R32[3 * pos], R1 = L.cells.R32[3 * pos + 1], R2 = L.cells.R32[3 * pos + 2];
        nr[0] = -R0.x; nr[1] = -R0.y; nr[2] = -R0.z;
        nr[3] = -R0.w; nr[4] = -R1.x; nr[5] = -R1.y;
        nr[6] = -R1.z; nr[7] = -R1.w; nr[8] = -R2.x;
        tau = (float)tau_cs(P.sin_d, P.cos_d, L.cells.trig[pos]);
        c0 = fmaf(-2.f, tau, 1.f);
    } else {
#pragma unroll
        for (int e = 0; e < 9; ++e) nr[e] = 0.f;
        tau = -1.f;
        c0 = 1.f;
    }
}

template <int CPT>
__global__ void __launch_bounds__(kThreads, 4) vote_simt_kernel(const VoteItem *__restrict__ items, int n_items,
                                                             const ProbRef *__restrict__ probs,
                                                             const LevelRef *__restrict__ lref, int level_stride,
                                                             int level, PairPool pool, ProbStats *stats,
                                                             int *item_counter, AmbQueue amb) {
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
            float nr[CPT][9], tau[CPT], c0[CPT];
            int cnt[CPT], pos[CPT];
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                pos[k] = sub + (int)threadIdx.x + k * kThreads;
                cnt[k] = 0;
                load_cell(L, P, pos[k], pos[k] < cell_end, nr[k], tau[k], c0[k]);
            }
            const int64_t g0 = P.pool_off + W.pair_begin;
            const int ntiles = (W.pair_end - W.pair_begin) / kTP;
            const int nvalid = (int)min((int64_t)(W.pair_end - W.pair_begin), P.n - W.pair_begin);
            const float4 *src = pool.p32 + 3 * g0;
            unsigned rechecked = 0;

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
                const int jn = max(0, min(kTP, nvalid - t * kTP));  // real pairs of this tile
#pragma unroll 2
                for (int j = 0; j < jn; ++j) {
                    const float4 p0 = S[3 * j], p1 = S[3 * j + 1], p2 = S[3 * j + 2];
                    float d[CPT];
                    bool flag = false;
#pragma unroll
                    for (int k = 0; k < CPT; ++k) {
                        float x = fmaf(nr[k][0], p0.x, c0[k]);
                        x = fmaf(nr[k][1], p0.y, x);
                        x = fmaf(nr[k][2], p0.z, x);
                        x = fmaf(nr[k][3], p0.w, x);
                        x = fmaf(nr[k][4], p1.x, x);
                        x = fmaf(nr[k][5], p1.y, x);
                        x = fmaf(nr[k][6], p1.z, x);
                        x = fmaf(nr[k][7], p1.w, x);
                        x = fmaf(nr[k][8], p2.x, x);
                        d[k] = x;
                        cnt[k] += (int)(__float_as_uint(x) >> 31);
                        flag |= fabsf(x) <= kBandR;
                    }
                    if (flag) {  // rare: re-check the flagged tests of this pair
                        const int64_t gp = g0 + (int64_t)t * kTP + j;
                        const float4 q0 = pool.pr[2 * gp], q1 = pool.pr[2 * gp + 1];
#pragma unroll
                        for (int k = 0; k < CPT; ++k) {
                            if (fabsf(d[k]) <= kBandR) {
                                const float4 R0 = L.cells.R32[3 * pos[k]], R1 = L.cells.R32[3 * pos[k] + 1],
                                             R2 = L.cells.R32[3 * pos[k] + 2];
                                const float v = recheck_v(R0, R1, R2, q0, q1);
                                const int dec = decide_or_defer(v, tau[k], L, pos[k], W.prob, gp, amb);
                                cnt[k] += (dec & 1) - (int)(__float_as_uint(d[k]) >> 31);
                                ++rechecked;
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
            if ((threadIdx.x & 31) == 0 && rc) atomicAdd(&stats[W.prob].rechecked, (unsigned long long)rc);
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

constexpr int kPP = kTP / 2;  // pair-pairs per shared-memory tile (5 float4 each)

template <int CPT, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) vote_simt2_kernel(const VoteItem *__restrict__ items, int n_items,
                                                              const ProbRef *__restrict__ probs,
                                                              const LevelRef *__restrict__ lref, int level_stride,
                                                              int level, PairPool pool, ProbStats *stats,
                                                              int *item_counter, AmbQueue amb) {
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
            uint64_t mm[CPT][9], nt[CPT];  // (-R_jk, -R_jk) and (c0, c0)
            float nr[CPT][9], tau[CPT], c0[CPT];
            int cnt[CPT], pos[CPT];
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                pos[k] = sub + (int)threadIdx.x + k * kThreads;
                cnt[k] = 0;
                load_cell(L, P, pos[k], pos[k] < cell_end, nr[k], tau[k], c0[k]);
#pragma unroll
                for (int e = 0; e < 9; ++e) mm[k][e] = pack2(nr[k][e], nr[k][e]);
                nt[k] = pack2(c0[k], c0[k]);
            }
            const int64_t g0 = P.pool_off + W.pair_begin;  // even: pool offsets and item bounds are multiples of kTP
            const int ntiles = (W.pair_end - W.pair_begin) / kTP;
            const int nvalid = (int)min((int64_t)(W.pair_end - W.pair_begin), P.n - W.pair_begin);
            const float4 *src = pool.p2x + (g0 >> 1) * 5;
            unsigned rechecked = 0;
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
                const float4 *St = sh[t & 1];
                const int jn = max(0, min(kTP, nvalid - t * kTP));  // real pairs of this tile
                const int npp = (jn + 1) >> 1;               // pair-pairs to test
                float mn[CPT];
#pragma unroll
                for (int k = 0; k < CPT; ++k) mn[k] = 4.f;
#pragma unroll 1
                for (int j0 = 0; j0 < npp; j0 += kPP / 2) {  // at most 32 pair-pairs per count decode
                    const int j1 = min(npp, j0 + kPP / 2);
                    uint32_t T[CPT];
#pragma unroll
                    for (int k = 0; k < CPT; ++k) T[k] = 0;
#pragma unroll 2
                    for (int j = j0; j < j1; ++j) {
                        const ulonglong2 *S2 = reinterpret_cast<const ulonglong2 *>(St + 5 * j);
                        const ulonglong2 v0 = S2[0], v1 = S2[1], v2 = S2[2], v3 = S2[3];
                        const uint64_t v8 = *reinterpret_cast<const uint64_t *>(S2 + 4);
                        const uint64_t sv[9] = {v0.x, v0.y, v1.x, v1.y, v2.x, v2.y, v3.x, v3.y, v8};
                        // term-major: consecutive packed FMAs share the pair operand
                        uint64_t d[CPT];
#pragma unroll
                        for (int k = 0; k < CPT; ++k) d[k] = ffma2(mm[k][0], sv[0], nt[k]);
#pragma unroll
                        for (int e = 1; e < 9; ++e)
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
                if (jn & 1) {  // the odd final pair-pair carries one padding pair: d = c0 exactly
#pragma unroll
                    for (int k = 0; k < CPT; ++k) cnt[k] -= (int)(__float_as_uint(c0[k]) >> 31);
                }
                // rare: a cell of this warp has a test of this tile within the band.  The
                // whole warp recomputes that cell's values (same order, 4 pairs per lane),
                // re-checks those within the band and returns the count correction to the
                // owning lane, so no thread rescans the tile alone.
                uint32_t flag = 0;
#pragma unroll
                for (int k = 0; k < CPT; ++k) flag |= (uint32_t)(mn[k] <= kBandR) << k;
                if (__any_sync(0xffffffffu, flag != 0)) {
                    const float *Sf = reinterpret_cast<const float *>(St);
                    const int lane = threadIdx.x & 31;
#pragma unroll
                    for (int k = 0; k < CPT; ++k) {
                        for (uint32_t who = __ballot_sync(0xffffffffu, (flag >> k) & 1u); who != 0; who &= who - 1) {
                            const int src_lane = __ffs((int)who) - 1;
                            float rb[9];
#pragma unroll
                            for (int e = 0; e < 9; ++e) rb[e] = __shfl_sync(0xffffffffu, nr[k][e], src_lane);
                            const float cb = __shfl_sync(0xffffffffu, c0[k], src_lane);
                            const float tb = __shfl_sync(0xffffffffu, tau[k], src_lane);
                            const int pb = __shfl_sync(0xffffffffu, pos[k], src_lane);
                            int corr = 0;
                            for (int i = lane; i < jn; i += 32) {
                                // P_t of pair i at float 20 (i/2) + 4 (t/2) + 2 (t%2) + i%2
                                const float *q = Sf + 20 * (i >> 1) + (i & 1);
                                float x = fmaf(rb[0], q[0], cb);
                                x = fmaf(rb[1], q[2], x);
                                x = fmaf(rb[2], q[4], x);
                                x = fmaf(rb[3], q[6], x);
                                x = fmaf(rb[4], q[8], x);
                                x = fmaf(rb[5], q[10], x);
                                x = fmaf(rb[6], q[12], x);
                                x = fmaf(rb[7], q[14], x);
                                x = fmaf(rb[8], q[16], x);
                                if (fabsf(x) <= kBandR) {
                                    const int64_t gp = g0 + (int64_t)t * kTP + i;
                                    const float4 p0 = pool.pr[2 * gp], p1 = pool.pr[2 * gp + 1];
                                    const float4 R0 = L.cells.R32[3 * pb], R1 = L.cells.R32[3 * pb + 1],
                                                 R2 = L.cells.R32[3 * pb + 2];
                                    const float v = recheck_v(R0, R1, R2, p0, p1);
                                    int vote = v <= tb;
                                    ++rechecked;
                                    if (fabsf(v - tb) <= kBand64) {  // decided by the FP64 pass
                                        vote = 0;
                                        defer_or_flag(amb, L.counts, W.prob, pb, gp);
                                    }
                                    corr += vote - (int)(__float_as_uint(x) >> 31);
                                }
                            }
                            corr = __reduce_add_sync(0xffffffffu, corr);
                            if (lane == src_lane) cnt[k] += corr;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < CPT; ++k)
                if (pos[k] < cell_end && cnt[k] != 0) atomicAdd(&L.counts[pos[k]], cnt[k]);
            const unsigned rc = __reduce_add_sync(0xffffffffu, rechecked);
            if ((threadIdx.x & 31) == 0 && rc) atomicAdd(&stats[W.prob].rechecked, (unsigned long long)rc);
        }
    }
}

}  // namespace

cudaError_t launch_vote_simt(const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                             int level_stride, int level, PairPool pool, ProbStats *stats, int variant,
                             int grid_blocks, int *item_counter, AmbQueue amb, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int grid = grid_blocks < n_items ? grid_blocks : n_items;
    if (variant > 100 && !pool.p2x) return cudaErrorInvalidValue;
    // grid_blocks assumes 4 resident CTAs per SM; the packed shapes 114 / 124 fit 5 / 6
    const int g5 = min(n_items, grid_blocks / 4 * 5), g6 = min(n_items, grid_blocks / 4 * 6);
#define RV_SIMT(G_, ...) \
    __VA_ARGS__<<<G_, kThreads, 0, s>>>(items, n_items, probs, lref, level_stride, level, pool, stats, item_counter, \
                                        amb)
    switch (variant) {
    case 4: RV_SIMT(grid, vote_simt_kernel<4>); break;
    case 8: RV_SIMT(grid, vote_simt_kernel<8>); break;
    case 102: RV_SIMT(grid, vote_simt2_kernel<2, 4>); break;
    case 104: RV_SIMT(grid, vote_simt2_kernel<4, 4>); break;
    case 114: RV_SIMT(g5, vote_simt2_kernel<4, 5>); break;
    case 124: RV_SIMT(g6, vote_simt2_kernel<4, 6>); break;
    default: return cudaErrorInvalidValue;
    }
#undef RV_SIMT
    return cudaGetLastError();
}

}  // namespace rv
