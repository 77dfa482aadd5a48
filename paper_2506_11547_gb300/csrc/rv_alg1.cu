// rv_alg1.cu -- Alg. 1 (Sec. 4.3.2), the paper's own voting: every pair's
// circle of rotations (Sec. 4.1) sampled at J angles, each sample projected
// stereographically (Sec. 4.3.1) and counted in an n^3 accumulator over
// [-1, 1]^3, then the argmax and the inverse projection of its centre.
//
// The accumulator holds 16-bit counters, two cells per 32-bit word (see
// Acc16).  The vote adds with return-less atomics; the argmax pass checks the
// sum of the counts against the samples cast, and only when a counter wrapped
// (a cell with 65536 or more votes) is the vote run again with atomics that
// return, which keep an exact record of the wraps.
//
// Launches per problem, on the context's stream:
//   alg1_prep_kernel    zeroes the counters (only the ball region's words
//             when the words outside it are known to be zero, else all 2 n^3
//             bytes) and the wrap record, and writes each pair's circle basis:
//             FP64 (the IEEE operation sequence of the formulas) and its FP32
//             rounding
//   alg1_vote_kernel<false>  persistent; the N J samples in FP32, 32
//             consecutive samples per warp instruction (coalesced angle-table
//             reads), four independent samples per thread, one return-less
//             atomic add each.  Samples that need FP64 go to a per-warp
//             shared-memory queue that the warp empties 32 at a time, so FP64
//             work runs in full warps
//   alg1_argmax_kernel<., false>  (count, -index) maximum over the ball
//             region's words (n a multiple of 8; otherwise every word), with
//             peaks also the count histogram, and the sum of the counts; the
//             last block writes the result (inverse projection, canonical
//             sign, rotation matrix) and sets path 1 when that sum misses the
//             samples cast (a counter wrapped, or a count fell outside the
//             region)
//   gated on path 1 (launched when N J >= 65536, returning at once
//             otherwise): alg1_rezero_kernel, alg1_vote_kernel<true> (atomics
//             with return and the wrap record), alg1_argmax_kernel<., true>
//             (the last block adds the words with wraps from the record)
//   path 2, after a problem with wraps: alg1_vote_kernel<true> and
//             alg1_argmax_kernel<., true> in place of the return-less pair
//   with peaks (Sec. 4.4): alg1_threshold_kernel, alg1_collect_kernel,
//             alg1_peaks_kernel (greedy suppression)
//   with the caller's int32 copy: alg1_expand_kernel
//
// Exactness.  A sample's cell is floor of x_k = (p_k + 1) n/2.  The FP32
// evaluation below differs from the FP64 one by at most 1.1e-6 (n/2) cells
// (error analysis at kEdgeRel); a sample whose FP32 x_k lies within
// kEdgeRel (n/2) of an integer, or whose FP32 q3 lies within kQ3Guard of 0
// (the sign choice), is evaluated again in FP64, operation for operation as
// the formulas are written, so every count equals the FP64 count.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rv_geom.cuh"
#include "rv_runtime.h"

namespace rv {

namespace {

constexpr int kA1Threads = 256;
constexpr int kA1Warps = kA1Threads / 32;
constexpr int kA1U = 4;         // samples per thread per round of the vote
constexpr int kWarpQ = 256;     // deferred FP64 samples per warp (emptied when above kWarpQ - 32 kA1U)
// FP32 error bound, with u = 2^-24 and basis norms within 1e-3 of 1 (pairs
// outside that take the FP64 path for every sample):
//   q_k  = fma(q1_k, c, q2_k s) from FP32-rounded q1, q2, c, s:  <= 6u  (3.6e-7)
//   den  = 1 + |q3| >= 1:                                        <= 8u
//   p_k  = q_k * rcp(den):                                       <= 9.6e-7
//   x_k  = fma(p_k, n/2, n/2):                                   <= 1.1e-6 (n/2)
// kEdgeRel is 7x that bound; kQ3Guard is 11x the bound on q3.
constexpr float kEdgeRel = 8e-6f;
constexpr float kQ3Guard = 4e-6f;
constexpr double kNormGuard = 1e-3;
// q1f.x (= w > 0 for a circle) doubles as the pair's flag:
constexpr float kNoCircle = -1.f;  // invalid input or a = -b
constexpr float kFp64Only = -2.f;  // basis norms outside 1 +- kNormGuard: every sample in FP64

struct A1Hdr {
    unsigned long long best_key;   // (count << 32) | (0xffffffff - index): max = argmax, ties to the smallest index
    unsigned long long cast;       // samples cast
    unsigned long long rechecked;  // samples evaluated in FP64
    int32_t invalid;               // an input vector failed validation
    uint32_t blocks_done;          // argmax blocks finished (the last one writes the result)
    int32_t peak_T;                // peak threshold (-1: not computed)
    uint32_t ncand;                // peak candidates collected
    unsigned long long decoded;    // sum of the counts as read after the return-less vote
    uint32_t path;                 // vote path (result field vote_path); nonzero: the recording vote runs
    uint32_t pad;
    rot_vote_alg1_result res;
};
static_assert(sizeof(A1Hdr) <= 256, "header slot");

// The accumulator in 16-bit counters, two cells per 32-bit word (cell c in word
// c >> 1, bits 16 (c & 1) .. +15), so that an n = 360 grid (93 MB) fits in L2.
// Counts stay exact through a record of the rare counter wraps: with E_L the
// wraps of a word's low half and E_H the wraps of the whole word, the low cell
// counts low + 65536 E_L and the high cell high + 65536 E_H - E_L (the low
// half's carries land in the high half).  Words with wraps are flagged in a
// bitmap and their counts kept in an open-addressing table.
struct Acc16 {
    uint32_t *w;     // [nw] counter words
    uint32_t *bits;  // [(nw + 31) / 32] words with wraps
    uint32_t *ekey;  // [emask + 1] word + 1 (0: empty slot)
    uint32_t *elo;   // [emask + 1] E_L
    uint32_t *ehi;   // [emask + 1] E_H
    uint32_t emask;
    int64_t nw;
};

__device__ __forceinline__ uint32_t a1_hash(uint32_t k) {
    k ^= k >> 16;
    k *= 0x7feb352du;
    k ^= k >> 15;
    k *= 0x846ca68bu;
    k ^= k >> 16;
    return k;
}

// Records wraps of word `word`.  The table holds twice the largest possible
// number of wrapping words (each wrap takes 65536 increments), so the probe ends.
__device__ __noinline__ void acc16_event(const Acc16 &A, uint32_t word, bool low_wrap, bool word_wrap) {
    atomicOr(&A.bits[word >> 5], 1u << (word & 31));
    uint32_t h = a1_hash(word) & A.emask;
    for (uint32_t probe = 0; probe <= A.emask; ++probe) {
        const uint32_t k = atomicCAS(&A.ekey[h], 0u, word + 1u);
        if (k == 0u || k == word + 1u) {
            if (low_wrap) atomicAdd(&A.elo[h], 1u);
            if (word_wrap) atomicAdd(&A.ehi[h], 1u);
            return;
        }
        h = (h + 1u) & A.emask;
    }
}

// One count into cell `cell`.  REC: an atomic with return that records the
// wraps it causes; otherwise a return-less atomic (a reduction in L2, about
// 1.6x the rate), exact as long as no counter wraps.
template <bool REC>
__device__ __forceinline__ void acc16_add(const Acc16 &A, uint32_t cell) {
    const uint32_t word = cell >> 1, inc = (cell & 1u) ? 0x10000u : 1u;
    if (!REC) {
        atomicAdd(&A.w[word], inc);
        return;
    }
    const uint32_t old = atomicAdd(&A.w[word], inc);
    const bool lw = inc == 1u && (old & 0xffffu) == 0xffffu;
    const bool ww = old > 0xffffffffu - inc;  // old + inc passes 2^32
    if (lw || ww) acc16_event(A, word, lw, ww);
}

// E_L, E_H of a flagged word (0, 0 if absent).
__device__ __forceinline__ void acc16_lookup(const Acc16 &A, uint32_t word, uint32_t &el, uint32_t &eh) {
    el = eh = 0;
    uint32_t h = a1_hash(word) & A.emask;
    for (uint32_t probe = 0; probe <= A.emask; ++probe) {
        const uint32_t k = A.ekey[h];
        if (k == word + 1u) {
            el = A.elo[h];
            eh = A.ehi[h];
            return;
        }
        if (k == 0u) return;
        h = (h + 1u) & A.emask;
    }
}

// ---- The ball region ----
// A pair whose basis norms lie within kNormGuard of 1 has samples with
// |q|^2 = c^2 |q_b1|^2 + s^2 |q_b2|^2 within 1e-3 of 1 (q_b1 . q_b2 = 0, since
// q_b2 is q_b1 times a pure quaternion), so |p| <= sqrt(1.001) < 1.0005 and its
// cell meets the ball |p| <= kRegionR.  When n is a multiple of 8 (rows of
// whole 16-byte vectors), the return-less path zeroes and scans only the
// vectors of those cells, about pi/6 of the accumulator.  A sample outside the
// region (only FP64-only pairs can stray there) is missing from the scanned
// sum of counts, so the count check sends the problem to the recording path,
// which zeroes and scans every word.
constexpr float kRegionR = 1.01f;

// The vectors [v0, v0 + len) of row `row` = iz n + iy holding its cells that
// meet the ball, with one cell of margin on each side (len = 0: none).  FP32
// with explicit rounding, so every kernel finds the same vectors.  Vector
// indices fit int32: n <= 1024 gives at most 2^27 vectors.
__device__ __forceinline__ void region_row(int side, int64_t row, int &v0, int &len) {
    v0 = 0;
    len = 0;
    if (row >= (int64_t)side * side) return;
    const int iy = (int)(row % side), iz = (int)(row / side);
    const float h = __fdiv_rn(2.f, (float)side);
    auto dist = [&](int i) {  // distance from 0 to the cell interval [-1 + i h, -1 + (i + 1) h]
        const float lo = __fmaf_rn((float)i, h, -1.f), hi = __fmaf_rn((float)(i + 1), h, -1.f);
        return lo > 0.f ? lo : (hi < 0.f ? -hi : 0.f);
    };
    const float dy = dist(iy), dz = dist(iz);
    const float r2 = __fsub_rn(__fsub_rn(kRegionR * kRegionR, __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (!(r2 >= 0.f)) return;
    const float rx = __fsqrt_rn(r2);
    const int lo = max((int)floorf(__fdiv_rn(__fsub_rn(1.f, rx), h)) - 1, 0);
    const int hi = min((int)floorf(__fdiv_rn(__fadd_rn(1.f, rx), h)) + 1, side - 1);
    const int64_t base = row * side;
    v0 = (int)((base + lo) >> 3);
    len = (int)((base + hi) >> 3) - v0 + 1;
}

// Visits the region's vectors: one warp per group of eight rows (lane r < 8
// finds row 8 g + r), f(k[4], m) on up to four vectors per lane at a time
// (k[u] valid for u < m), so that their loads can be in flight together.
template <class F>
__device__ __forceinline__ void region_scan(int side, F &&f) {
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = ((int64_t)side * side + 7) >> 3;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroups; g += nwarps) {
        int v0, len;
        region_row(side, 8 * g + (lane & 7), v0, len);
        int off = len;  // inclusive prefix over lanes 0..7, then exclusive
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, off, d);
            if ((lane & 7) >= d) off += t;
        }
        const int total = __shfl_sync(0xffffffffu, off, 7);
        off -= len;
        int roff[8], rbase[8];  // vector k = rbase[r] + j for flat index j in row r
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            roff[r] = __shfl_sync(0xffffffffu, off, r);
            rbase[r] = __shfl_sync(0xffffffffu, v0, r) - roff[r];
        }
        for (int j0 = lane; j0 < total; j0 += 128) {
            int k[4];
            int m = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + 32 * u;
                int b = rbase[0];
#pragma unroll
                for (int r = 1; r < 8; ++r)
                    if (j >= roff[r]) b = rbase[r];  // roff is nondecreasing; empty rows are skipped
                k[u] = b + j;
                m += j < total;
            }
            f(k, m);
        }
    }
}

// q_b1, q_b2 of pair (a, b) (Sec. 4.1), each value the written sequence of
// IEEE double operations.  False when w = 0 (a = -b: no circle).
__device__ __forceinline__ bool alg1_basis(double a0, double a1, double a2, double b0, double b1, double b2,
                                           double q1[4], double q2[4]) {
    const double c = dadd(dadd(dmul(a0, b0), dmul(a1, b1)), dmul(a2, b2));
    const double w = dsqrt(dmul(dadd(1.0, c), 0.5));
    if (!(w > 0.0)) return false;
    const double w2 = dmul(2.0, w);
    const double vx = ddiv(dsub(dmul(a1, b2), dmul(a2, b1)), w2);
    const double vy = ddiv(dsub(dmul(a2, b0), dmul(a0, b2)), w2);
    const double vz = ddiv(dsub(dmul(a0, b1), dmul(a1, b0)), w2);
    q1[0] = w;
    q1[1] = vx;
    q1[2] = vy;
    q1[3] = vz;
    const double bv = dadd(dadd(dmul(b0, vx), dmul(b1, vy)), dmul(b2, vz));
    q2[0] = -bv;
    q2[1] = dadd(dmul(w, b0), dsub(dmul(b1, vz), dmul(b2, vy)));
    q2[2] = dadd(dmul(w, b1), dsub(dmul(b2, vx), dmul(b0, vz)));
    q2[3] = dadd(dmul(w, b2), dsub(dmul(b0, vy), dmul(b1, vx)));
    return true;
}

// The cell of sample (c, s) = (cos, sin)(alpha_j / 2) in FP64: q = q1 c + q2 s,
// the sign with q3 <= 0, p = q_012 / (1 - q3), i_k = clamp(floor((p_k + 1) n/2)).
__device__ __forceinline__ int alg1_cell64(const double q1[4], const double q2[4], double c, double s, int n,
                                           double half) {
    double q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = dadd(dmul(q1[k], c), dmul(q2[k], s));
    if (q[3] > 0.0)
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = -q[k];
    const double den = dsub(1.0, q[3]);
    int i[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x = dmul(dadd(ddiv(q[k], den), 1.0), half);
        long long v = (long long)floor(x);
        v = v < 0 ? 0 : (v > n - 1 ? n - 1 : v);
        i[k] = (int)v;
    }
    return (i[2] * n + i[1]) * n + i[0];
}

// Zeroes the accumulator (every word, or with !full only the region's, the
// others being zero already) and its wrap record, sets the vote path (0, or 2
// for the recording vote alone) and writes every pair's basis: q1f, q2f the
// FP32 roundings of q_b1, q_b2 (q1f.x = kNoCircle / kFp64Only flags the pair),
// qd[4 i .. 4 i + 3] = q_b1, q_b2 in FP64.
__global__ void __launch_bounds__(kA1Threads) alg1_prep_kernel(const float *__restrict__ a,
                                                               const float *__restrict__ b, int64_t n,
                                                               float4 *__restrict__ q1f, float4 *__restrict__ q2f,
                                                               double2 *__restrict__ qd, Acc16 A, int J, A1Hdr *hdr,
                                                               uint32_t path, int side, bool full) {
    const int64_t T = (int64_t)gridDim.x * kA1Threads;
    const int64_t g = (int64_t)blockIdx.x * kA1Threads + threadIdx.x;
    if (g == 0) hdr->path = path;
    {
        uint4 *v = reinterpret_cast<uint4 *>(A.w);
        if (full) {
            const int64_t nvec = A.nw >> 2;
            for (int64_t k = g; k < nvec; k += T) v[k] = make_uint4(0u, 0u, 0u, 0u);
            for (int64_t r = (nvec << 2) + g; r < A.nw; r += T) A.w[r] = 0u;
        } else {  // the words outside the region are already zero
            region_scan(side, [&](const int *k, int m) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u < m) v[k[u]] = make_uint4(0u, 0u, 0u, 0u);
            });
        }
        for (int64_t r = g; r < (A.nw + 31) / 32; r += T) A.bits[r] = 0u;
        for (int64_t r = g; r <= (int64_t)A.emask; r += T) {
            A.ekey[r] = 0u;
            A.elo[r] = 0u;
            A.ehi[r] = 0u;
        }
    }
    unsigned circles = 0;
    for (int64_t i = g; i < n; i += T) {
        const float a0 = a[3 * i], a1 = a[3 * i + 1], a2 = a[3 * i + 2];
        const float b0 = b[3 * i], b1 = b[3 * i + 1], b2 = b[3 * i + 2];
        const float na = fmaf(a0, a0, fmaf(a1, a1, a2 * a2));
        const float nb = fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
        const bool ok = isfinite(a0) && isfinite(a1) && isfinite(a2) && isfinite(b0) && isfinite(b1) &&
                        isfinite(b2) && fabsf(na - 1.f) <= 1e-5f && fabsf(nb - 1.f) <= 1e-5f;
        double q1[4] = {0.0, 0.0, 0.0, 0.0}, q2[4] = {0.0, 0.0, 0.0, 0.0};
        float4 A = make_float4(kNoCircle, 0.f, 0.f, 0.f), B = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!ok) {
            atomicOr(&hdr->invalid, 1);
        } else if (alg1_basis(a0, a1, a2, b0, b1, b2, q1, q2)) {
            const double n1 = q1[0] * q1[0] + q1[1] * q1[1] + q1[2] * q1[2] + q1[3] * q1[3];
            const double n2 = q2[0] * q2[0] + q2[1] * q2[1] + q2[2] * q2[2] + q2[3] * q2[3];
            A = make_float4((float)q1[0], (float)q1[1], (float)q1[2], (float)q1[3]);  // w >= 2^-27: A.x > 0
            B = make_float4((float)q2[0], (float)q2[1], (float)q2[2], (float)q2[3]);
            if (!(fabs(n1 - 1.0) <= kNormGuard && fabs(n2 - 1.0) <= kNormGuard)) A.x = kFp64Only;
            ++circles;
        }
        // streaming (evict-first) stores: the basis is read once per warp round and must
        // not displace the accumulator from L2
        __stcs(&q1f[i], A);
        __stcs(&q2f[i], B);
        __stcs(&qd[4 * i + 0], make_double2(q1[0], q1[1]));
        __stcs(&qd[4 * i + 1], make_double2(q1[2], q1[3]));
        __stcs(&qd[4 * i + 2], make_double2(q2[0], q2[1]));
        __stcs(&qd[4 * i + 3], make_double2(q2[2], q2[3]));
    }
    const unsigned cw = __reduce_add_sync(0xffffffffu, circles);
    if ((threadIdx.x & 31) == 0 && cw) atomicAdd(&hdr->cast, (unsigned long long)cw * (unsigned long long)J);
}

// A warp's queued samples (pair << 16 | angle), 32 per pass, in FP64.
template <bool REC>
__device__ __forceinline__ void alg1_drain(const unsigned long long *wq, int qn, const double2 *__restrict__ qd,
                                           const double2 *__restrict__ t64, int side, double hd, const Acc16 &A,
                                           int lane) {
    for (int k = lane; k < qn; k += 32) {
        const unsigned long long e = wq[k];
        const int64_t i = (int64_t)(e >> 16);
        const int jj = (int)(e & 0xffffull);
        const double2 u0 = qd[4 * i], u1 = qd[4 * i + 1], u2 = qd[4 * i + 2], u3 = qd[4 * i + 3];
        const double q1[4] = {u0.x, u0.y, u1.x, u1.y}, q2[4] = {u2.x, u2.y, u3.x, u3.y};
        const double2 cs = t64[jj];
        acc16_add<REC>(A, (uint32_t)alg1_cell64(q1, q2, cs.x, cs.y, side, hd));
    }
}

// Sample s in [0, N J) is (pair s / J, angle s % J).  Warp w takes the 32 kA1U
// samples from w 32 kA1U on, lane l the samples w 32 kA1U + 32 k + l, then
// moves on by the whole grid's share (adv_p pairs, adv_j angles).
// REC = false: the return-less vote.  REC = true: the vote with the wrap
// record, which runs only when hdr->path is nonzero.
// The recording vote waits on each atomic's return: five resident blocks per
// SM hide more of that latency (measured: 1.71 -> 1.52 ms at 1e6 pairs, 50% outliers); the
// return-less vote runs best at four.
template <bool REC>
__global__ void __launch_bounds__(kA1Threads, REC ? 5 : 4) alg1_vote_kernel(const float4 *__restrict__ q1f,
                                                               const float4 *__restrict__ q2f,
                                                               const double2 *__restrict__ qd,
                                                               const float2 *__restrict__ t32,
                                                               const double2 *__restrict__ t64, int J, int side,
                                                               Acc16 acc, A1Hdr *hdr, int64_t total, int64_t adv_p,
                                                               int adv_j) {
    if (REC && !hdr->path) return;
    __shared__ unsigned long long queue[kA1Warps][kWarpQ];
    const int lane = threadIdx.x & 31;
    unsigned long long *wq = queue[threadIdx.x >> 5];
    const int64_t w = (int64_t)blockIdx.x * kA1Warps + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kA1Warps * 32 * kA1U;
    const float hf = 0.5f * (float)side;
    const double hd = 0.5 * (double)side;
    const float tol = hf * kEdgeRel;
    const int p32 = 32 / J, j32 = 32 % J;
    int64_t base = w * 32 * kA1U;
    int64_t pair = (base + lane) / J;
    int j = (int)(base + lane - pair * J);
    int qn = 0;  // the warp's queue length (the same in every lane)
    unsigned queued = 0;
    for (; base < total; base += stride) {
        int64_t pp = pair;
        int jj = j;
#pragma unroll
        for (int k = 0; k < kA1U; ++k) {
            bool slow = false;
            if (base + 32 * k + lane < total) {
                const float4 A = __ldcs(&q1f[pp]);
                if (A.x > 0.f) {
                    const float4 B = __ldcs(&q2f[pp]);
                    const float2 cs = __ldg(&t32[jj]);
                    const float q0 = fmaf(A.x, cs.x, B.x * cs.y);
                    const float q1 = fmaf(A.y, cs.x, B.y * cs.y);
                    const float q2 = fmaf(A.z, cs.x, B.z * cs.y);
                    const float q3 = fmaf(A.w, cs.x, B.w * cs.y);
                    // the sign with q3 <= 0 makes 1 - q3 = 1 + |q3| either way
                    const float r = copysignf(__frcp_rn(1.f + fabsf(q3)), -q3);
                    const float x0 = fmaf(q0 * r, hf, hf), x1 = fmaf(q1 * r, hf, hf), x2 = fmaf(q2 * r, hf, hf);
                    const float f0 = floorf(x0), f1 = floorf(x1), f2 = floorf(x2);
                    const float e0 = x0 - f0, e1 = x1 - f1, e2 = x2 - f2;  // exact
                    const float e = fminf(fminf(fminf(e0, 1.f - e0), fminf(e1, 1.f - e1)), fminf(e2, 1.f - e2));
                    if (fabsf(q3) <= kQ3Guard || e <= tol) {
                        slow = true;
                    } else {
                        const int i0 = min(max((int)f0, 0), side - 1);
                        const int i1 = min(max((int)f1, 0), side - 1);
                        const int i2 = min(max((int)f2, 0), side - 1);
                        acc16_add<REC>(acc, (uint32_t)((i2 * side + i1) * side + i0));
                    }
                } else {
                    slow = A.x == kFp64Only;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, slow);
            if (slow) wq[qn + __popc(m & ((1u << lane) - 1u))] = ((unsigned long long)pp << 16) | (unsigned)jj;
            qn += __popc(m);
            jj += j32;
            pp += p32;
            if (jj >= J) {
                jj -= J;
                ++pp;
            }
        }
        if (qn > kWarpQ - 32 * kA1U) {
            __syncwarp();
            alg1_drain<REC>(wq, qn, qd, t64, side, hd, acc, lane);
            queued += qn;
            qn = 0;
            __syncwarp();
        }
        pair += adv_p;
        j += adv_j;
        if (j >= J) {
            j -= J;
            ++pair;
        }
    }
    __syncwarp();
    alg1_drain<REC>(wq, qn, qd, t64, side, hd, acc, lane);
    queued += qn;
    if (lane == 0 && queued) atomicAdd(&hdr->rechecked, (unsigned long long)queued);
}

__device__ __forceinline__ unsigned long long a1_key(int count, uint32_t idx) {
    return ((unsigned long long)(uint32_t)count << 32) | (unsigned long long)(0xffffffffu - idx);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long x, unsigned long long y) {
    return x > y ? x : y;
}

constexpr int kArgThreads = 256;
constexpr int kHistBins = 65536;   // count histogram for the peak threshold; counts >= 65535 share the top bin
constexpr int kHistSmem = 2048;    // bins counted in shared memory per block
constexpr int kPeakCand = ROT_VOTE_ALG1_PEAK_CANDIDATES;
constexpr int kPeakThreads = 1024;

// Rotation of the centre of accumulator cell idx: the inverse projection
// (Sec. 4.3.1) of p* = -1 + (i + 1/2) 2/n, q = (2 p*, |p*|^2 - 1) / (1 + |p*|^2),
// with the sign w > 0 (w = 0: the first nonzero component > 0).
__device__ __forceinline__ void alg1_centre64(int side, uint32_t idx, double q[4]) {
    const int64_t n = side;
    const int64_t ix = idx % n, iy = (idx / n) % n, iz = idx / (n * n);
    const double h = ddiv(2.0, (double)side);
    const double p[3] = {dadd(-1.0, dmul(dadd((double)ix, 0.5), h)), dadd(-1.0, dmul(dadd((double)iy, 0.5), h)),
                         dadd(-1.0, dmul(dadd((double)iz, 0.5), h))};
    const double pp = dadd(dadd(dmul(p[0], p[0]), dmul(p[1], p[1])), dmul(p[2], p[2]));
    const double den = dadd(1.0, pp);
    q[0] = ddiv(dmul(2.0, p[0]), den);
    q[1] = ddiv(dmul(2.0, p[1]), den);
    q[2] = ddiv(dmul(2.0, p[2]), den);
    q[3] = ddiv(dsub(pp, 1.0), den);
    for (int c = 0; c < 4; ++c) {
        if (q[c] > 0.0) break;
        if (q[c] < 0.0) {
            for (int m = 0; m < 4; ++m) q[m] = -q[m];
            break;
        }
    }
}

// One cell's count into the histogram: counts 1..15 in sixteen 4-bit fields of
// a register (flushed to shared memory when a field reaches 15), 16..2047 in
// shared memory, larger counts in global memory (65535 and above in one bin).
__device__ __forceinline__ void hist_add(int c, unsigned long long &nib, unsigned *sh, unsigned *hist) {
    if (c <= 0) return;
    if (c < 16) {
        const int s = 4 * c;
        nib += 1ull << s;
        if (((nib >> s) & 15ull) == 15ull) {
            atomicAdd(&sh[c], 15u);
            nib -= 15ull << s;
        }
    } else if (c < kHistSmem) {
        atomicAdd(&sh[c], 1u);
    } else {
        atomicAdd(&hist[min(c, kHistBins - 1)], 1u);
    }
}

// The counts of one word's two cells (cells 2 wi, 2 wi + 1) from its stored
// halves and, for a word with wraps, its record.
__device__ __forceinline__ void acc16_pair(const Acc16 &A, uint32_t x, uint32_t wi, bool ev, int64_t &lo,
                                           int64_t &hi) {
    lo = x & 0xffffu;
    hi = x >> 16;
    if (ev) {
        uint32_t el, eh;
        acc16_lookup(A, wi, el, eh);
        lo += 65536ll * el;
        hi += 65536ll * eh - el;
    }
}

// Visits every word of the accumulator: f(x, word index, has wraps), with
// four 16-byte loads in flight per thread and the wrap bitmap read once per
// four words.
template <class F>
__device__ __forceinline__ void acc16_scan(const Acc16 &A, F &&f) {
    const int64_t nvec = A.nw >> 2;
    const uint4 *v = reinterpret_cast<const uint4 *>(A.w);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k + 3 * stride < nvec; k += 4 * stride) {
        uint4 c[4];
        uint32_t bm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldcs(v + k + u * stride);
            bm[u] = A.bits[(k + u * stride) >> 3] >> (((k + u * stride) & 7) * 4);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t wi = (uint32_t)((k + u * stride) << 2);
            f(c[u].x, wi, (bm[u] & 1u) != 0);
            f(c[u].y, wi + 1, (bm[u] & 2u) != 0);
            f(c[u].z, wi + 2, (bm[u] & 4u) != 0);
            f(c[u].w, wi + 3, (bm[u] & 8u) != 0);
        }
    }
    for (; k < nvec; k += stride) {
        const uint4 c = __ldcs(v + k);
        const uint32_t bm = A.bits[k >> 3] >> ((k & 7) * 4);
        const uint32_t wi = (uint32_t)(k << 2);
        f(c.x, wi, (bm & 1u) != 0);
        f(c.y, wi + 1, (bm & 2u) != 0);
        f(c.z, wi + 2, (bm & 4u) != 0);
        f(c.w, wi + 3, (bm & 8u) != 0);
    }
    for (int64_t r = (nvec << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < A.nw; r += stride)
        f(A.w[r], (uint32_t)r, ((A.bits[r >> 5] >> (r & 31)) & 1u) != 0);
}

// (count, -index) maximum over the accumulator; with HIST also the count
// histogram.  Words with wraps are left to the last block, which counts them
// from the wrap record and writes the result.  A cell past the grid (the high
// half of the last word when n^3 is odd) is never incremented: its count 0 and
// index cannot win and add nothing to the histogram.
//
// REDO = false follows the return-less vote and checks it: every cast sample
// added one count, and each counter wrap lowers the sum of the counts as read
// by 65535 (a low half passing 0xffff carries into the high half) or 65536 (a
// word passing 2^32), so that sum equals hdr->cast exactly when nothing
// wrapped.  With n a multiple of 8 it reads only the ball region's words; a
// sample outside the region is then missing from the sum as well.  Otherwise the last block sets hdr->path = 1, and the gated
// kernels that follow (alg1_rezero_kernel, alg1_vote_kernel<true>, this kernel
// with REDO = true) count again with the wrap record.  REDO = true (on path 1
// or 2) also counts the words with wraps.
template <bool HIST, bool REDO>
__global__ void __launch_bounds__(kArgThreads) alg1_argmax_kernel(Acc16 A, int side, A1Hdr *hdr,
                                                                  unsigned *__restrict__ hist) {
    if (REDO && !hdr->path) return;
    __shared__ unsigned sh[HIST ? kHistSmem : 1];
    if (HIST) {
        for (int b = threadIdx.x; b < kHistSmem; b += kArgThreads) sh[b] = 0;
        __syncthreads();
    }
    unsigned long long nib = 0;
    // cell 0 with count 0: the winner when nothing was counted (a region scan does not visit it)
    unsigned long long best = a1_key(0, 0u), sum = 0;
    auto visit = [&](uint32_t x, uint32_t wi, bool ev) {
        if (ev) return;
        const int lo = (int)(x & 0xffffu), hi = (int)(x >> 16);
        sum += (unsigned)(lo + hi);
        best = umax64(best, a1_key(lo, 2u * wi));
        best = umax64(best, a1_key(hi, 2u * wi + 1u));
        if (HIST) {
            hist_add(lo, nib, sh, hist);
            hist_add(hi, nib, sh, hist);
        }
    };
    if (!REDO && side % 8 == 0) {  // after the return-less vote: the region's words (the wrap record is empty)
        const uint4 *v = reinterpret_cast<const uint4 *>(A.w);
        region_scan(side, [&](const int *k, int m) {
            uint4 c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) c[u] = u < m ? __ldcs(v + k[u]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < m) {
                    const uint32_t wi = (uint32_t)k[u] << 2;
                    visit(c[u].x, wi, false);
                    visit(c[u].y, wi + 1, false);
                    visit(c[u].z, wi + 2, false);
                    visit(c[u].w, wi + 3, false);
                }
        });
    } else {
        acc16_scan(A, visit);
    }
    if (HIST) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int c = 1; c < 16; ++c) {
            const unsigned f = __reduce_add_sync(0xffffffffu, (unsigned)((nib >> (4 * c)) & 15ull));
            if (lane == 0 && f) atomicAdd(&sh[c], f);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < kHistSmem; b += kArgThreads)
            if (sh[b]) atomicAdd(&hist[b], sh[b]);
    }
    __shared__ unsigned long long wbest[kArgThreads / 32], wsum[kArgThreads / 32];
    __shared__ bool last;
    __shared__ int wrapped;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        wbest[threadIdx.x >> 5] = best;
        wsum[threadIdx.x >> 5] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kArgThreads / 32; ++w) {
            best = umax64(best, wbest[w]);
            sum += wsum[w];
        }
        atomicMax(&hdr->best_key, best);
        if (!REDO) atomicAdd(&hdr->decoded, sum);
        __threadfence();
        last = atomicAdd(&hdr->blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // The last block: every other block's maximum is in best_key.  The words
    // with wraps, from the record.
    __threadfence();
    const int64_t cells = (int64_t)side * side * side;
    best = 0;
    if (threadIdx.x == 0) wrapped = 0;
    __syncthreads();
    // The return-less vote leaves the wrap record empty: with REDO = false this
    // loop finds no words.
    for (uint32_t h = threadIdx.x; h <= A.emask; h += kArgThreads) {
        const uint32_t key = A.ekey[h];
        if (!key) continue;
        atomicAdd(&wrapped, 1);
        const uint32_t wi = key - 1u;
        const uint32_t x = A.w[wi];
        const int64_t lo = (int64_t)(x & 0xffffu) + 65536ll * A.elo[h];
        const int64_t hi = (int64_t)(x >> 16) + 65536ll * A.ehi[h] - A.elo[h];
        best = umax64(best, a1_key((int)lo, 2u * wi));
        if (2ll * wi + 1 < cells) best = umax64(best, a1_key((int)hi, 2u * wi + 1u));
        if (HIST) {
            if (lo >= 1) atomicAdd(&hist[min(lo, (int64_t)kHistBins - 1)], 1u);
            if (hi >= 1) atomicAdd(&hist[min(hi, (int64_t)kHistBins - 1)], 1u);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 0; w < kArgThreads / 32; ++w) best = umax64(best, wbest[w]);
    if (!REDO && atomicAdd(&hdr->decoded, 0ull) != hdr->cast) hdr->path = 1u;
    const unsigned long long key = umax64(best, atomicAdd(&hdr->best_key, 0ull));
    hdr->best_key = key;
    const uint32_t idx = 0xffffffffu - (uint32_t)(key & 0xffffffffull);
    double q[4];
    alg1_centre64(side, idx, q);
    double R[9];
    quat_to_R(q, R);
    rot_vote_alg1_result &res = hdr->res;
    for (int c = 0; c < 4; ++c) res.q[c] = q[c];
    for (int c = 0; c < 9; ++c) res.R[c] = R[c];
    res.best_count = (int32_t)(key >> 32);
    res.status = hdr->invalid ? ROT_VOTE_EINVAL : ROT_VOTE_OK;
    res.best_cell = idx;
    res.samples_cast = (int64_t)hdr->cast;
    res.rechecked = (int64_t)hdr->rechecked;
    res.ms_gpu = 0.f;
    res.npeaks = 0;
    res.peak_threshold = 0;
    res.vote_path = (int32_t)hdr->path;
    res.wrapped_words = wrapped;
}

// Path 1, before the vote with the wrap record: clears the counters, the
// histogram and the return-less vote's sums (the wrap record is still empty).
__global__ void __launch_bounds__(kArgThreads) alg1_rezero_kernel(Acc16 A, A1Hdr *hdr, unsigned *__restrict__ hist) {
    if (hdr->path != 1u) return;
    const int64_t T = (int64_t)gridDim.x * kArgThreads;
    const int64_t g = (int64_t)blockIdx.x * kArgThreads + threadIdx.x;
    uint4 *v = reinterpret_cast<uint4 *>(A.w);
    const int64_t nvec = A.nw >> 2;
    for (int64_t k = g; k < nvec; k += T) v[k] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t r = (nvec << 2) + g; r < A.nw; r += T) A.w[r] = 0u;
    if (hist)
        for (int64_t b = g; b < kHistBins; b += T) hist[b] = 0u;
    if (g == 0) {
        hdr->best_key = 0ull;
        hdr->blocks_done = 0u;
        hdr->rechecked = 0ull;
    }
}

// The accumulator as int32 counts (the caller's copy).
__global__ void __launch_bounds__(kArgThreads) alg1_expand_kernel(Acc16 A, int64_t cells, int32_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * kArgThreads;
    for (int64_t r = (int64_t)blockIdx.x * kArgThreads + threadIdx.x; r < A.nw; r += stride) {
        int64_t lo, hi;
        acc16_pair(A, A.w[r], (uint32_t)r, ((A.bits[r >> 5] >> (r & 31)) & 1u) != 0, lo, hi);
        out[2 * r] = (int32_t)lo;
        if (2 * r + 1 < cells) out[2 * r + 1] = (int32_t)hi;
    }
}

// Peak threshold T = max(min_count, the smallest t >= 1 with
// #{cells: count >= t} <= kPeakCand), from the histogram; -1 when even the top
// bin holds more than kPeakCand cells.  One block: thread t sums bins
// [64 t, 64 t + 64) (16-byte loads), a shuffle scan gives the suffix sums
// S_t = #{count >= 64 t}, and the one thread whose range holds T walks its
// 64 bins.
__global__ void __launch_bounds__(kPeakThreads) alg1_threshold_kernel(const unsigned *__restrict__ hist,
                                                                      int min_count, A1Hdr *hdr) {
    constexpr int per = kHistBins / kPeakThreads;  // 64
    __shared__ unsigned long long wsum[kPeakThreads / 32];
    __shared__ int first;  // smallest thread index t with S_t <= kPeakCand
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) first = kPeakThreads;
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hist + t * per);
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < per / 4; ++k) {
        const uint4 v = h4[k];
        s += (unsigned long long)v.x + v.y + v.z + v.w;
    }
    // inclusive suffix scan within the warp (lanes above)
    unsigned long long suf = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += v;
    }
    if (lane == 0) wsum[w] = suf;  // the warp's total
    __syncthreads();
    unsigned long long above = 0;  // totals of the warps after this one
    for (int k = w + 1; k < kPeakThreads / 32; ++k) above += wsum[k];
    const unsigned long long S = suf + above;  // #{count >= 64 t}
    if (S <= (unsigned long long)kPeakCand) atomicMin(&first, t);
    __syncthreads();
    const int f = first;
    // T lies in (64 (f - 1), 64 f]: thread f - 1 walks down its bins (f = 0: T = 1)
    const int walker = f == 0 ? -1 : f - 1;
    if (t == 0 && f == 0) {
        hdr->peak_T = max(1, max(min_count, 1));
        hdr->ncand = 0;
    }
    if (t == walker) {
        unsigned long long ge = S - s;  // #{count >= 64 (t + 1)}
        // T = 64 (t + 1) itself fits when t + 1 = f (S_f <= kPeakCand); above the last bin nothing is known
        int best = t + 1 < kPeakThreads ? (t + 1) * per : INT_MAX;
        for (int k = per - 1; k >= 0; --k) {
            const int u = t * per + k;
            ge += hist[u];
            if (u >= 1 && ge <= (unsigned long long)kPeakCand) best = u;
        }
        hdr->peak_T = best == INT_MAX ? -1 : max(best, max(min_count, 1));
        hdr->ncand = 0;
    }
}

// (count, -(iz << 20 | iy << 10 | ix)) key of cell idx: the packed coordinates
// order as the linear index (iz n + iy) n + ix does, and decode with shifts.
__device__ __forceinline__ unsigned long long a1_pkey(int count, uint32_t idx, uint32_t n) {
    const uint32_t ix = idx % n, iy = (idx / n) % n, iz = idx / (n * n);
    return a1_key(count, (iz << 20) | (iy << 10) | ix);
}

// Candidates: every cell with count >= T, as packed keys (words with wraps
// from their record).
__global__ void __launch_bounds__(kArgThreads) alg1_collect_kernel(Acc16 A, int side, A1Hdr *hdr,
                                                                   unsigned long long *cand) {
    const int T = hdr->peak_T;
    if (T < 1) return;
    const int64_t cells = (int64_t)side * side * side;
    auto put = [&](int64_t c, uint32_t i) {
        if (c >= T) {
            const unsigned pos = atomicAdd(&hdr->ncand, 1u);
            if (pos < (unsigned)kPeakCand) cand[pos] = a1_pkey((int)c, i, (uint32_t)side);
        }
    };
    acc16_scan(A, [&](uint32_t x, uint32_t wi, bool ev) {
        if (ev) return;
        put(x & 0xffffu, 2u * wi);
        put(x >> 16, 2u * wi + 1u);
    });
    const int64_t stride = (int64_t)gridDim.x * kArgThreads;
    for (int64_t h = (int64_t)blockIdx.x * kArgThreads + threadIdx.x; h <= (int64_t)A.emask; h += stride) {
        const uint32_t key = A.ekey[h];
        if (!key) continue;
        const uint32_t wi = key - 1u, x = A.w[wi];
        put((int64_t)(x & 0xffffu) + 65536ll * A.elo[h], 2u * wi);
        if (2ll * wi + 1 < cells) put((int64_t)(x >> 16) + 65536ll * A.ehi[h] - A.elo[h], 2u * wi + 1u);
    }
}

// A cell's grid coordinates and 1 + |p|^2 of its centre p = -1 + (i + 1/2) h, in FP32.
struct CellF {
    int ix, iy, iz;
    float s;
};

__device__ __forceinline__ CellF alg1_cellf(float h, uint32_t packed) {
    CellF c;
    c.ix = (int)(packed & 1023u);
    c.iy = (int)((packed >> 10) & 1023u);
    c.iz = (int)(packed >> 20);
    const float p0 = fmaf((float)c.ix + 0.5f, h, -1.f);
    const float p1 = fmaf((float)c.iy + 0.5f, h, -1.f);
    const float p2 = fmaf((float)c.iz + 0.5f, h, -1.f);
    c.s = 1.f + fmaf(p0, p0, fmaf(p1, p1, p2 * p2));
    return c;
}

// e = 1 - q.q' for the centre rotations q = P'(p), q' = P'(p') of two cells, by
// the chordal identity of the inverse projection,
//   |P'(p) - P'(p')|^2 = 4 |p - p'|^2 / ((1 + |p|^2)(1 + |p'|^2)) = 2 - 2 q.q',
// with p - p' = (i - i') h exact up to h, so e = 2 h^2 m / (s s'), m the integer
// sum of squared index differences.  Relative error (FP32): h^2 3u, each s 5u
// (p to 2u, |p|^2 and the sum 3u), product and quotient 2u: <= 16u.
__device__ __forceinline__ float alg1_one_minus_dot(const CellF &a, const CellF &b, float h2) {
    const int dx = a.ix - b.ix, dy = a.iy - b.iy, dz = a.iz - b.iz;
    const float m = (float)(dx * dx + dy * dy + dz * dz);  // <= 3 * 1023^2 < 2^24: exact
    return __fdiv_rn(2.f * h2 * m, a.s * b.s);
}

// Picks up to M peaks by greedy suppression.  Each round takes the largest
// (count, -packed index) key among the candidates not yet suppressed -- the first
// unsuppressed candidate in (count desc, index asc) order -- and suppresses
// every candidate within the angle of it (setting its key to 0).  One block,
// the keys in shared memory.
// |q.q'| >= cos(theta/2) <=> e <= 1 - cos(theta/2) or e >= 1 + cos(theta/2), e = 1 - q.q'.
// The FP32 e is within 16u e of the exact value and the FP64 dot product of the
// definition within 1e-15 of it; an e within 32u e + 1e-12 of either bound is
// decided by the FP64 definition.
__global__ void __launch_bounds__(kPeakThreads) alg1_peaks_kernel(const unsigned long long *__restrict__ cand,
                                                                  int side, int M, double cth, A1Hdr *hdr,
                                                                  rot_vote_peak *out) {
    extern __shared__ unsigned long long keys[];
    __shared__ double pq[4];
    __shared__ CellF pcell;
    __shared__ unsigned long long wmax[kPeakThreads / 32];
    __shared__ unsigned long long s_pick;
    const int t = threadIdx.x;
    const int T = hdr->peak_T;
    const int nc = T < 1 ? 0 : (int)min(hdr->ncand, (unsigned)kPeakCand);
    for (int i = t; i < nc; i += kPeakThreads) keys[i] = cand[i];
    __syncthreads();
    const float h = __fdiv_rn(2.f, (float)side), h2 = h * h;
    const float em = (float)(1.0 - cth), ep = (float)(1.0 + cth);
    int np = 0;
    while (np < M) {
        unsigned long long best = 0;
        for (int i = t; i < nc; i += kPeakThreads) best = keys[i] > best ? keys[i] : best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v > best ? v : best;
        }
        if ((t & 31) == 0) wmax[t >> 5] = best;
        __syncthreads();
        if (t == 0) {
            unsigned long long m = 0;
            for (int w = 0; w < kPeakThreads / 32; ++w) m = wmax[w] > m ? wmax[w] : m;
            s_pick = m;
            if (m) {
                const uint32_t pk3 = 0xffffffffu - (uint32_t)(m & 0xffffffffull);
                const uint32_t idx = ((pk3 >> 20) * (uint32_t)side + ((pk3 >> 10) & 1023u)) * (uint32_t)side +
                                     (pk3 & 1023u);
                double q[4];
                alg1_centre64(side, idx, q);
                for (int c = 0; c < 4; ++c) pq[c] = q[c];
                pcell = alg1_cellf(h, pk3);
                rot_vote_peak pk;
                for (int c = 0; c < 4; ++c) pk.q[c] = q[c];
                pk.cell = idx;
                pk.count = (int32_t)(m >> 32);
                pk.pad = 0;
                out[np] = pk;
            }
        }
        __syncthreads();
        const unsigned long long pick = s_pick;
        if (!pick) break;
        const CellF a = pcell;
        for (int i = t; i < nc; i += kPeakThreads) {
            const unsigned long long k = keys[i];
            if (!k) continue;
            if (k == pick) {
                keys[i] = 0;
                continue;
            }
            const uint32_t pk3 = 0xffffffffu - (uint32_t)(k & 0xffffffffull);
            const CellF cb = alg1_cellf(h, pk3);
            const float e = alg1_one_minus_dot(a, cb, h2);
            const float b = 32.f * 5.9604645e-8f * e + 1e-12f;
            bool sup = e <= em || e >= ep;
            if (fabsf(e - em) <= b || fabsf(e - ep) <= b) {  // near a bound: the FP64 definition decides
                double q[4];
                alg1_centre64(side, ((uint32_t)cb.iz * (uint32_t)side + (uint32_t)cb.iy) * (uint32_t)side + (uint32_t)cb.ix, q);
                const double d64 = dadd(dadd(dadd(dmul(q[0], pq[0]), dmul(q[1], pq[1])), dmul(q[2], pq[2])),
                                        dmul(q[3], pq[3]));
                sup = fabs(d64) >= cth;
            }
            if (sup) keys[i] = 0;
        }
        ++np;
        __syncthreads();
    }
    if (t == 0) {
        hdr->res.npeaks = np;
        hdr->res.peak_threshold = T;
    }
}

constexpr int64_t kA1MaxPairs = (int64_t)1 << 30;
constexpr int kA1MaxSamples = 65536;
constexpr int kA1MaxSide = 1024;

bool a1_on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

void Context::alg1_release() {
    if (a1_mem) {
        cudaStreamSynchronize(stream);
        cudaFree(a1_mem);
        bytes_held -= a1_cap;
    }
    a1_mem = nullptr;
    a1_cap = 0;
    a1_J = 0;
    a1_wrapped = false;
    a1_clean_side = -1;
    if (a1_hdr_h) cudaFreeHost(a1_hdr_h);
    a1_hdr_h = nullptr;
    for (auto &e : a1_ev)
        if (e) cudaEventDestroy(e);
    a1_ev[0] = a1_ev[1] = nullptr;
}

int Context::alg1(const rot_vote_alg1_problem *p, int np, rot_vote_alg1_result *out) {
    if (!a1_hdr_h && cudaMallocHost(&a1_hdr_h, 256) != cudaSuccess) {
        cudaGetLastError();
        a1_hdr_h = nullptr;
        return fail(ROT_VOTE_ENOMEM, "pinned header allocation failed");
    }
    for (auto &ev : a1_ev)
        if (!ev && cudaEventCreate(&ev) != cudaSuccess) {
            ev = nullptr;
            return fail(ROT_VOTE_ECUDA, "creating events");
        }
    for (int k = 0; k < np; ++k) {
        rot_vote_alg1_result &r = out[k];
        memset(&r, 0, sizeof r);
        const rot_vote_alg1_problem &P = p[k];
        const int J = P.samples == 0 ? 180 : P.samples;
        const int side = P.accum_side == 0 ? 360 : P.accum_side;
        const int M = P.peaks;
        if (!P.a || !P.b || P.n < 2 || P.n > kA1MaxPairs || J < 1 || J > kA1MaxSamples || side < 2 ||
            side > kA1MaxSide || P.n * (int64_t)J > (int64_t)INT_MAX || M < 0 || M > ROT_VOTE_ALG1_MAX_PEAKS ||
            (M > 0 && (!P.peak_out || !(P.nms_angle >= 0.f) || !isfinite(P.nms_angle) || P.min_count < 0))) {
            r.status = ROT_VOTE_EINVAL;
            last_error = "alg1 problem " + std::to_string(k) + ": bad argument";
            continue;
        }
        const bool dev_in = a1_on_device(P.a) && a1_on_device(P.b);
        const int64_t cells = (int64_t)side * side * side;
        // layout: header | 16-bit counter words | wrap bitmap | wrap table (3 arrays) | FP32 angle table |
        //         FP64 angle table | FP32 basis (2 x 16 B per pair) | FP64 basis (64 B per pair) | peak buffers |
        //         int32 copy of the counts (host output only) | staged inputs
        const int64_t nw = (cells + 1) / 2;
        const int64_t total = P.n * (int64_t)J;
        uint32_t esize = 1024;  // >= twice the most words that can wrap (each wrap takes 65536 increments)
        while ((int64_t)esize < 2 * (2 * (total >> 16) + 2)) esize <<= 1;
        const bool acc_dev = P.accumulator && a1_on_device(P.accumulator);
        const size_t off_w = 256;
        const size_t off_bits = align_up(off_w + sizeof(uint32_t) * (size_t)nw, 256);
        const size_t off_ek = align_up(off_bits + sizeof(uint32_t) * (size_t)((nw + 31) / 32), 256);
        const size_t off_el = align_up(off_ek + sizeof(uint32_t) * esize, 256);
        const size_t off_eh = align_up(off_el + sizeof(uint32_t) * esize, 256);
        const size_t off_t32 = align_up(off_eh + sizeof(uint32_t) * esize, 256);
        const size_t off_t64 = align_up(off_t32 + sizeof(float2) * J, 256);
        const size_t off_q1f = align_up(off_t64 + sizeof(double2) * J, 256);
        const size_t off_q2f = align_up(off_q1f + sizeof(float4) * (size_t)P.n, 256);
        const size_t off_qd = align_up(off_q2f + sizeof(float4) * (size_t)P.n, 256);
        const size_t off_hist = align_up(off_qd + 4 * sizeof(double2) * (size_t)P.n, 256);
        const size_t off_cand = align_up(off_hist + (M > 0 ? sizeof(unsigned) * kHistBins : 0), 256);
        const size_t off_pk = align_up(off_cand + (M > 0 ? sizeof(unsigned long long) * kPeakCand : 0), 256);
        const size_t off_o32 = align_up(off_pk + (M > 0 ? sizeof(rot_vote_peak) * ROT_VOTE_ALG1_MAX_PEAKS : 0), 256);
        const size_t off_in =
            align_up(off_o32 + (P.accumulator && !acc_dev ? sizeof(int32_t) * (size_t)cells : 0), 256);
        const size_t in_bytes = dev_in ? 0 : align_up(sizeof(float) * 3 * (size_t)P.n, 256);
        const size_t need = off_in + 2 * in_bytes;
        if (need > a1_cap) {
            cudaStreamSynchronize(stream);
            if (a1_mem) {
                cudaFree(a1_mem);
                bytes_held -= a1_cap;
            }
            a1_mem = nullptr;
            a1_cap = 0;
            a1_J = 0;
            if (bytes_held + need > budget) return fail(ROT_VOTE_ENOMEM, "alg1 workspace exceeds the device memory budget");
            if (cudaMalloc(&a1_mem, need) != cudaSuccess) {
                cudaGetLastError();
                a1_mem = nullptr;
                return fail(ROT_VOTE_ENOMEM, "cudaMalloc of the alg1 workspace failed");
            }
            a1_cap = need;
            a1_clean_side = -1;
            bytes_held += need;
        }
        unsigned char *base = static_cast<unsigned char *>(a1_mem);
        A1Hdr *hdr = reinterpret_cast<A1Hdr *>(base);
        float2 *t32 = reinterpret_cast<float2 *>(base + off_t32);
        double2 *t64 = reinterpret_cast<double2 *>(base + off_t64);
        Acc16 acc;
        acc.w = reinterpret_cast<uint32_t *>(base + off_w);
        acc.bits = reinterpret_cast<uint32_t *>(base + off_bits);
        acc.ekey = reinterpret_cast<uint32_t *>(base + off_ek);
        acc.elo = reinterpret_cast<uint32_t *>(base + off_el);
        acc.ehi = reinterpret_cast<uint32_t *>(base + off_eh);
        acc.emask = esize - 1;
        acc.nw = nw;
        cudaError_t e = cudaSuccess;
        if (a1_J != J || a1_toff != off_t32) {
            // (cos, sin)(alpha_j / 2), alpha_j = -pi + 2 pi j / J: the uniform samples of [-pi, pi) of Alg. 1
            std::vector<double2> h64(J);
            std::vector<float2> h32(J);
            for (int jj = 0; jj < J; ++jj) {
                const double alpha = -M_PI + (2.0 * M_PI * (double)jj) / (double)J;
                h64[jj] = make_double2(cos(alpha / 2.0), sin(alpha / 2.0));
                h32[jj] = make_float2((float)h64[jj].x, (float)h64[jj].y);
            }
            e = cudaMemcpyAsync(t64, h64.data(), sizeof(double2) * J, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(t32, h32.data(), sizeof(float2) * J, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // the host vectors die here
            if (e != cudaSuccess) return cuda_fail(e, "uploading the alg1 angle table");
            a1_J = J;
            a1_toff = off_t32;
        }
        const float *da = P.a, *db = P.b;
        if (!dev_in) {
            float *ia = reinterpret_cast<float *>(base + off_in), *ib = reinterpret_cast<float *>(base + off_in + in_bytes);
            e = cudaMemcpyAsync(ia, P.a, sizeof(float) * 3 * P.n, cudaMemcpyDefault, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ib, P.b, sizeof(float) * 3 * P.n, cudaMemcpyDefault, stream);
            if (e != cudaSuccess) return cuda_fail(e, "copying alg1 inputs");
            da = ia;
            db = ib;
        }
        // keep_trace >= 2: an event pair around each stage (kinds 5, 6, 7), for rot_vote_stage_times
        const bool profile = cfg.keep_trace >= 2;
        if (profile) {
            prof.clear();
            while (prof_ev.size() < 6) {
                cudaEvent_t ev;
                if (cudaEventCreate(&ev) != cudaSuccess) return fail(ROT_VOTE_ECUDA, "creating events");
                prof_ev.push_back(ev);
            }
        }
        auto mark = [&](int stage, bool begin, int kernels = 0) {
            if (!profile || e != cudaSuccess) return;
            if (begin) prof.push_back(rot_vote_stage{5 + stage, -1, 0.f, kernels});
            e = cudaEventRecord(prof_ev[2 * stage + (begin ? 0 : 1)], stream);
        };
        float4 *q1f = reinterpret_cast<float4 *>(base + off_q1f), *q2f = reinterpret_cast<float4 *>(base + off_q2f);
        double2 *qd = reinterpret_cast<double2 *>(base + off_qd);
        if (e == cudaSuccess) e = cudaEventRecord(a1_ev[0], stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(A1Hdr), stream);
        // Vote path.  Fewer than 65536 counts cannot wrap a counter: the
        // return-less vote alone.  After a problem with wraps the recording
        // vote runs alone (path 2).  Otherwise the return-less vote runs and
        // the gated recording vote follows, returning at once unless the
        // counters wrapped (path 1).
        const bool may_wrap = total >= 65536;
        const uint32_t path0 = may_wrap && a1_wrapped ? 2u : 0u;
        // Zeroing: the ball region's words alone when the words outside it are
        // known to be zero (the last problem had this n, took path 0 and so
        // counted nothing outside the region); otherwise every word.
        const bool full_zero = side % 8 != 0 || a1_clean_side != side;
        a1_clean_side = -1;  // until this problem is known to have taken path 0
        mark(0, true, 1);
        if (e == cudaSuccess) {
            const int64_t want = (std::max<int64_t>(P.n, nw / 4) + kA1Threads - 1) / kA1Threads;
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count * 8));
            alg1_prep_kernel<<<blocks, kA1Threads, 0, stream>>>(da, db, P.n, q1f, q2f, qd, acc, J, hdr, path0, side,
                                                                full_zero);
            e = cudaGetLastError();
        }
        mark(0, false);
        // persistent vote grid: resident blocks, or fewer when there are fewer samples
        auto vote = [&](auto kernel) {
            if (e != cudaSuccess) return;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kA1Threads, 0);
            const int64_t want = (total + kA1Threads * kA1U - 1) / (kA1Threads * kA1U);
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count * std::max(per_sm, 1)));
            const int64_t stride = (int64_t)blocks * kA1Threads * kA1U;
            if (e == cudaSuccess) {
                kernel<<<blocks, kA1Threads, 0, stream>>>(q1f, q2f, qd, t32, t64, J, side, acc, hdr, total, stride / J,
                                                          (int)(stride % J));
                e = cudaGetLastError();
            }
        };
        mark(1, true, 1);
        if (path0 == 2u)
            vote(alg1_vote_kernel<true>);
        else
            vote(alg1_vote_kernel<false>);
        mark(1, false);
        // argmax, the three gated kernels after a return-less vote that could wrap, the peak search
        mark(2, true, 1 + (path0 != 2u && may_wrap ? 3 : 0) + (M > 0 ? 3 : 0));
        unsigned *hist = reinterpret_cast<unsigned *>(base + off_hist);
        unsigned long long *cand = reinterpret_cast<unsigned long long *>(base + off_cand);
        rot_vote_peak *pk = reinterpret_cast<rot_vote_peak *>(base + off_pk);
        const int64_t want_arg = (nw / 4 + kArgThreads - 1) / kArgThreads;
        const int arg_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want_arg, (int64_t)sm_count * 8));
        auto argmax = [&](auto k_hist, auto k_plain) {
            if (e != cudaSuccess) return;
            if (M > 0)
                k_hist<<<arg_blocks, kArgThreads, 0, stream>>>(acc, side, hdr, hist);
            else
                k_plain<<<arg_blocks, kArgThreads, 0, stream>>>(acc, side, hdr, nullptr);
            e = cudaGetLastError();
        };
        if (e == cudaSuccess && M > 0) e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * kHistBins, stream);
        if (path0 == 2u) {
            argmax(alg1_argmax_kernel<true, true>, alg1_argmax_kernel<false, true>);
        } else {
            argmax(alg1_argmax_kernel<true, false>, alg1_argmax_kernel<false, false>);
            if (may_wrap) {
                if (e == cudaSuccess) {
                    alg1_rezero_kernel<<<arg_blocks, kArgThreads, 0, stream>>>(acc, hdr, M > 0 ? hist : nullptr);
                    e = cudaGetLastError();
                }
                vote(alg1_vote_kernel<true>);
                argmax(alg1_argmax_kernel<true, true>, alg1_argmax_kernel<false, true>);
            }
        }
        if (e == cudaSuccess && M > 0) {
            // peaks (Sec. 4.4): threshold, candidates, sort and greedy suppression
            alg1_threshold_kernel<<<1, kPeakThreads, 0, stream>>>(hist, P.min_count, hdr);
            e = cudaGetLastError();
            if (e == cudaSuccess) {
                alg1_collect_kernel<<<arg_blocks, kArgThreads, 0, stream>>>(acc, side, hdr, cand);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && !a1_peaks_attr) {
                e = cudaFuncSetAttribute(alg1_peaks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kPeakCand * sizeof(unsigned long long)));
                a1_peaks_attr = e == cudaSuccess;
            }
            if (e == cudaSuccess) {
                const double cth = cos((double)P.nms_angle / 2.0);
                alg1_peaks_kernel<<<1, kPeakThreads, kPeakCand * sizeof(unsigned long long), stream>>>(
                    cand, side, M, cth, hdr, pk);
                e = cudaGetLastError();
            }
        }
        mark(2, false);
        if (e == cudaSuccess) e = cudaEventRecord(a1_ev[1], stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(a1_hdr_h, hdr, sizeof(A1Hdr), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess && P.accumulator) {  // the counts as int32, into the caller's buffer
            int32_t *o32 = acc_dev ? P.accumulator : reinterpret_cast<int32_t *>(base + off_o32);
            alg1_expand_kernel<<<arg_blocks, kArgThreads, 0, stream>>>(acc, cells, o32);
            e = cudaGetLastError();
            if (e == cudaSuccess && !acc_dev)
                e = cudaMemcpyAsync(P.accumulator, o32, sizeof(int32_t) * (size_t)cells, cudaMemcpyDeviceToHost, stream);
        }
        if (e == cudaSuccess && M > 0)
            e = cudaMemcpyAsync(P.peak_out, pk, sizeof(rot_vote_peak) * M, cudaMemcpyDefault, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "running alg1");
        const A1Hdr *hh = static_cast<const A1Hdr *>(a1_hdr_h);
        r = hh->res;
        a1_wrapped = r.wrapped_words > 0;
        if (side % 8 == 0 && r.vote_path == 0) a1_clean_side = side;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a1_ev[0], a1_ev[1]);
        r.ms_gpu = ms;
        for (size_t q = 0; profile && q < prof.size(); ++q)
            cudaEventElapsedTime(&prof[q].ms, prof_ev[2 * q], prof_ev[2 * q + 1]);
    }
    return ROT_VOTE_OK;
}

}  // namespace rv

extern "C" int rot_vote_alg1(rot_vote_ctx *ctx, const rot_vote_alg1_problem *p, int n_problems,
                             rot_vote_alg1_result *out) {
    if (!ctx || !p || !out || n_problems < 1) return ROT_VOTE_EINVAL;
    rv::Context *c = reinterpret_cast<rv::Context *>(ctx);
    std::lock_guard<std::mutex> g(c->launch_mu);
    return c->alg1(p, n_problems, out);
}
