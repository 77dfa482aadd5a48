// k_tables.cu -- the coarse level table and the pair step (S_i entries,
// re-check records, tensor-core operand tiles).  The children of kept cells are
// written by the ranking kernels (k_select_fit.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

// ---------------------------------------------------------------------------
// Coarse table: cells of the n^3 grid meeting the unit ball, in increasing
// linear index.  rows[] lists the non-empty (iy, iz) rows: {first position,
// ix_lo, ix_hi, iz*n + iy}; within a row the member ix form one interval.
// ---------------------------------------------------------------------------
__global__ void build_level0_kernel(const int4 *__restrict__ rows, int nrows, int n, int chart, int64_t ncells,
                                    CellSoA out) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= ncells) return;
    int lo = 0, hi = nrows - 1;  // last row with first <= pos
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)rows[mid].x <= pos) lo = mid;
        else hi = mid - 1;
    }
    const int4 r = rows[lo];
    const int64_t ix = r.y + (pos - r.x);
    const int64_t iy = r.w % n, iz = r.w / n;
    write_cell(out, pos, n, chart, ix, iy, iz);
}

cudaError_t launch_build_level0(const int4 *rows, int nrows, int n, int chart, int64_t ncells, CellSoA out,
                                cudaStream_t s) {
    if (ncells <= 0) return cudaSuccess;
    const int bs = 256;
    const int64_t nb = (ncells + bs - 1) / bs;
    build_level0_kernel<<<(unsigned)nb, bs, 0, s>>>(rows, nrows, n, chart, ncells, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pair step.
//   s  = [S00 S11 S22 S33 S01 S02 S03 S12 S13 S23] of S = (I - M)/2, written
//        with the bilinear closed form of M = L(a)^T L'(b) (App. A):
//        S00 = (1 - a.b)/2, S0k = -(a x b)_k/2, Sjj = (1 + a.b - 2 a_j b_j)/2,
//        Sjk = -(a_j b_k + a_k b_j)/2.
//   pr = (a, b, c), c = (|a|^2 + |b|^2 - 2)/4, for the FP32 re-check.
//   tcb: the tensor-core B operand (see k_vote_tc.cu for the layout).
// Validation: finite, | |a|^2 - 1 | <= 1e-5 and | |b|^2 - 1 | <= 1e-5.
// ---------------------------------------------------------------------------
template <typename T16>
__device__ __forceinline__ T16 to16(float x);
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }

// Byte offset of element (row r, column k) of a kPairTile-row, K-column operand
// tile in the canonical no-swizzle K-major layout: 8x(16 B) core matrices
// stored contiguously; core matrices consecutive in the row direction are 128 B
// apart (SBO), consecutive in K are kPairTile*16 B apart (LBO).
__device__ __forceinline__ int tc_off(int r, int k) {
    return (k >> 3) * (kPairTile * 16) + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

template <typename T16>
__device__ __forceinline__ void write_tc_row(uint8_t *tile, int r, int K, const float s[10], bool pad) {
    // B row of a pair: K = 16: [s(10), 1, 1, lo(s_0)..lo(s_3)] (the padding carries the low
    // halves of the four diagonal entries); K = 32: [s_hi(10), s_lo(10), s_hi(10), 1, 1]
    T16 v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = to16<T16>(0.f);
    (void)pad;  // padding rows arrive with s = (4, 4, 4, 4, 0, ...): exact in 16 bits
    {
        if (K == 16) {
#pragma unroll
            for (int k = 0; k < 10; ++k) v[k] = to16<T16>(s[k]);
            v[10] = to16<T16>(1.f);
            v[11] = to16<T16>(1.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) v[12 + k] = to16<T16>(s[k] - from16(v[k]));
        } else {
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                const T16 hi = to16<T16>(s[k]);
                const T16 lo = to16<T16>(s[k] - from16(hi));
                v[k] = hi;
                v[10 + k] = lo;
                v[20 + k] = hi;
            }
            v[30] = to16<T16>(1.f);
            v[31] = to16<T16>(1.f);
        }
    }
    for (int j = 0; j < K / 8; ++j) {
        uint4 w;
        uint16_t *h = reinterpret_cast<uint16_t *>(&w);
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = *reinterpret_cast<const uint16_t *>(&v[8 * j + e]);
        *reinterpret_cast<uint4 *>(tile + tc_off(r, 8 * j)) = w;
    }
}

__global__ void pair_prep_kernel(const ProbRef *__restrict__ probs, const int2 *__restrict__ tiles, int ntiles,
                                 PairPool pool, int tc_prec, ProbStats *stats) {
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const int2 tl = tiles[t];
    const ProbRef P = probs[tl.x];
    const int64_t i = (int64_t)tl.y * kPairTile + threadIdx.x;  // local pair index
    const int64_t g = P.pool_off + i;                            // pool index
    const bool valid = i < P.n;
    // Padding pairs get S = 4 I: q^T S q = 4 |q|^2 = 4 > any threshold + band, so
    // they never vote and never need a re-check (no masking in the vote loops).
    float s[10] = {4.f, 4.f, 4.f, 4.f, 0, 0, 0, 0, 0, 0};
    float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
    if (valid) {
        const float a0 = P.a[3 * i], a1 = P.a[3 * i + 1], a2 = P.a[3 * i + 2];
        const float b0 = P.b[3 * i], b1 = P.b[3 * i + 1], b2 = P.b[3 * i + 2];
        const float na = fmaf(a0, a0, fmaf(a1, a1, a2 * a2));
        const float nb = fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
        const bool ok = isfinite(a0) && isfinite(a1) && isfinite(a2) && isfinite(b0) && isfinite(b1) &&
                        isfinite(b2) && fabsf(na - 1.f) <= 1e-5f && fabsf(nb - 1.f) <= 1e-5f;
        if (!ok) atomicOr(&stats[tl.x].invalid, 1);
        const float ab = fmaf(a0, b0, fmaf(a1, b1, a2 * b2));
        s[0] = 0.5f * (1.f - ab);
        s[1] = 0.5f * fmaf(-2.f * a0, b0, 1.f + ab);
        s[2] = 0.5f * fmaf(-2.f * a1, b1, 1.f + ab);
        s[3] = 0.5f * fmaf(-2.f * a2, b2, 1.f + ab);
        s[4] = -0.5f * fmaf(a1, b2, -a2 * b1);  // -(a x b)_x / 2
        s[5] = -0.5f * fmaf(a2, b0, -a0 * b2);  // -(a x b)_y / 2
        s[6] = -0.5f * fmaf(a0, b1, -a1 * b0);  // -(a x b)_z / 2
        s[7] = -0.5f * fmaf(a0, b1, a1 * b0);
        s[8] = -0.5f * fmaf(a0, b2, a2 * b0);
        s[9] = -0.5f * fmaf(a1, b2, a2 * b1);
        p0 = make_float4(a0, a1, a2, b0);
        p1 = make_float4(b1, b2, 0.25f * ((na + nb) - 2.f), 0.f);
    }
    // the FP32 form's operand P = b a^T (each product rounded once; 0 for padding pairs)
    float pp[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const float bv[3] = {p0.w, p1.x, p1.y}, av[3] = {p0.x, p0.y, p0.z};
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) pp[3 * j + k] = bv[j] * av[k];
    }
    pool.p32[3 * g + 0] = make_float4(pp[0], pp[1], pp[2], pp[3]);
    pool.p32[3 * g + 1] = make_float4(pp[4], pp[5], pp[6], pp[7]);
    pool.p32[3 * g + 2] = make_float4(pp[8], 0.f, 0.f, 0.f);
    pool.pr[2 * g + 0] = p0;
    pool.pr[2 * g + 1] = p1;
    if (pool.p2x) {  // pair-interleaved copy for the packed FP32 vote
        float *x = reinterpret_cast<float *>(pool.p2x + (g >> 1) * 5);
#pragma unroll
        for (int t = 0; t < 9; ++t) x[4 * (t >> 1) + 2 * (t & 1) + (g & 1)] = pp[t];
        x[18 + (g & 1)] = 0.f;
    }
    if (tc_prec != ROT_PREC_FP32 && pool.tcb) {
        const int K = pool.tc_k;
        uint8_t *tile = reinterpret_cast<uint8_t *>(pool.tcb) + (g / kPairTile) * (int64_t)(kPairTile * K * 2);
        const int r = (int)(g % kPairTile);
        if (tc_prec == ROT_PREC_FP16 || tc_prec == ROT_PREC_FP16X2)
            write_tc_row<__half>(tile, r, K, s, !valid);
        else
            write_tc_row<__nv_bfloat16>(tile, r, K, s, !valid);
    }
}

cudaError_t launch_pair_prep(const ProbRef *probs, const int2 *tiles, int ntiles, PairPool pool, int tc_prec,
                                   ProbStats *stats, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    pair_prep_kernel<<<ntiles, kPairTile, 0, s>>>(probs, tiles, ntiles, pool, tc_prec, stats);
    return cudaGetLastError();
}

}  // namespace rv
