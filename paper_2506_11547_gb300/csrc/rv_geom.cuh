// rv_geom.cuh -- cell geometry and thresholds on the device, FP64.
//
// Every operation is an explicit round-to-nearest intrinsic, so nvcc never
// fuses a multiply and an add: each value is the written sequence of IEEE
// double operations, the same on every GPU and for every batch composition.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rv_internal.h"

namespace rv {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

// The delta-independent part of the threshold: cos r = 1 - 2x^2 and
// sin r = 2x sqrt(1 - x^2) of r = 2 asin(x), x = min(1, chord/2).
__device__ __forceinline__ double2 cell_trig(double chord) {
    double x = ddiv(chord, 2.0);
    if (x > 1.0) x = 1.0;
    const double cr = dsub(1.0, dmul(dmul(2.0, x), x));
    const double sr = dmul(dmul(2.0, x), dsqrt(dsub(1.0, dmul(x, x))));
    return make_double2(cr, sr);
}

// Threshold of a cell: tau = sin^2(delta + r) with r = 2 asin(x), x = min(1,
// chord/2), and 1 once delta + r >= pi/2; from the cell's (cos r, sin r) =
// (1 - 2x^2, 2x sqrt(1 - x^2)) (cell_trig), so no transcendental function is
// needed on the device; sin(delta), cos(delta) come from the host once per
// problem.
__device__ __forceinline__ double tau_cs(double sin_d, double cos_d, double2 cs) {
    const double cos_sum = dsub(dmul(cos_d, cs.x), dmul(sin_d, cs.y));
    if (cos_sum <= 0.0) return 1.0;
    const double s = dadd(dmul(sin_d, cs.x), dmul(cos_d, cs.y));
    return dmul(s, s);
}

__device__ __forceinline__ double dist0(double lo, double hi) {
    if (lo > 0.0) return lo;
    if (hi < 0.0) return -hi;
    return 0.0;
}

// Does box i of an n-grid (per axis) meet the closed unit ball?  Exact: all
// quantities are dyadic rationals with few bits.
__device__ __forceinline__ bool cell_exists(int n, int64_t ix, int64_t iy, int64_t iz) {
    if (ix < 0 || iy < 0 || iz < 0 || ix >= n || iy >= n || iz >= n) return false;
    const double h = ddiv(2.0, (double)n);
    const int64_t id[3] = {ix, iy, iz};
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double lo = dadd(-1.0, dmul((double)id[k], h));
        const double hi = dadd(lo, h);
        const double d = dist0(lo, hi);
        d2 = dadd(d2, dmul(d, d));
    }
    return d2 <= 1.0;
}

// Centre quaternion q = (sqrt(1 - |c'|^2), c') of a cell, c' the box centre
// pulled onto the ball, and a covering chord: every point p of (box cap ball),
// mapped to (sqrt(1 - |p|^2), p), lies within chord of q in R^4, because
//   |p - c'|                       <= (sqrt 3 / 2) h + max(0, |c| - 1)       = dv
//   |sqrt(1-|p|^2) - sqrt(1-|c'|^2)| <= min(sqrt(D), D / w),
//   D = max_p | |p|^2 - |c'|^2 |   (|p|^2 clamped to 1)                      = dw
// and chord = sqrt(dv^2 + dw^2).
__device__ __forceinline__ void cell_geom_ortho(int n, int64_t ix, int64_t iy, int64_t iz, double q[4],
                                                double *chord) {
    const double h = ddiv(2.0, (double)n);
    const int64_t id[3] = {ix, iy, iz};
    double c[3];
    double c2 = 0.0, maxv2 = 0.0, minv2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double lo = dadd(-1.0, dmul((double)id[k], h));
        const double hi = dadd(lo, h);
        c[k] = dadd(-1.0, dmul(dadd((double)id[k], 0.5), h));
        c2 = dadd(c2, dmul(c[k], c[k]));
        const double l2 = dmul(lo, lo), h2 = dmul(hi, hi);
        maxv2 = dadd(maxv2, l2 > h2 ? l2 : h2);
        const double d = dist0(lo, hi);
        minv2 = dadd(minv2, dmul(d, d));
    }
    const double cn = dsqrt(c2);
    double cp[3], cp2;
    if (cn > 1.0) {
        cp2 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cp[k] = ddiv(c[k], cn);
            cp2 = dadd(cp2, dmul(cp[k], cp[k]));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) cp[k] = c[k];
        cp2 = c2;
    }
    const double w2 = dsub(1.0, cp2);
    q[0] = w2 > 0.0 ? dsqrt(w2) : 0.0;
    q[1] = cp[0];
    q[2] = cp[1];
    q[3] = cp[2];
    const double dv = dadd(dmul(ddiv(dsqrt(3.0), 2.0), h), cn > 1.0 ? dsub(cn, 1.0) : 0.0);
    const double hi2 = maxv2 < 1.0 ? maxv2 : 1.0;
    const double d1 = fabs(dsub(hi2, cp2)), d2 = fabs(dsub(cp2, minv2));
    const double D = d1 > d2 ? d1 : d2;
    double dw = dsqrt(D);
    if (q[0] > 0.0) {
        const double alt = ddiv(D, q[0]);
        if (alt < dw) dw = alt;
    }
    *chord = dsqrt(dadd(dmul(dv, dv), dmul(dw, dw)));
}

// Stereographic chart (Sec. 4.3.1): the box maps onto S^3 by the inverse
// projection P'(p) = (2 p, |p|^2 - 1) / (1 + |p|^2), read as (q0, q1, q2, q3)
// (the unit ball is the half q3 <= 0).  Centre q = P'(c).  For p in the box
//   |P'(p) - P'(c)| = 2 |p - c| / sqrt((1 + |p|^2)(1 + |c|^2))
//                  <= sqrt(3) h / sqrt((1 + min_box |p|^2)(1 + |c|^2)) = chord.
__device__ __forceinline__ void cell_geom_stereo(int n, int64_t ix, int64_t iy, int64_t iz, double q[4],
                                                 double *chord) {
    const double h = ddiv(2.0, (double)n);
    const int64_t id[3] = {ix, iy, iz};
    double c[3];
    double c2 = 0.0, minv2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double lo = dadd(-1.0, dmul((double)id[k], h));
        const double hi = dadd(lo, h);
        c[k] = dadd(-1.0, dmul(dadd((double)id[k], 0.5), h));
        c2 = dadd(c2, dmul(c[k], c[k]));
        const double d = dist0(lo, hi);
        minv2 = dadd(minv2, dmul(d, d));
    }
    const double den = dadd(1.0, c2);
    q[0] = ddiv(dmul(2.0, c[0]), den);
    q[1] = ddiv(dmul(2.0, c[1]), den);
    q[2] = ddiv(dmul(2.0, c[2]), den);
    q[3] = ddiv(dsub(c2, 1.0), den);
    *chord = ddiv(dmul(dsqrt(3.0), h), dsqrt(dmul(dadd(1.0, minv2), den)));
}

// Cell geometry in the context's chart (rot_vote_config.chart): 0 orthographic
// (vector part of q, w >= 0), 1 stereographic.
__device__ __forceinline__ void cell_geom(int chart, int n, int64_t ix, int64_t iy, int64_t iz, double q[4],
                                          double *chord) {
    if (chart == 1)
        cell_geom_stereo(n, ix, iy, iz, q, chord);
    else
        cell_geom_ortho(n, ix, iy, iz, q, chord);
}

// Rotation matrix of a unit quaternion (App. A), row-major.
__device__ __forceinline__ void quat_to_R(const double q[4], double R[9]) {
    const double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    const double a = dmul(q0, q0), b = dmul(q1, q1), c = dmul(q2, q2), d = dmul(q3, q3);
    R[0] = dsub(dsub(dadd(a, b), c), d);
    R[1] = dmul(2.0, dsub(dmul(q1, q2), dmul(q0, q3)));
    R[2] = dmul(2.0, dadd(dmul(q1, q3), dmul(q0, q2)));
    R[3] = dmul(2.0, dadd(dmul(q1, q2), dmul(q0, q3)));
    R[4] = dsub(dsub(dadd(a, c), b), d);
    R[5] = dmul(2.0, dsub(dmul(q2, q3), dmul(q0, q1)));
    R[6] = dmul(2.0, dsub(dmul(q1, q3), dmul(q0, q2)));
    R[7] = dmul(2.0, dadd(dmul(q2, q3), dmul(q0, q1)));
    R[8] = dsub(dsub(dadd(a, d), b), c);
}

// Monomials m(q) with q^T S q = m(q) . s for s = [S00 S11 S22 S33 S01 S02 S03 S12 S13 S23].
__device__ __forceinline__ void monomials(const double q[4], double m[10]) {
    m[0] = dmul(q[0], q[0]);
    m[1] = dmul(q[1], q[1]);
    m[2] = dmul(q[2], q[2]);
    m[3] = dmul(q[3], q[3]);
    m[4] = dmul(2.0, dmul(q[0], q[1]));
    m[5] = dmul(2.0, dmul(q[0], q[2]));
    m[6] = dmul(2.0, dmul(q[0], q[3]));
    m[7] = dmul(2.0, dmul(q[1], q[2]));
    m[8] = dmul(2.0, dmul(q[1], q[3]));
    m[9] = dmul(2.0, dmul(q[2], q[3]));
}

// Writes one cell record (FP64 geometry, f32 monomials and rotation).
template <class CellSoAT>
__device__ __forceinline__ void write_cell(const CellSoAT &t, int64_t pos, int n, int chart, int64_t ix, int64_t iy,
                                           int64_t iz) {
    double q[4], chord;
    cell_geom(chart, n, ix, iy, iz, q, &chord);
    t.q[pos] = make_double4_32a(q[0], q[1], q[2], q[3]);
    t.chord[pos] = chord;
    t.trig[pos] = cell_trig(chord);
    t.idx[pos] = (iz * (int64_t)n + iy) * (int64_t)n + ix;
    double m[10], R[9];
    monomials(q, m);
    quat_to_R(q, R);
    t.m32[3 * pos + 0] = make_float4((float)m[0], (float)m[1], (float)m[2], (float)m[3]);
    t.m32[3 * pos + 1] = make_float4((float)m[4], (float)m[5], (float)m[6], (float)m[7]);
    t.m32[3 * pos + 2] = make_float4((float)m[8], (float)m[9], 0.f, 0.f);
    t.R32[3 * pos + 0] = make_float4((float)R[0], (float)R[1], (float)R[2], (float)R[3]);
    t.R32[3 * pos + 1] = make_float4((float)R[4], (float)R[5], (float)R[6], (float)R[7]);
    t.R32[3 * pos + 2] = make_float4((float)R[8], 0.f, 0.f, 0.f);
}

// FP32 re-check of one (cell, pair) test: v = |b - R a|^2 / 4 - c equals
// q^T S q (with S from the bilinear closed form) for any input norms, and
// carries an absolute error below 7e-7 for |R a - b| <= 2.
__device__ __forceinline__ float recheck_v(const float4 &R0, const float4 &R1, const float4 &R2, const float4 &p0,
                                           const float4 &p1) {
    // p0 = (a0 a1 a2 b0), p1 = (b1 b2 c 0); R0..R2 hold R row-major (R[0..8])
    const float ra0 = fmaf(R0.x, p0.x, fmaf(R0.y, p0.y, R0.z * p0.z));
    const float ra1 = fmaf(R0.w, p0.x, fmaf(R1.x, p0.y, R1.y * p0.z));
    const float ra2 = fmaf(R1.z, p0.x, fmaf(R1.w, p0.y, R2.x * p0.z));
    const float e0 = p0.w - ra0, e1 = p1.x - ra1, e2 = p1.y - ra2;
    const float e2s = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
    return fmaf(0.25f, e2s, -p1.z);
}

// ---------------------------------------------------------------------------
// FP64 resolution of the tests next to the threshold.
//
// A test is ambiguous when |v - tau| <= 1e-6 in FP64 (v = q_c^T S_i q_c).  The
// FP32 re-check value v32 is within 7e-7 of the exact real v, and tau32 =
// fl32(tau) within 6e-8 of tau, so once |v32 - tau32| > kBand64 = 2e-6 the
// test is not ambiguous and v32 <= tau32 is the FP64 decision.  Inside that
// band the test is evaluated in IEEE double, one rounded operation at a time
// in the order of the definition:
//   1. the products a_j b_k of the float32 inputs (exact in double);
//   2. M = L(a)^T L'(b) of App. A, entry (r, c) accumulated over k = 0..3
//      from 0.0 (the products that are structurally zero add nothing);
//   3. S = (I - M) / 2 (Lemma 1: S = I - P);
//   4. v = sum over (r, c) in row-major order of (q_r S_rc) q_c, from 0.0;
// and it votes iff v <= tau, tau = sin^2(delta + r_c) from the cell's FP64
// (cos r, sin r).  Every such value is the unique IEEE result of those
// operations, so the decision and the ambiguity flag are those of any FP64
// program that writes the definition in that order.
// ---------------------------------------------------------------------------
constexpr float kBand64 = 2e-6f;  // |v32 - tau32| <= this: decided in FP64
constexpr double kAmbig64 = 1e-6; // |v - tau| <= this (FP64): reported ambiguous

static __device__ __noinline__ double quad_fp64(double q0, double q1, double q2, double q3, const float4 &p0,
                                         const float4 &p1) {
    const double a0 = p0.x, a1 = p0.y, a2 = p0.z, b0 = p0.w, b1 = p1.x, b2 = p1.y;
    // p_jk = a_j b_k, exact (24-bit significands)
    const double p00 = dmul(a0, b0), p01 = dmul(a0, b1), p02 = dmul(a0, b2);
    const double p10 = dmul(a1, b0), p11 = dmul(a1, b1), p12 = dmul(a1, b2);
    const double p20 = dmul(a2, b0), p21 = dmul(a2, b1), p22 = dmul(a2, b2);
    // M_rc = sum_k L(a)_kr L'(b)_kc: the non-zero products in k order
    const double m00 = dadd(dadd(p00, p11), p22);
    const double m01 = dsub(p12, p21);            // k = 2: a1 b2, k = 3: -a2 b1
    const double m02 = dsub(p20, p02);            // k = 1: -a0 b2, k = 3: a2 b0
    const double m03 = dsub(p01, p10);            // k = 1: a0 b1, k = 2: -a1 b0
    const double m11 = dsub(dsub(p00, p22), p11); // k = 0, 2, 3
    const double m12 = dadd(p01, p10);
    const double m13 = dadd(p02, p20);
    const double m22 = dsub(dsub(p11, p22), p00); // k = 0, 1, 3
    const double m23 = dadd(p12, p21);
    const double m33 = dsub(dsub(p22, p11), p00); // k = 0, 1, 2
    // S = (I - M) / 2; M is symmetric entry by entry (two-term sums commute)
    const double s00 = dmul(dsub(1.0, m00), 0.5), s11 = dmul(dsub(1.0, m11), 0.5);
    const double s22 = dmul(dsub(1.0, m22), 0.5), s33 = dmul(dsub(1.0, m33), 0.5);
    const double s01 = dmul(dsub(0.0, m01), 0.5), s02 = dmul(dsub(0.0, m02), 0.5);
    const double s03 = dmul(dsub(0.0, m03), 0.5), s12 = dmul(dsub(0.0, m12), 0.5);
    const double s13 = dmul(dsub(0.0, m13), 0.5), s23 = dmul(dsub(0.0, m23), 0.5);
    const double q[4] = {q0, q1, q2, q3};
    const double S[16] = {s00, s01, s02, s03, s01, s11, s12, s13, s02, s12, s22, s23, s03, s13, s23, s33};
    double v = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) v = dadd(v, dmul(dmul(q[r], S[4 * r + c]), q[c]));
    return v;
}

// The FP64 decision of one test against an FP64 threshold: bit 0 vote, bit 1
// ambiguous.
__device__ __forceinline__ int decide_fp64(const double4_32a &q, double tau64, const float4 &p0, const float4 &p1) {
    const double v = quad_fp64(q.x, q.y, q.z, q.w, p0, p1);
    return (v <= tau64 ? 1 : 0) | (fabs(dsub(v, tau64)) <= kAmbig64 ? 2 : 0);
}

// Hands one test whose FP32 re-check lies within kBand64 of its threshold to
// the FP64 resolution pass: appends it to the level's queue, or, once the queue
// is full, flags its cell (kOvfBit in its count) so that the pass recounts the
// whole cell.  A full queue takes no further atomics, so its counter stays
// within a few thousand of cap.  The caller counts no vote for the test.
__device__ __forceinline__ void defer_or_flag(const AmbQueue &Q, int32_t *counts, int prob, int pos, int64_t gp) {
    if (!__ldcg(Q.ovf)) {
        const unsigned slot = (unsigned)atomicAdd(Q.count, 1);
        if (slot < (unsigned)Q.cap) {
            Q.q[slot] = Amb64{prob, pos, gp};
            return;
        }
    }
    atomicOr(&counts[pos], kOvfBit);
    *Q.ovf = 1;
}

// The decision of one re-checked test of a level-table cell: 1 vote, 0 no
// vote, 8 handed to the FP64 pass (no vote counted here).
__device__ __forceinline__ int decide_or_defer(float v32, float tau32, const LevelRef &L, int pos, int prob,
                                               int64_t gp, const AmbQueue &Q) {
    if (!(fabsf(v32 - tau32) <= kBand64)) return v32 <= tau32 ? 1 : 0;
    defer_or_flag(Q, L.counts, prob, pos, gp);
    return 8;
}

}  // namespace rv
