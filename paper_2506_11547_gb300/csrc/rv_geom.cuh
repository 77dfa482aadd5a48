// rv_geom.cuh -- cell geometry and thresholds on the device, FP64.
//
// Every operation is an explicit round-to-nearest intrinsic, so nvcc never
// fuses a multiply and an add: each value is the written sequence of IEEE
// double operations, the same on every GPU and for every batch composition.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rv {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

// Threshold of a cell: sin^2(delta + r) with r = 2 asin(x), x = min(1, chord/2),
// and 1 once delta + r >= pi/2.  Uses cos r = 1 - 2x^2 and
// sin r = 2x sqrt(1 - x^2), so no transcendental function is needed on the
// device; sin(delta), cos(delta) come from the host once per problem.
__device__ __forceinline__ double tau_of(double sin_d, double cos_d, double chord) {
    double x = ddiv(chord, 2.0);
    if (x > 1.0) x = 1.0;
    const double cr = dsub(1.0, dmul(dmul(2.0, x), x));
    const double sr = dmul(dmul(2.0, x), dsqrt(dsub(1.0, dmul(x, x))));
    const double cos_sum = dsub(dmul(cos_d, cr), dmul(sin_d, sr));
    if (cos_sum <= 0.0) return 1.0;
    const double s = dadd(dmul(sin_d, cr), dmul(cos_d, sr));
    return dmul(s, s);
}

// The delta-independent part of the threshold: cos r = 1 - 2x^2 and
// sin r = 2x sqrt(1 - x^2) of r = 2 asin(x), x = min(1, chord/2).
__device__ __forceinline__ double2 cell_trig(double chord) {
    double x = ddiv(chord, 2.0);
    if (x > 1.0) x = 1.0;
    const double cr = dsub(1.0, dmul(dmul(2.0, x), x));
    const double sr = dmul(dmul(2.0, x), dsqrt(dsub(1.0, dmul(x, x))));
    return make_double2(cr, sr);
}

// tau = sin^2(delta + r) from the cell's (cos r, sin r): the same operations,
// in the same order, as tau_of(), without its square root and division.
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

}  // namespace rv
