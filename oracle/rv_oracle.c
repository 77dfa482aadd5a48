/*
 * rv_oracle.c -- plain FP64 CPU oracle for the rotation-voting hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, link or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or constant table with the
 * CUDA library.
 *
 * Everything is computed in double from double casts of the float32 inputs,
 * one (cell, pair) test at a time, in the order the method states it:
 *
 *   1. pair step   -- M_i = L(a)^T L'(b) from the two 4x4 matrices printed in
 *                     App. A; S_i = (I - M_i)/2 = I - P_i, the projector onto
 *                     the orthogonal complement of the quaternion-circle plane
 *                     (Lemma 1, Sec. 4.2; App. A shows the circle is the +1
 *                     eigenspace of M_i).
 *   2. grid        -- cells of an n^3 grid over the cube [-1,1]^3 that meet
 *                     the closed unit ball of quaternion vector parts, w >= 0
 *                     (the hemisphere of Sec. 4.3.1, charted by (x, y, z)).
 *   3. cell radius -- a covering radius r_cell on S^3.
 *   4. threshold   -- tau = sin^2(delta + r_cell), 1 once delta + r >= pi/2.
 *   5. vote        -- cell votes for pair i iff q_cell^T S_i q_cell <= tau
 *                     (the dense "cell tests every circle" dual of Alg. 1).
 *   6. rank        -- score = count - N tau (EXCESS) or count (RAW),
 *                     order (score desc, idx asc), keep the top K.
 *   7. children    -- the 8 octants of each kept cell at the next level.
 *   8. fit         -- smallest eigenvector of sum_{inliers} S_i, i.e. of
 *                     Q^T Q of Eq. (stack), Sec. 4.2; refit with the
 *                     delta-only inlier rule.
 *
 * and, separately, the paper's own Alg. 1 (Sec. 4.3.2): circle samples,
 * stereographic projection (Sec. 4.3.1), a counting grid over [-1,1]^3 and
 * its argmax (rvo_alg1*).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * arithmetic is the written sequence of IEEE double operations).
 *
 * Pins (tests/test_oracle_pins.py): steps 1-7 and the fit of a given inlier
 * set are each checked against the paper's closed forms, brute force, an
 * independent lattice count or numpy/SVD.  The refit iteration of step 8 is
 * pinned step by step: the fit with cap T returns the T-th iterate, which is
 * the smallest eigenvector of the sum of App. D's S_i over {i : q^T S_i q <=
 * sin^2(delta)} for the previous iterate q (numpy eigh), and at a repeated
 * inlier set q is a fixed point of that rule.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RVO_PI 3.14159265358979323846 /* the double nearest pi */
#define RVO_AMBIG 1e-6 /* |v - tau| <= this: the (cell, pair) decision is reported ambiguous */

enum { RVO_OK = 0, RVO_EINVAL = -1, RVO_EDEGENERATE = -6 };

/* ------------------------------------------------------------------ */
/* 1. pair step (App. A)                                              */
/* ------------------------------------------------------------------ */

/* The two 4x4 matrices of App. A with q^T L(a)^T L'(b) q = b^T R(q) a. */
static void appA_L(const double a[3], double L[16]) {
    const double a1 = a[0], a2 = a[1], a3 = a[2];
    const double m[16] = {0.0, -a1, -a2, -a3,
                          a1, 0.0, a3, -a2,
                          a2, -a3, 0.0, a1,
                          a3, a2, -a1, 0.0};
    memcpy(L, m, sizeof m);
}

static void appA_Lp(const double b[3], double L[16]) {
    const double b1 = b[0], b2 = b[1], b3 = b[2];
    const double m[16] = {0.0, -b1, -b2, -b3,
                          b1, 0.0, -b3, b2,
                          b2, b3, 0.0, -b1,
                          b3, -b2, b1, 0.0};
    memcpy(L, m, sizeof m);
}

/* M = L(a)^T L'(b) (App. A); row-major 4x4. */
void rvo_pair_M(const float a32[3], const float b32[3], double M[16]) {
    double a[3] = {a32[0], a32[1], a32[2]}, b[3] = {b32[0], b32[1], b32[2]};
    double La[16], Lb[16];
    appA_L(a, La);
    appA_Lp(b, Lb);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) acc += La[k * 4 + r] * Lb[k * 4 + c];
            M[r * 4 + c] = acc;
        }
}

/* S = (I - M)/2: for unit a, b, M has eigenvalues (1,1,-1,-1) and the +1
 * eigenspace is the circle plane, so (I - M)/2 = I - P. */
void rvo_pair_S(const float a32[3], const float b32[3], double S[16]) {
    double M[16];
    rvo_pair_M(a32, b32, M);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) S[r * 4 + c] = ((r == c ? 1.0 : 0.0) - M[r * 4 + c]) / 2.0;
}

/* q^T S q */
double rvo_quad(const double S[16], const double q[4]) {
    double v = 0.0;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) v += q[r] * S[r * 4 + c] * q[c];
    return v;
}

/* Rotation matrix of q (App. A), row-major. */
void rvo_quat_to_R(const double q[4], double R[9]) {
    const double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    R[0] = q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3;
    R[1] = 2.0 * (q1 * q2 - q0 * q3);
    R[2] = 2.0 * (q1 * q3 + q0 * q2);
    R[3] = 2.0 * (q1 * q2 + q0 * q3);
    R[4] = q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3;
    R[5] = 2.0 * (q2 * q3 - q0 * q1);
    R[6] = 2.0 * (q1 * q3 - q0 * q2);
    R[7] = 2.0 * (q2 * q3 + q0 * q1);
    R[8] = q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3;
}

/* ------------------------------------------------------------------ */
/* 2-4. grid, cell radius, threshold                                  */
/* ------------------------------------------------------------------ */

static double dist0(double lo, double hi) { /* distance from 0 to [lo, hi] */
    if (lo > 0.0) return lo;
    if (hi < 0.0) return -hi;
    return 0.0;
}

/* Cell (ix, iy, iz) of an n^3 grid over [-1,1]^3 exists iff its box meets
 * the closed unit ball. */
int rvo_cell_exists(int n, int64_t ix, int64_t iy, int64_t iz) {
    const double h = 2.0 / (double)n;
    const int64_t id[3] = {ix, iy, iz};
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (id[k] < 0 || id[k] >= n) return 0;
        const double lo = -1.0 + (double)id[k] * h, hi = lo + h;
        const double d = dist0(lo, hi);
        d2 += d * d;
    }
    return d2 <= 1.0;
}

int64_t rvo_cell_index(int n, int64_t ix, int64_t iy, int64_t iz) {
    return (iz * (int64_t)n + iy) * (int64_t)n + ix;
}

/* Cell centre quaternion and covering chord.
 *   c = box centre; c' = c, or c/|c| when |c| > 1; q = (sqrt(1 - |c'|^2), c').
 *   Every point p of (box cap ball) maps to (sqrt(1-|p|^2), p); its chord to q
 *   is at most sqrt(dv^2 + dw^2) with
 *     dv = |p - c'| <= (sqrt 3 / 2) h + max(0, |c| - 1)
 *     dw = |sqrt(1-|p|^2) - sqrt(1-|c'|^2)| <= min(sqrt(D), D / w_c),
 *     D  = max over the box of | |p|^2 - |c'|^2 |, |p|^2 clamped to [.., 1].
 *   The geodesic covering radius is r = 2 asin(chord / 2). */
void rvo_cell_geom(int n, int64_t ix, int64_t iy, int64_t iz, double q[4], double *chord) {
    const double h = 2.0 / (double)n;
    const int64_t id[3] = {ix, iy, iz};
    double c[3], c2 = 0.0, maxv2 = 0.0, minv2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double lo = -1.0 + (double)id[k] * h, hi = lo + h;
        c[k] = -1.0 + ((double)id[k] + 0.5) * h;
        c2 += c[k] * c[k];
        const double m = (lo * lo > hi * hi) ? lo * lo : hi * hi;
        maxv2 += m;
        const double d = dist0(lo, hi);
        minv2 += d * d;
    }
    const double cn = sqrt(c2);
    double cp[3], cp2;
    if (cn > 1.0) {
        cp2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            cp[k] = c[k] / cn;
            cp2 += cp[k] * cp[k];
        }
    } else {
        for (int k = 0; k < 3; ++k) cp[k] = c[k];
        cp2 = c2;
    }
    const double w2 = 1.0 - cp2;
    q[0] = w2 > 0.0 ? sqrt(w2) : 0.0;
    q[1] = cp[0];
    q[2] = cp[1];
    q[3] = cp[2];

    const double dv = (sqrt(3.0) / 2.0) * h + (cn > 1.0 ? cn - 1.0 : 0.0);
    const double hi2 = maxv2 < 1.0 ? maxv2 : 1.0;
    const double d1 = fabs(hi2 - cp2), d2 = fabs(cp2 - minv2);
    const double D = d1 > d2 ? d1 : d2;
    double dw = sqrt(D);
    if (q[0] > 0.0) {
        const double alt = D / q[0];
        if (alt < dw) dw = alt;
    }
    *chord = sqrt(dv * dv + dw * dw);
}

/* The stereographic chart of Sec. 4.3.1: the cell's box in p-space maps onto
 * S^3 by the inverse projection P'(p) = (2 p, |p|^2 - 1) / (1 + |p|^2), read
 * as (q0, q1, q2, q3); the closed unit ball is the half q3 <= 0.  Centre
 * q = P'(c).  Covering chord: for p in the box,
 *   |P'(p) - P'(c)| = 2 |p - c| / sqrt((1 + |p|^2)(1 + |c|^2))
 * (the chordal distance of the inverse stereographic projection), and
 * |p - c| <= (sqrt 3 / 2) h, |p|^2 >= min over the box, so
 *   chord = sqrt(3) h / sqrt((1 + min |p|^2)(1 + |c|^2)). */
void rvo_cell_geom_stereo(int n, int64_t ix, int64_t iy, int64_t iz, double q[4], double *chord) {
    const double h = 2.0 / (double)n;
    const int64_t id[3] = {ix, iy, iz};
    double c[3], c2 = 0.0, minv2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double lo = -1.0 + (double)id[k] * h, hi = lo + h;
        c[k] = -1.0 + ((double)id[k] + 0.5) * h;
        c2 += c[k] * c[k];
        const double d = dist0(lo, hi);
        minv2 += d * d;
    }
    const double den = 1.0 + c2;
    q[0] = 2.0 * c[0] / den;
    q[1] = 2.0 * c[1] / den;
    q[2] = 2.0 * c[2] / den;
    q[3] = (c2 - 1.0) / den;
    *chord = sqrt(3.0) * h / sqrt((1.0 + minv2) * den);
}

/* Cell geometry in the chosen chart: 0 orthographic (the vector part of q,
 * w >= 0), 1 stereographic (Sec. 4.3.1). */
void rvo_cell_geom_chart(int chart, int n, int64_t ix, int64_t iy, int64_t iz, double q[4], double *chord) {
    if (chart == 1)
        rvo_cell_geom_stereo(n, ix, iy, iz, q, chord);
    else
        rvo_cell_geom(n, ix, iy, iz, q, chord);
}

/* tau = sin^2(delta + r), r = 2 asin(x), x = min(1, chord / 2); tau = 1 once
 * delta + r >= pi/2.  Written with cos r = 1 - 2x^2, sin r = 2x sqrt(1-x^2)
 * (an identity), so that it needs only sqrt. */
double rvo_tau(double sin_d, double cos_d, double chord) {
    double x = chord / 2.0;
    if (x > 1.0) x = 1.0;
    const double cr = 1.0 - 2.0 * x * x;
    const double sr = 2.0 * x * sqrt(1.0 - x * x);
    const double cos_sum = cos_d * cr - sin_d * sr; /* cos(delta + r) */
    if (cos_sum <= 0.0) return 1.0;
    const double s = sin_d * cr + cos_d * sr; /* sin(delta + r) */
    return s * s;
}

/* Level-0 cells in increasing linear index; returns the count. */
int64_t rvo_level_cells(int n, int64_t *idx_out) {
    int64_t cnt = 0;
    for (int64_t iz = 0; iz < n; ++iz)
        for (int64_t iy = 0; iy < n; ++iy)
            for (int64_t ix = 0; ix < n; ++ix)
                if (rvo_cell_exists(n, ix, iy, iz)) {
                    if (idx_out) idx_out[cnt] = rvo_cell_index(n, ix, iy, iz);
                    ++cnt;
                }
    return cnt;
}

static void unpack_idx(int n, int64_t idx, int64_t *ix, int64_t *iy, int64_t *iz) {
    *ix = idx % n;
    *iy = (idx / n) % n;
    *iz = idx / ((int64_t)n * n);
}

/* ------------------------------------------------------------------ */
/* 5. vote                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    const double *S;  /* [n_pairs][16] */
    int64_t n_pairs;
    int n_side;
    int chart;
    const int64_t *cells;
    int64_t c0, c1;
    double sin_d, cos_d;
    int32_t *count, *amb;
    double *tau_out;
} vote_job;

static void *vote_worker(void *arg) {
    vote_job *j = (vote_job *)arg;
    for (int64_t c = j->c0; c < j->c1; ++c) {
        int64_t ix, iy, iz;
        unpack_idx(j->n_side, j->cells[c], &ix, &iy, &iz);
        double q[4], chord;
        rvo_cell_geom_chart(j->chart, j->n_side, ix, iy, iz, q, &chord);
        const double tau = rvo_tau(j->sin_d, j->cos_d, chord);
        int32_t cnt = 0, amb = 0;
        for (int64_t i = 0; i < j->n_pairs; ++i) {
            const double v = rvo_quad(j->S + 16 * i, q);
            if (v <= tau) ++cnt;
            if (fabs(v - tau) <= RVO_AMBIG) ++amb;
        }
        j->count[c] = cnt;
        if (j->amb) j->amb[c] = amb;
        if (j->tau_out) j->tau_out[c] = tau;
    }
    return NULL;
}

static void vote_cells_S(const double *S, int64_t n, int n_side, int chart, const int64_t *cells,
                         int64_t ncells, double sin_d, double cos_d, int32_t *count, int32_t *amb,
                         double *tau_out, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > ncells) nthreads = ncells > 0 ? (int)ncells : 1;
    vote_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (vote_job){S, n, n_side, chart, cells, ncells * t / nthreads, ncells * (t + 1) / nthreads,
                             sin_d, cos_d, count, amb, tau_out};
    }
    if (nthreads == 1) {
        vote_worker(&jobs[0]);
        return;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, vote_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

static double *all_pair_S(const float *a, const float *b, int64_t n) {
    double *S = (double *)malloc(sizeof(double) * 16 * (size_t)(n > 0 ? n : 1));
    if (!S) return NULL;
    for (int64_t i = 0; i < n; ++i) rvo_pair_S(a + 3 * i, b + 3 * i, S + 16 * i);
    return S;
}

/* Counts (and ambiguous counts, and tau) for an arbitrary list of cells of
 * the n_side grid in the given chart. */
int rvo_vote_cells(const float *a, const float *b, int64_t n, double delta, int n_side, int chart,
                   const int64_t *cells, int64_t ncells, int32_t *count, int32_t *amb, double *tau_out,
                   int nthreads) {
    double *S = all_pair_S(a, b, n);
    if (!S) return RVO_EINVAL;
    vote_cells_S(S, n, n_side, chart, cells, ncells, sin(delta), cos(delta), count, amb, tau_out, nthreads);
    free(S);
    return RVO_OK;
}

/* ------------------------------------------------------------------ */
/* 6. rank                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    double score;
    int64_t idx;
    int64_t pos;
} rank_item;

static int rank_cmp(const void *x, const void *y) {
    const rank_item *a = (const rank_item *)x, *b = (const rank_item *)y;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

/* Order cells by (score desc, idx asc); score = count - n*tau (EXCESS,
 * rank_mode 0) or count (RAW, rank_mode 1).  Writes the positions (into the
 * input arrays) of the first k in rank order; returns how many. */
int64_t rvo_rank(const int32_t *count, const double *tau, const int64_t *idx, int64_t ncells, int64_t n_pairs,
                 int rank_mode, int64_t k, int64_t *pos_out, double *score_out) {
    rank_item *it = (rank_item *)malloc(sizeof(rank_item) * (size_t)(ncells > 0 ? ncells : 1));
    if (!it) return -1;
    for (int64_t c = 0; c < ncells; ++c) {
        const double score = rank_mode == 1 ? (double)count[c] : (double)count[c] - (double)n_pairs * tau[c];
        it[c] = (rank_item){score, idx[c], c};
    }
    qsort(it, (size_t)ncells, sizeof(rank_item), rank_cmp);
    const int64_t kk = k < ncells ? k : ncells;
    for (int64_t r = 0; r < kk; ++r) {
        pos_out[r] = it[r].pos;
        if (score_out) score_out[r] = it[r].score;
    }
    free(it);
    return kk;
}

/* ------------------------------------------------------------------ */
/* 8. fit                                                             */
/* ------------------------------------------------------------------ */

/* Cyclic Jacobi eigen-decomposition of a symmetric 4x4 (row-major).
 * Eigenvalues ascending in evals; eigenvector k is column k of V. */
void rvo_jacobi4(const double A_in[16], double evals[4], double V_out[16]) {
    double A[4][4], V[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            A[r][c] = A_in[r * 4 + c];
            V[r][c] = r == c ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) off += A[p][q] * A[p][q];
        if (off < 1e-300) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation that zeroes A[p][q]: t = tan(phi), theta = cot(2 phi) */
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 4; ++k) { /* A <- A J */
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) { /* A <- J^T A */
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) { /* V <- V J */
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int order[4] = {0, 1, 2, 3};
    for (int i = 1; i < 4; ++i) /* insertion sort by eigenvalue, ascending */
        for (int j = i; j > 0 && A[order[j]][order[j]] < A[order[j - 1]][order[j - 1]]; --j) {
            const int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (int k = 0; k < 4; ++k) {
        evals[k] = A[order[k]][order[k]];
        for (int r = 0; r < 4; ++r) V_out[r * 4 + k] = V[r][order[k]];
    }
}

/* Sign convention: w > 0; if w == 0, the first nonzero component > 0. */
void rvo_canonical(double q[4]) {
    for (int k = 0; k < 4; ++k) {
        if (q[k] > 0.0) return;
        if (q[k] < 0.0) {
            for (int j = 0; j < 4; ++j) q[j] = -q[j];
            return;
        }
    }
}

/* Smallest eigenvector of sum_{i in set} S_i (Eq. stack: the least-squares
 * solution of Q q = 0 is the eigenvector of Q^T Q with the smallest
 * eigenvalue; Q^T Q = sum_i (q_b3 q_b3^T + q_b4 q_b4^T) = sum_i S_i).
 * Returns 1 if the two smallest eigenvalues are within 1e-12 * trace. */
static int fit_set(const double *S, const unsigned char *in, int64_t n, double q[4]) {
    double A[16] = {0};
    for (int64_t i = 0; i < n; ++i)
        if (in[i])
            for (int k = 0; k < 16; ++k) A[k] += S[16 * i + k];
    double ev[4], V[16];
    rvo_jacobi4(A, ev, V);
    for (int r = 0; r < 4; ++r) q[r] = V[r * 4 + 0];
    const double tr = A[0] + A[5] + A[10] + A[15];
    return (ev[1] - ev[0]) <= 1e-12 * tr;
}

/* ------------------------------------------------------------------ */
/* full solve                                                         */
/* ------------------------------------------------------------------ */

typedef struct {
    double q[4];
    double R[9];
    int32_t best_count;
    int32_t inliers;
    int64_t best_cell; /* linear index at the last level */
    int64_t tests;     /* cells x pairs over all levels */
    int64_t ambiguous; /* (cell, pair) tests with |v - tau| <= 1e-6 */
    int32_t status;
    int32_t refits;    /* refit iterations performed */
} rvo_result;

/* Optional per-level trace: for level l, up to cap cells (idx, count, amb,
 * tau) in table order and the top-k positions in rank order. */
typedef struct {
    int64_t cap;
    int64_t *ncells;   /* [levels+1] */
    int64_t *idx;      /* [levels+1][cap] */
    int32_t *count;    /* [levels+1][cap] */
    int32_t *amb;      /* [levels+1][cap] */
    double *tau;       /* [levels+1][cap] */
    int64_t *topk_idx; /* [levels+1][top_k] */
    double *topk_score;
    int64_t *nkept;    /* [levels+1] */
} rvo_trace;

static int fit_from_cell(const double *S, int64_t n, double sd, double cd, int n_side, int chart, int64_t idx,
                         int refit_iters, rvo_result *res);

int rvo_solve(const float *a, const float *b, int64_t n, double delta, int grid_n, int levels, int top_k,
              int rank_mode, int refit_iters, int chart, int nthreads, rvo_result *res, rvo_trace *tr) {
    memset(res, 0, sizeof *res);
    if (n < 2 || grid_n < 1 || levels < 0 || top_k < 1 || !(delta > 0.0)) {
        res->status = RVO_EINVAL;
        return RVO_EINVAL;
    }
    double *S = all_pair_S(a, b, n);
    if (!S) return RVO_EINVAL;
    const double sd = sin(delta), cd = cos(delta);

    int64_t nc = rvo_level_cells(grid_n, NULL);
    int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    rvo_level_cells(grid_n, cells);
    int64_t win_idx = -1, win_n = grid_n;
    int32_t win_count = 0;
    double win_tau = 0.0;

    for (int lev = 0; lev <= levels; ++lev) {
        const int n_side = grid_n << lev;
        int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
        int32_t *amb = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
        double *tau = (double *)malloc(sizeof(double) * (size_t)nc);
        vote_cells_S(S, n, n_side, chart, cells, nc, sd, cd, count, amb, tau, nthreads);
        res->tests += nc * n;
        for (int64_t c = 0; c < nc; ++c) res->ambiguous += amb[c];

        int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)top_k);
        double *score = (double *)malloc(sizeof(double) * (size_t)top_k);
        const int64_t kept = rvo_rank(count, tau, cells, nc, n, rank_mode, top_k, pos, score);

        if (tr) {
            tr->ncells[lev] = nc;
            tr->nkept[lev] = kept;
            const int64_t m = nc < tr->cap ? nc : tr->cap;
            for (int64_t c = 0; c < m; ++c) {
                tr->idx[lev * tr->cap + c] = cells[c];
                tr->count[lev * tr->cap + c] = count[c];
                tr->amb[lev * tr->cap + c] = amb[c];
                tr->tau[lev * tr->cap + c] = tau[c];
            }
            for (int64_t r = 0; r < kept; ++r) {
                tr->topk_idx[lev * top_k + r] = cells[pos[r]];
                tr->topk_score[lev * top_k + r] = score[r];
            }
        }
        win_idx = cells[pos[0]];
        win_count = count[pos[0]];
        win_tau = tau[pos[0]];
        win_n = n_side;

        if (lev < levels) { /* 7. children of the kept cells */
            int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(8 * kept));
            int64_t nn = 0;
            for (int64_t r = 0; r < kept; ++r) {
                int64_t ix, iy, iz;
                unpack_idx(n_side, cells[pos[r]], &ix, &iy, &iz);
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            const int64_t cx = 2 * ix + dx, cy = 2 * iy + dy, cz = 2 * iz + dz;
                            if (rvo_cell_exists(2 * n_side, cx, cy, cz))
                                next[nn++] = rvo_cell_index(2 * n_side, cx, cy, cz);
                        }
            }
            free(cells);
            cells = next;
            nc = nn;
        }
        free(count);
        free(amb);
        free(tau);
        free(pos);
        free(score);
    }
    free(cells);
    (void)win_tau;
    res->best_cell = win_idx;
    res->best_count = win_count;
    const int status = fit_from_cell(S, n, sd, cd, (int)win_n, chart, win_idx, refit_iters, res);
    free(S);
    return status;
}

/* 8. fit, from the winning cell (index idx of the n_side grid):
 * I_0 = voters of the cell, q_0 = smallest eigenvector of sum_{I_0} S_i; then
 * I_t = {i : q_{t-1}^T S_i q_{t-1} <= sin^2(delta)}, stopping when |I_t| < 2 or
 * I_t = I_{t-1}; the cell centre is returned if the first fit is degenerate. */
static int fit_from_cell(const double *S, int64_t n, double sd, double cd, int n_side, int chart, int64_t idx,
                         int refit_iters, rvo_result *res) {
    int64_t ix, iy, iz;
    unpack_idx(n_side, idx, &ix, &iy, &iz);
    double qc[4], chord;
    rvo_cell_geom_chart(chart, n_side, ix, iy, iz, qc, &chord);
    const double win_tau = rvo_tau(sd, cd, chord);

    unsigned char *in0 = (unsigned char *)calloc((size_t)n, 1);
    unsigned char *in1 = (unsigned char *)calloc((size_t)n, 1);
    int64_t n_in = 0;
    for (int64_t i = 0; i < n; ++i)
        if (rvo_quad(S + 16 * i, qc) <= win_tau) {
            in0[i] = 1;
            ++n_in;
        }
    double q[4] = {qc[0], qc[1], qc[2], qc[3]};
    int status = RVO_OK;
    if (n_in < 2 || fit_set(S, in0, n, q)) {
        memcpy(q, qc, sizeof q);
        status = RVO_EDEGENERATE;
    } else {
        const double thr = sd * sd; /* sin^2(delta) */
        for (int t = 1; t <= refit_iters; ++t) {
            int64_t m = 0, changed = 0;
            for (int64_t i = 0; i < n; ++i) {
                in1[i] = rvo_quad(S + 16 * i, q) <= thr;
                m += in1[i];
                changed += in1[i] != in0[i];
            }
            if (m < 2 || changed == 0) break;
            double qn[4];
            if (fit_set(S, in1, n, qn)) break;
            memcpy(q, qn, sizeof q);
            unsigned char *tmp = in0;
            in0 = in1;
            in1 = tmp;
            n_in = m;
            res->refits = t;
        }
    }
    rvo_canonical(q);
    memcpy(res->q, q, sizeof q);
    rvo_quat_to_R(q, res->R);
    res->inliers = (int32_t)n_in;
    res->status = status;
    free(in0);
    free(in1);
    return status;
}

/* The fit alone, from a given winning cell. */
int rvo_fit_cell(const float *a, const float *b, int64_t n, double delta, int n_side, int chart, int64_t idx,
                 int refit_iters, rvo_result *res) {
    memset(res, 0, sizeof *res);
    double *S = all_pair_S(a, b, n);
    if (!S) return RVO_EINVAL;
    res->best_cell = idx;
    const int status = fit_from_cell(S, n, sin(delta), cos(delta), n_side, chart, idx, refit_iters, res);
    free(S);
    return status;
}

/* ------------------------------------------------------------------ */
/* Alg. 1 (Sec. 4.3.2): the paper's own voting -- every quaternion    */
/* circle sampled at J angles, each sample stereographically          */
/* projected (Sec. 4.3.1) and counted in a grid over [-1,1]^3.        */
/* ------------------------------------------------------------------ */

/* Orthonormal basis (q_b1, q_b2) of the circle of pair (a, b), Sec. 4.1:
 * q_b1 is the quaternion of the minimal rotation R_a^b, written with the
 * half-angle identities w = cos(theta/2) = sqrt((1 + a.b)/2) and
 * sin(theta/2) c = (a x b) / (2 w) (no trigonometry, no normalisation of
 * a x b); q_b2 = [-b.v, w b + b x v] with v the vector part of q_b1.
 * Returns 0 when a = -b exactly (w = 0: no circle is defined; such a pair
 * casts no vote).  Every operation is a separate IEEE double operation. */
int rvo_alg1_basis(const float a32[3], const float b32[3], double q1[4], double q2[4]) {
    const double a0 = a32[0], a1 = a32[1], a2 = a32[2], b0 = b32[0], b1 = b32[1], b2 = b32[2];
    const double c = (a0 * b0 + a1 * b1) + a2 * b2;
    const double w = sqrt((1.0 + c) * 0.5);
    if (!(w > 0.0)) return 0;
    const double w2 = 2.0 * w;
    const double vx = (a1 * b2 - a2 * b1) / w2, vy = (a2 * b0 - a0 * b2) / w2, vz = (a0 * b1 - a1 * b0) / w2;
    q1[0] = w;
    q1[1] = vx;
    q1[2] = vy;
    q1[3] = vz;
    const double bv = (b0 * vx + b1 * vy) + b2 * vz;
    q2[0] = -bv;
    q2[1] = w * b0 + (b1 * vz - b2 * vy);
    q2[2] = w * b1 + (b2 * vx - b0 * vz);
    q2[3] = w * b2 + (b0 * vy - b1 * vx);
    return 1;
}

/* Sample q(alpha_j) = q_b1 cos(alpha_j/2) + q_b2 sin(alpha_j/2), taken with
 * the sign that puts it in the q3 <= 0 half (q and -q are one rotation; that
 * half projects into the unit ball), projected p = (q0, q1, q2) / (1 - q3)
 * (Sec. 4.3.1), and located in the n^3 grid over [-1,1]^3:
 * i_k = floor((p_k + 1) n/2) clamped to [0, n-1].  Returns the linear index
 * (iz n + iy) n + ix. */
int64_t rvo_alg1_cell(const double q1[4], const double q2[4], double cj, double sj, int n) {
    double q[4];
    for (int k = 0; k < 4; ++k) q[k] = q1[k] * cj + q2[k] * sj;
    if (q[3] > 0.0)
        for (int k = 0; k < 4; ++k) q[k] = -q[k];
    const double den = 1.0 - q[3];
    const double half = 0.5 * (double)n;
    int64_t i[3];
    for (int k = 0; k < 3; ++k) {
        const double x = (q[k] / den + 1.0) * half;
        int64_t v = (int64_t)floor(x);
        if (v < 0) v = 0;
        if (v > n - 1) v = n - 1;
        i[k] = v;
    }
    return (i[2] * n + i[1]) * n + i[0];
}

/* The whole of Alg. 1 for one problem: acc[n^3] (zeroed here) gets one count
 * per sample; the winner is the largest count, ties to the smallest index; q
 * is the inverse projection of the winner's centre
 * p* = -1 + (i + 1/2) 2/n: q = [2 p*, |p*|^2 - 1] / (1 + |p*|^2), canonical
 * sign.  cs holds (cos(alpha_j/2), sin(alpha_j/2)) for j < J.  Returns the
 * number of samples cast. */
void rvo_alg1_centre(int n, int64_t idx, double q[4]);

int64_t rvo_alg1(const float *a, const float *b, int64_t n_pairs, const double *cs, int J, int n, int32_t *acc,
                 int64_t *best_idx, int32_t *best_count, double q[4]) {
    const int64_t cells = (int64_t)n * n * n;
    memset(acc, 0, sizeof(int32_t) * (size_t)cells);
    int64_t cast = 0;
    for (int64_t i = 0; i < n_pairs; ++i) {
        double q1[4], q2[4];
        if (!rvo_alg1_basis(a + 3 * i, b + 3 * i, q1, q2)) continue;
        for (int j = 0; j < J; ++j) {
            ++acc[rvo_alg1_cell(q1, q2, cs[2 * j], cs[2 * j + 1], n)];
            ++cast;
        }
    }
    int64_t bi = 0;
    for (int64_t c = 1; c < cells; ++c)
        if (acc[c] > acc[bi]) bi = c;
    *best_idx = bi;
    *best_count = acc[bi];
    rvo_alg1_centre(n, bi, q);
    return cast;
}

/* Rotation of the centre of accumulator cell idx (n^3 grid): the inverse
 * projection (Sec. 4.3.1) of p* = -1 + (i + 1/2) 2/n,
 * q = [2 p*, |p*|^2 - 1] / (1 + |p*|^2), canonical sign. */
void rvo_alg1_centre(int n, int64_t idx, double q[4]) {
    const int64_t ix = idx % n, iy = (idx / n) % n, iz = idx / ((int64_t)n * n);
    const double h = 2.0 / (double)n;
    const double p[3] = {-1.0 + ((double)ix + 0.5) * h, -1.0 + ((double)iy + 0.5) * h, -1.0 + ((double)iz + 0.5) * h};
    const double pp = (p[0] * p[0] + p[1] * p[1]) + p[2] * p[2];
    const double den = 1.0 + pp;
    q[0] = (2.0 * p[0]) / den;
    q[1] = (2.0 * p[1]) / den;
    q[2] = (2.0 * p[2]) / den;
    q[3] = (pp - 1.0) / den;
    rvo_canonical(q);
}

typedef struct {
    int32_t count;
    int64_t idx;
} peak_cand;

static int peak_cmp(const void *x, const void *y) { /* count desc, index asc */
    const peak_cand *a = (const peak_cand *)x, *b = (const peak_cand *)y;
    if (a->count != b->count) return a->count > b->count ? -1 : 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Multiple rotations (Sec. 4.4): up to M peaks of the accumulator, by greedy
 * non-maximum suppression.  The candidates are the cells with count >= T,
 * T = max(min_count, the smallest t >= 1 with #{cells: count >= t} <= kmax),
 * taken in (count desc, index asc) order.  A candidate becomes a peak unless
 * its centre rotation lies within theta of an earlier peak's:
 * |q . q_peak| >= cos(theta / 2), the dot product summed as
 * ((q0 q0' + q1 q1') + q2 q2') + q3 q3'.  Writes the peaks' index, count and
 * centre rotation; returns how many were found and sets *T_out. */
int rvo_alg1_peaks(const int32_t *acc, int n, int M, int min_count, int64_t kmax, double theta, int64_t *pidx,
                   int32_t *pcount, double *pq, int32_t *T_out) {
    const int64_t cells = (int64_t)n * n * n;
    int32_t maxc = 0;
    for (int64_t c = 0; c < cells; ++c)
        if (acc[c] > maxc) maxc = acc[c];
    /* ge[t] = number of cells with count >= t */
    int64_t *ge = (int64_t *)calloc((size_t)maxc + 2, sizeof(int64_t));
    for (int64_t c = 0; c < cells; ++c) ge[acc[c]] += 1;
    for (int64_t t = (int64_t)maxc - 1; t >= 0; --t) ge[t] += ge[t + 1];
    int64_t T = 1;
    while (T <= maxc && ge[T] > kmax) ++T;
    if (T < min_count) T = min_count;
    *T_out = (int32_t)T;
    const int64_t ncand = T <= maxc ? ge[T] : 0;
    free(ge);
    peak_cand *cand = (peak_cand *)malloc(sizeof(peak_cand) * (size_t)(ncand > 0 ? ncand : 1));
    int64_t k = 0;
    for (int64_t c = 0; c < cells; ++c)
        if (acc[c] >= T) cand[k++] = (peak_cand){acc[c], c};
    qsort(cand, (size_t)ncand, sizeof(peak_cand), peak_cmp);
    const double cth = cos(theta / 2.0);
    int np = 0;
    for (int64_t i = 0; i < ncand && np < M; ++i) {
        double q[4];
        rvo_alg1_centre(n, cand[i].idx, q);
        int near = 0;
        for (int m = 0; m < np && !near; ++m) {
            const double *o = pq + 4 * m;
            const double d = ((q[0] * o[0] + q[1] * o[1]) + q[2] * o[2]) + q[3] * o[3];
            near = fabs(d) >= cth;
        }
        if (near) continue;
        pidx[np] = cand[i].idx;
        pcount[np] = cand[i].count;
        for (int j = 0; j < 4; ++j) pq[4 * np + j] = q[j];
        ++np;
    }
    free(cand);
    return np;
}

/* (cos(alpha_j/2), sin(alpha_j/2)) for alpha_j = -pi + 2 pi j / J, j < J: the
 * uniform discretisation of [-pi, pi) of Alg. 1. */
void rvo_alg1_table(int J, double *cs) {
    for (int j = 0; j < J; ++j) {
        const double alpha = -RVO_PI + (2.0 * RVO_PI * (double)j) / (double)J;
        cs[2 * j] = cos(alpha / 2.0);
        cs[2 * j + 1] = sin(alpha / 2.0);
    }
}

/* ------------------------------------------------------------------ */
/* Rigid pose (Sec. 4.5): pairwise differences with the length check,  */
/* rotation from the kept pairs, translation by voting.                */
/* ------------------------------------------------------------------ */

/* For every i < j (in lexicographic order): m = x_i - x_j, n = y_i - y_j
 * (from the float32 points, in double), |m| = sqrt(m.m), |n| = sqrt(n.n).
 * The pair is kept iff |m| > lmin, |n| > lmin and | |m| - |n| | <= mu (the
 * rotation-invariant length check of Sec. 4.5.1), and then becomes the unit
 * correspondence (m / |m|, n / |n|), rounded to float32, written to a_out,
 * b_out when they are not NULL (up to cap pairs).  Returns the number kept. */
int64_t rvo_pose_pairs(const float *x, const float *y, int64_t n, double mu, double lmin, float *a_out, float *b_out,
                       int64_t cap) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double m[3], v[3];
            for (int c = 0; c < 3; ++c) {
                m[c] = (double)x[3 * i + c] - (double)x[3 * j + c];
                v[c] = (double)y[3 * i + c] - (double)y[3 * j + c];
            }
            const double lm = sqrt((m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]);
            const double ln = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
            if (!(lm > lmin && ln > lmin && fabs(lm - ln) <= mu)) continue;
            if (a_out && b_out && k < cap)
                for (int c = 0; c < 3; ++c) {
                    a_out[3 * k + c] = (float)(m[c] / lm);
                    b_out[3 * k + c] = (float)(v[c] / ln);
                }
            ++k;
        }
    return k;
}

static int cmp_i64(const void *p, const void *q) {
    const int64_t a = *(const int64_t *)p, b = *(const int64_t *)q;
    return (a > b) - (a < b);
}

/* Translation by voting (Sec. 4.5.2): each correspondence gives the
 * candidate t_i = y_i - R x_i (row k: y_k - ((R_k0 x_0 + R_k1 x_1) + R_k2 x_2)),
 * counted in the cell c = floor((t + L) / s), s = 2L / G, of a G^3 grid over
 * [-L, L]^3 (candidates outside are not counted).  The winner is the largest
 * count, ties to the smallest linear index (c_z G + c_y) G + c_x; t is its
 * centre -L + (c + 1/2) s.  Returns the winner's count (0: no candidate). */
int32_t rvo_pose_translation(const float *x, const float *y, int64_t n, const double R[9], double L, int G, double t[3],
                             int64_t *cell) {
    const double s = (2.0 * L) / (double)G;
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nk = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c3[3];
        int ok = 1;
        for (int r = 0; r < 3; ++r) {
            const double rx = (R[3 * r] * (double)x[3 * i] + R[3 * r + 1] * (double)x[3 * i + 1]) +
                              R[3 * r + 2] * (double)x[3 * i + 2];
            const double tk = (double)y[3 * i + r] - rx;
            const double f = floor((tk + L) / s);
            if (!(f >= 0.0 && f < (double)G)) ok = 0;
            c3[r] = ok ? (int64_t)f : 0;
        }
        if (ok) key[nk++] = (c3[2] * G + c3[1]) * G + c3[0];
    }
    /* counts by sorting the keys */
    qsort(key, (size_t)nk, sizeof(int64_t), cmp_i64);
    int64_t best = -1;
    int32_t bc = 0;
    for (int64_t a = 0; a < nk;) {
        int64_t b = a;
        while (b < nk && key[b] == key[a]) ++b;
        if (b - a > bc) { /* strictly larger: the first (smallest) key keeps ties */
            bc = (int32_t)(b - a);
            best = key[a];
        }
        a = b;
    }
    free(key);
    *cell = best;
    if (best < 0) {
        t[0] = t[1] = t[2] = 0.0;
        return 0;
    }
    const int64_t cx = best % G, cy = (best / G) % G, cz = best / ((int64_t)G * G);
    t[0] = -L + ((double)cx + 0.5) * s;
    t[1] = -L + ((double)cy + 0.5) * s;
    t[2] = -L + ((double)cz + 0.5) * s;
    return bc;
}
