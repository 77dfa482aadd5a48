/*
 * rot_vote.h -- C ABI of the GB300 (sm_103a) rotation-voting library.
 *
 * Method: "Linearly Solving Robust Rotation Estimation" (arXiv 2506.11547).
 * Each correspondence (a_i, b_i), b_i ~ R a_i, confines the unit quaternion
 * of R to a great circle of S^3 (Sec. 4.1).  Lemma 1 (Sec. 4.2) writes that
 * circle as two linear equations; App. A shows the circle is the +1
 * eigenspace of the symmetric M_i = L(a_i)^T L'(b_i), so with
 * S_i = (I - M_i)/2 = I - P_i the quadratic form q^T S_i q is
 * sin^2(distance on S^3 from q to circle i).  App. D gives the same S_i as
 * A_i^T A_i / 4 for the rank-2 skew matrix A_i with A_i q = 0.
 *
 * The library votes over a grid on the w >= 0 hemisphere charted by the
 * quaternion's vector part (x, y, z) in the unit ball (Sec. 4.3.1 reduces
 * the search to a hemisphere and to a 3-D accumulator): cell c votes for
 * pair i iff q_c^T S_i q_c <= tau_c = sin^2(delta + r_c), r_c a covering
 * radius of the cell.  That is the dense "each cell tests each circle" dual
 * of Alg. 1 (Sec. 4.3.2).  It then ranks cells, refines the top K by 2x2x2
 * subdivision for `levels` levels, and fits the rotation as the smallest
 * eigenvector of sum_{inliers} S_i -- the least-squares solution of the
 * stacked system Q q = 0 of Eq. (stack), Sec. 4.2.
 *
 * Vote counts are exact: every (cell, pair) decision is that of the FP64
 * evaluation of q^T S_i q <= tau written as the definition's sequence of
 * IEEE double operations (App. A's M = L(a)^T L'(b) summed over k, S =
 * (I - M)/2, v = sum over (r, c) of q_r S_rc q_c, tau = sin^2(delta + r_c)).
 * A fast value (FP32, or FP16/BF16 on the tensor cores) decides a test when it
 * lies outside a rigorous error band of the threshold, an FP32 re-check when
 * it lies inside, and the FP64 evaluation itself when the re-check lies within
 * 2e-6 of the threshold.  Tests with |v - tau| <= 1e-6 in FP64 are counted as
 * that evaluation decides and reported in rot_vote_result.ambiguous.
 *
 * Conventions
 *   - Quaternions are (w, x, y, z), scalar first; rotation matrices are
 *     row-major 3x3 (App. A).
 *   - Every call returns a rot_vote_status.  Per-problem outcomes go in
 *     rot_vote_result.status.
 *   - Pointers a, b may be host or device memory (the library asks the CUDA
 *     driver which).  Host inputs are copied to the device inside the call.
 *     The caller owns a and b; they must stay valid until rot_vote_solve
 *     returns, or until rot_vote_poll returns a terminal status for the
 *     ticket.  The library never frees caller memory.
 *   - A context is not thread-safe: use one context per thread, or lock.
 *     (rot_vote_submit / rot_vote_poll may be called from one thread while
 *     the context's own scheduler thread runs.)
 *   - The library never prints; rot_vote_last_error describes the last
 *     failure on a context.
 *   - Device memory is allocated with cudaMalloc by the context (workspace
 *     grown on demand up to config.device_mem_budget) and freed by
 *     rot_vote_destroy.
 */
#ifndef ROT_VOTE_H
#define ROT_VOTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rot_vote_ctx rot_vote_ctx;

typedef enum {
    ROT_VOTE_OK = 0,
    ROT_VOTE_PENDING = 1,       /* rot_vote_poll: not finished within the timeout */
    ROT_VOTE_EINVAL = -1,       /* bad argument or invalid input data */
    ROT_VOTE_ENOMEM = -2,       /* device (or pinned host) allocation failed or over budget */
    ROT_VOTE_ECUDA = -3,        /* a CUDA runtime call failed; see rot_vote_last_error */
    ROT_VOTE_EAGAIN = -4,       /* rot_vote_submit: admission queue full */
    ROT_VOTE_ETIMEDOUT = -5,    /* a bounded device-side wait gave up */
    ROT_VOTE_EDEGENERATE = -6,  /* fit degenerate: < 2 inliers or a repeated smallest eigenvalue */
    ROT_VOTE_ENOTFOUND = -7,    /* rot_vote_poll: unknown or already collected ticket */
    ROT_VOTE_ETOOLARGE = -8     /* rot_vote_count_cells_static: n or ncells above its static limits */
} rot_vote_status;

/* Arithmetic of the dominant (cell, pair) contraction.  All modes give the
 * same exact counts; they differ in speed and in how many tests need the
 * FP32 re-check.
 *   FP32    -- CUDA-core FP32 form: 9 fused multiply-adds per test, the cell's
 *              rotation against the pair's outer product b a^T (App. A's
 *              bilinear form q^T M q = b^T R(q) a).
 *   FP16    -- tcgen05 tensor-core form, monomials and S entries in FP16
 *              (K = 10 + 2 threshold columns, padded to 16; the padding
 *              carries the low halves of the four diagonal S entries), FP32
 *              accumulation in tensor memory.
 *   BF16    -- as FP16 with BF16 operands.
 *   FP16X2, BF16X2 -- hi/lo split operands (K = 32): far fewer re-checks. */
typedef enum {
    ROT_PREC_FP32 = 0,
    ROT_PREC_FP16 = 1,
    ROT_PREC_BF16 = 2,
    ROT_PREC_FP16X2 = 3,
    ROT_PREC_BF16X2 = 4
} rot_vote_precision;

typedef enum { ROT_RANK_EXCESS = 0, ROT_RANK_RAW = 1 } rot_vote_rank_mode;

/* Context configuration.  Every field has a default; 0 selects it. */
typedef struct {
    int grid_n;               /* coarse cells per axis over [-1,1]^3; power of two in [2, 256]; default 32 */
    int levels;               /* refinement levels (2x2x2 split of the kept cells); default 0 */
    int top_k;                /* cells kept per level; default 16, at most 64 */
    int precision;            /* rot_vote_precision; default ROT_PREC_FP32 */
    float recheck_band;       /* requested low-precision re-check band; the band used is
                                 max(requested, the rigorous error bound of the mode) */
    int rank_mode;            /* rot_vote_rank_mode: EXCESS (score = count - N tau, default) or RAW */
    int refit_iters;          /* refit iterations T; default 8; negative = no refit */
    size_t device_mem_budget; /* bytes of device workspace the context may hold; default 16 GiB */
    int max_inflight;         /* serving: problems in flight at once; default 256 */
    void *cuda_stream;        /* cudaStream_t to run on (e.g. torch's current stream); NULL = own stream */
    int use_graphs;           /* 1 = capture the solve pipeline in a CUDA graph and replay it for
                                 repeated solves of the same shape; default 1; negative = off */
    int keep_trace;           /* 1 = keep per-level cell counts for rot_vote_level_trace; 2 = that and
                                 per-kernel timing for rot_vote_stage_times; default 0 */
    int autotune;             /* 1 = on the first solve of each shape class (precision, size bucket), time
                                 every vote tile-shape candidate on its coarse level and keep the fastest
                                 (cached per context; appended to the file named by the environment
                                 variable ROT_VOTE_TUNE_CACHE if set); default 1; negative = off
                                 (a fixed default shape); >= 2 = always use the tile shape with this
                                 code (tests, diagnostics): FP32 form 4, 8 (scalar kernel, cells per
                                 thread) or 102, 104, 114, 124 (packed f32x2 kernel; 114 / 124 with 5 /
                                 6 CTAs per SM); tensor-core forms 2, 4
                                 (epilogue warpgroups) + 10 (16-column TMEM chunks) + 100 (128-pair
                                 MMA units), i.e. 2, 4, 12, 14, 102, 104, 112, 114.  A code that
                                 does not exist for the precision fails the solve with EINVAL. */
    int chart;                /* chart of the cell grid over [-1,1]^3: 0 = orthographic (default), the
                                 quaternion's vector part with w >= 0; 1 = stereographic (Sec. 4.3.1),
                                 q = P'(p) = (2p, |p|^2 - 1) / (1 + |p|^2) read as (q0, q1, q2, q3), so
                                 the unit ball is the half q3 <= 0.  In the stereographic chart every
                                 cell's covering radius is within a factor ~2 of every other's on a
                                 level; rot_vote_level_trace indices refer to the chosen chart */
} rot_vote_config;

/* One problem.  a, b: [n, 3] row-major float32 unit vectors (host or device).
 * Inputs are valid iff n >= 2, every value is finite, and | |a_i|^2 - 1 |,
 * | |b_i|^2 - 1 | <= 1e-5; otherwise the problem's status is ROT_VOTE_EINVAL. */
typedef struct {
    const float *a;
    const float *b;
    int64_t n;
    float delta;  /* vote tolerance: an angle on S^3 in radians, 0 < delta < pi/2.
                     The residual angle angle(R a_i, b_i) is 2x the S^3 distance. */
    int grid_n;   /* 0 = context default */
    int levels;   /* 0 = context default; negative = force 0 levels */
} rot_vote_problem;

typedef struct {
    double q[4];          /* fitted rotation, unit quaternion with w > 0 (or first nonzero > 0) */
    double R[9];          /* its rotation matrix, row-major */
    int32_t best_count;   /* vote count of the winning cell (rank 1 at the last level) */
    int32_t inliers;      /* pairs in the final fit */
    int64_t best_cell;    /* linear index (iz*n + iy)*n + ix of the winner at its level */
    int32_t best_level;   /* level of the winner */
    int32_t refits;       /* refit iterations performed */
    int64_t tests;        /* (cell, pair) tests over all levels */
    int64_t rechecked;    /* tests re-evaluated by the FP32 re-check */
    int64_t ambiguous;    /* tests with |v - tau| <= 1e-6 in FP64 (decided by the FP64 evaluation) */
    int32_t status;       /* rot_vote_status of this problem */
    float ms_gpu;         /* device time of the solve call that produced it (batched: the batch) */
    float latency_ms;     /* serving: submit -> completion observed; else 0 */
    int64_t resolved;     /* re-checked tests within 2e-6 of the threshold in FP32, decided by the
                             FP64 evaluation of q^T S q <= tau */
} rot_vote_result;

/* Create a context on the current CUDA device.  cfg may be NULL (all defaults).
 * Errors: EINVAL (bad config), ECUDA, ENOMEM. */
int rot_vote_create(const rot_vote_config *cfg, rot_vote_ctx **out);

/* Solve n_problems independent problems and block until their results are
 * in out[0..n_problems).  n_problems > 1 runs them batched: each kernel of
 * the path covers every problem in one launch.  A problem's result does not
 * depend on which other problems share the call.
 * Returns OK when the call ran (per-problem status in out[k].status), or
 * EINVAL / ENOMEM / ECUDA when it could not run at all. */
int rot_vote_solve(rot_vote_ctx *ctx, const rot_vote_problem *p, int n_problems, rot_vote_result *out);

/* Serving: queue one problem without blocking.  The context's scheduler
 * admits queued problems as in-flight slots and device memory free up and
 * launches them in waves that overlap on the device (continuous batching).
 * Returns OK and a ticket, or EAGAIN when the admission queue is full. */
int rot_vote_submit(rot_vote_ctx *ctx, const rot_vote_problem *p, uint64_t *ticket);

/* Serving: wait up to timeout_us (0 = just check) for a ticket.  Returns OK
 * (result written, ticket released), PENDING, or ENOTFOUND. */
int rot_vote_poll(rot_vote_ctx *ctx, uint64_t ticket, rot_vote_result *out, int timeout_us);

/* Test/diagnostic: the cells of one level of one problem of the last
 * rot_vote_solve on a context created with keep_trace = 1.  Writes up to cap
 * (linear index, count) pairs in table order and up to top_k kept cells in
 * rank order.  Returns OK, EINVAL (no trace / out of range) or ECUDA. */
int rot_vote_level_trace(rot_vote_ctx *ctx, int problem, int level, int64_t *idx, int32_t *count,
                         int64_t cap, int64_t *ncells, int64_t *kept_idx, int32_t *nkept);

/* Diagnostic: device time of each stage of the last rot_vote_solve (or rot_vote_alg1) on
 * a context created with keep_trace = 2.  Such a context launches the
 * pipeline stage by stage (no CUDA graph) with a pair of CUDA events on its
 * stream around every stage; `kernels` is the number of kernel launches the
 * stage made (the coarse top-K is two kernels, the fit one per refit
 * iteration for problems above 32768 pairs).  kind: 0 pair step, 1 vote,
 * 2 top-K with the next level's children, 4 fit (3 is unused); level: the
 * level (-1 for pair step and fit).  After rot_vote_alg1 the entries are the
 * stages of its last problem: kind 5 accumulator zeroing and circle bases,
 * 6 sampling vote, 7 argmax, the kernels gated on a counter wrap, the peak
 * search and the result (level -1).
 * Writes up to cap entries and their total count.  Returns OK or EINVAL. */
typedef struct {
    int32_t kind;
    int32_t level;
    float ms;
    int32_t kernels;
} rot_vote_stage;

int rot_vote_stage_times(rot_vote_ctx *ctx, rot_vote_stage *out, int cap, int *count);

/* Diagnostic of the serving loop (rot_vote_submit / rot_vote_poll): the
 * device-time span of every serving batch completed so far on the context,
 * in completion order (at most the last 65536).  t_start_ms / t_end_ms are
 * the times of the events recorded on the wave's stream before the batch's
 * first launch and after its last, in ms after serving started (the first
 * submit); two batches overlapped on the device when their spans intersect.
 * The paper has no counterpart: this measures the build's continuous
 * batching.  Writes up to cap spans (the oldest first) and their total count.
 * Returns OK or EINVAL. */
typedef struct {
    float t_start_ms;
    float t_end_ms;
    int32_t wave;      /* serving wave (stream) that ran the batch */
    int32_t problems;  /* problems in the batch */
} rot_vote_batch_span;

int rot_vote_serve_spans(rot_vote_ctx *ctx, rot_vote_batch_span *out, int cap, int *count);

/* Destroy a context: waits for in-flight work, frees its memory. */
void rot_vote_destroy(rot_vote_ctx *ctx);

/* Text of the last error on ctx ("" if none); valid until the next call on ctx. */
const char *rot_vote_last_error(const rot_vote_ctx *ctx);

/* ---- Allocation-free vote (the paper has no counterpart: a deployment aid) ----
 *
 * rot_vote_count_cells_static counts, for each of ncells caller-given cells of
 * the grid_n^3 grid (linear index (iz*grid_n + iy)*grid_n + ix), how many of
 * the n pairs vote for it: the same FP32 CUDA-core vote, with the same exact
 * counts, as a context's solve in ROT_PREC_FP32.  It allocates no device
 * memory and calls no allocating library routine: its pair pool, cell table
 * and work lists live in one file-scope static device array of
 * ROT_VOTE_STATIC_SCRATCH_BYTES that every GPU which loads the library holds
 * until the process exits.  It is for callers that cannot allocate device
 * memory: code running inside a framework whose caching allocator owns the
 * device's memory (a cudaMalloc behind its back can fail or fragment it), and
 * per-frame real-time loops that cannot take the device-wide synchronisation
 * of cudaFree.
 *
 * Arguments
 *   a, b    float32 [n][3] unit vectors, b_i ~ R a_i, in device memory of the
 *           current device (or managed memory)
 *   n       2 <= n <= ROT_VOTE_STATIC_MAX_PAIRS
 *   delta   inlier angle threshold, 0 < delta < pi/2 (rounded to float, as in
 *           rot_vote_problem)
 *   grid_n  grid side, a power of two in [2, 2^20]
 *   cells   int64 [ncells] linear cell indices (current device); each cell's box must
 *           meet the unit ball (a cell of the level table)
 *   ncells  1 <= ncells <= ROT_VOTE_STATIC_MAX_CELLS
 *   counts  int32 [ncells] (current device), written (the call zeroes it first)
 *   cuda_stream  cudaStream_t to run on (NULL = the legacy default stream)
 * The call runs on the current device and returns after the counts are
 * written (it synchronises cuda_stream).  The caller owns every buffer.
 *
 * Returns OK; ETOOLARGE (n or ncells above the limits, nothing launched);
 * EINVAL (bad argument, a pointer that is not memory of the current device
 * nor managed memory, a non-unit or
 * non-finite input vector, or a cell index outside the level table -- counts
 * are then unspecified); ECUDA.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the process; make that first call
 * before any stream capture.  cudaDeviceReset on that device unloads the
 * module and may move the array, so after a reset the entry point must not be
 * called again in that process.
 * Every call on a device shares the one array and leaves its contents behind;
 * each call rewrites everything it reads before reading it.  Calls whose work
 * overlaps on the GPU (other host threads, other streams) race on the array:
 * serialise them. */
#define ROT_VOTE_STATIC_SCRATCH_BYTES (4 << 20)
#define ROT_VOTE_STATIC_MAX_PAIRS 32768
#define ROT_VOTE_STATIC_MAX_CELLS 8192
int rot_vote_count_cells_static(const float *a, const float *b, int64_t n, double delta, int grid_n,
                                const int64_t *cells, int32_t ncells, int32_t *counts, void *cuda_stream);

/* ---- Alg. 1: the paper's own voting by sampled circles (Sec. 4.3.2) ----
 *
 * For every pair the circle of rotations taking a_i to b_i (Sec. 4.1) is
 *   q(alpha) = q_b1 cos(alpha/2) + q_b2 sin(alpha/2),
 * with q_b1 the quaternion of the minimal rotation from a to b, written with
 * the half-angle identities
 *   w = sqrt((1 + a.b)/2),  q_b1 = (w, (a x b) / (2 w)),
 * and q_b2 = (-b.v, w b + b x v), v the vector part of q_b1 (q_b2 = [0, b] q_b1:
 * the half turn about b after the minimal rotation).  Alg. 1 samples alpha_j = -pi + 2 pi j / J,
 * j = 0 .. J-1, takes each sample with the sign that gives q3 <= 0 (q and -q
 * are one rotation; Sec. 4.3.1), projects it stereographically,
 *   p = (q0, q1, q2) / (1 - q3),            a point of the closed unit ball,
 * and counts it in the cell i_k = clamp(floor((p_k + 1) n / 2), 0, n - 1) of
 * an n^3 accumulator over [-1, 1]^3, linear index (i2 n + i1) n + i0.  The
 * winner is the largest count (ties: the smallest index); the rotation is
 * the inverse projection of the winner's centre p* = -1 + (i + 1/2) 2/n,
 *   q = (2 p*, |p*|^2 - 1) / (1 + |p*|^2),
 * with the sign w > 0 (w = 0: the first nonzero component > 0).
 *
 * The cell of every sample is the cell that the same formulas give in IEEE
 * double arithmetic, operation by operation in the order written above
 * (products a_k b_k formed from the float32 inputs; (cos, sin)(alpha_j / 2)
 * from the host C library).  The device evaluates each sample in FP32 and
 * repeats it in FP64 when the FP32 result lies within a proven error bound
 * (times a safety factor) of a cell boundary or of q3 = 0; the accumulator is
 * therefore exact.  A pair with a = -b (w = 0, no circle) casts no sample.
 */
/* Multiple rotations (Sec. 4.4: several motions in one scene vote several
 * peaks).  With rot_vote_alg1_problem.peaks = M >= 1 the call also returns up
 * to M peaks of the accumulator by greedy non-maximum suppression:
 *   - T = max(min_count, the smallest t >= 1 with at most
 *     ROT_VOTE_ALG1_PEAK_CANDIDATES cells of count >= t);
 *   - the candidates, the cells with count >= T, are taken in (count desc,
 *     index asc) order;
 *   - a candidate becomes a peak unless its centre rotation lies within
 *     nms_angle of an earlier peak's, i.e. |q . q_peak| >= cos(nms_angle / 2)
 *     with the dot product summed as ((q0 q0' + q1 q1') + q2 q2') + q3 q3' in
 *     IEEE double arithmetic; q of a cell is the inverse projection of its
 *     centre, as for the winner.
 * The decisions equal that FP64 definition exactly.  When more than
 * ROT_VOTE_ALG1_PEAK_CANDIDATES cells reach 65535 counts, T is not computed:
 * peak_threshold = -1 and no peak is returned. */
#define ROT_VOTE_ALG1_MAX_PEAKS 64
#define ROT_VOTE_ALG1_PEAK_CANDIDATES 16384
typedef struct {
    double q[4];            /* centre rotation of the peak's cell, canonical sign */
    int64_t cell;           /* its linear index */
    int32_t count;          /* its count */
    int32_t pad;
} rot_vote_peak;

typedef struct {
    const float *a;         /* [n,3] row-major float32 unit vectors, host or device memory; */
    const float *b;         /*   validity as in rot_vote_problem */
    int64_t n;              /* pairs, 2 <= n <= 2^30 */
    int samples;            /* J, samples per circle, 1 <= J <= 65536, n J <= 2^31 - 1 (counts are
                               int32); 0 = 180 */
    int accum_side;         /* n of the n^3 accumulator, 2 <= n <= 1024; 0 = 360 */
    int32_t *accumulator;   /* optional (NULL: not returned): host or device int32 [n^3], receives the
                               counts in linear-index order; owned by the caller */
    int peaks;              /* M, 0 <= M <= ROT_VOTE_ALG1_MAX_PEAKS: 0 = no peak list */
    int min_count;          /* peaks: the smallest count a peak may have; 0 = 1 */
    float nms_angle;        /* peaks: suppression radius theta, a rotation angle in radians, >= 0 */
    rot_vote_peak *peak_out; /* peaks: host array of M entries, written in peak order; owned by the caller */
} rot_vote_alg1_problem;

typedef struct {
    double q[4];            /* rotation of the winning cell, canonical sign */
    double R[9];            /* its rotation matrix, row-major */
    int32_t best_count;     /* count of the winning cell */
    int32_t status;         /* rot_vote_status of this problem */
    int64_t best_cell;      /* linear index of the winning cell */
    int64_t samples_cast;   /* J x (pairs with a circle) */
    int64_t rechecked;      /* samples whose cell the device decided in FP64 */
    float ms_gpu;           /* device time of this problem (accumulator zeroing to result) */
    int32_t npeaks;         /* peaks written to peak_out */
    int32_t peak_threshold; /* T of the peak search (-1: not computed), 0 without peaks */
    int32_t vote_path;      /* how the counts were taken (exact on every path): 0 one vote with
                               return-less atomics; 1 that vote, whose 16-bit counters wrapped, then
                               the vote again with atomics that record the wraps; 2 the recording
                               vote alone, chosen when the context's previous problem had wraps */
    int32_t wrapped_words;  /* counter words (two cells each) holding a cell with 65536 or more votes */
} rot_vote_alg1_result;

/* Run Alg. 1 on n_problems problems, one after another on the context's
 * stream (each needs its own n^3 accumulator; the context keeps one, of
 * 16-bit counters with an exact record of their wraps, about 2 n^3 bytes,
 * inside config.device_mem_budget), and block until out[] is
 * written.  Returns OK when the call ran (per-problem status in
 * out[k].status: OK, or EINVAL for bad arguments or inputs -- non-finite
 * or non-unit vectors -- with the rest of out[k] unspecified), or ENOMEM /
 * ECUDA / EINVAL when it could not run at all. */
int rot_vote_alg1(rot_vote_ctx *ctx, const rot_vote_alg1_problem *p, int n_problems, rot_vote_alg1_result *out);

/* ---- Rigid pose (Sec. 4.5): rotation and translation from point correspondences ----
 *
 * y_i = R x_i + t for the inliers.  Every pair i < j gives the translation-free
 * correspondence R m = n with m = x_i - x_j, n = y_i - y_j; the rotation-invariant
 * length check of Sec. 4.5.1 keeps the pair iff
 *   |m| > min_length,  |n| > min_length  and  | |m| - |n| | <= mu
 * (lengths sqrt((v0^2 + v1^2) + v2^2) in IEEE double from the float32 points).
 * The kept pairs, as the float32 unit vectors (m / |m|, n / |n|) in (i, j)
 * lexicographic order, are solved by the context's rotation vote
 * (rot_vote_solve with delta, grid_n, levels).  Translation (Sec. 4.5.2): every
 * correspondence gives t_i = y_i - R x_i with the solved R (row r:
 * y_r - ((R_r0 x_0 + R_r1 x_1) + R_r2 x_2), double), counted in the cell
 * floor((t + L) / s), s = 2L / G, of a G^3 grid over [-L, L]^3; the winner is
 * the largest count (ties: the smallest index (c_z G + c_y) G + c_x) and t is its
 * centre -L + (c + 1/2) s.  The kept pairs equal the IEEE double definition
 * exactly: each length check is made in FP32 and, within its rigorous error
 * band of a threshold, in FP64. */
typedef struct {
    const float *x;         /* [n][3] float32 points, host or device; finite, |coordinate| <= 1e15 */
    const float *y;
    int64_t n;              /* 2 <= n <= 65536 */
    float mu;               /* length tolerance mu_t > 0 */
    float min_length;       /* >= 0: shorter differences are dropped (no direction) */
    float delta;            /* rotation vote tolerance, as rot_vote_problem.delta */
    int grid_n;             /* rotation grid, as rot_vote_problem (0 = context defaults) */
    int levels;
    float t_half;           /* L, the translation domain [-L, L]^3; 0 = 5 */
    int t_cells;            /* G, cells per axis, 1..1024; 0 = 400 (step 0.025 for L = 5) */
    float *pairs_a;         /* optional (pairs_cap > 0): host or device float32 [pairs_cap][3] receiving */
    float *pairs_b;         /*   the first pairs_cap kept unit pairs; owned by the caller */
    int64_t pairs_cap;
} rot_vote_pose_problem;

typedef struct {
    rot_vote_result rot;    /* the rotation solve over the kept pairs (its own status and ms_gpu) */
    double t[3];            /* translation: the centre of the winning cell */
    int64_t t_cell;         /* its linear index; -1 when no candidate fell inside [-L, L]^3 */
    int64_t pairs_tested;   /* n (n - 1) / 2 */
    int64_t pairs_kept;
    int64_t pairs_rechecked; /* length checks decided in FP64 */
    int32_t t_count;        /* candidates in the winning cell */
    int32_t status;         /* OK; EINVAL (bad argument or point); EDEGENERATE (fewer than 2 pairs kept, or
                               the rotation fit degenerate); otherwise the rotation solve's status */
    float ms_gpu;           /* device time of the pair stage and the translation vote */
    float pad;
} rot_vote_pose_result;

/* Solve n_problems pose problems one after another on the context's stream and
 * block until out[] is written.  Device memory for the kept pairs (24 bytes per
 * pair) counts against config.device_mem_budget.  Returns OK when the call ran
 * (per-problem status in out[k].status), or ENOMEM / ECUDA / EINVAL. */
int rot_vote_pose(rot_vote_ctx *ctx, const rot_vote_pose_problem *p, int n_problems, rot_vote_pose_result *out);

#ifdef __cplusplus
}
#endif

#endif /* ROT_VOTE_H */
