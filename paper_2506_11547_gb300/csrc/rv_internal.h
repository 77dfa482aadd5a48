// rv_internal.h -- data layouts and kernel launch interfaces shared by the
// translation units of librot_vote.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rot_vote.h"

namespace rv {

constexpr int kMaxLevels = 12;      // refinement levels per problem
constexpr int kMaxTopK = 64;
constexpr int kPairTile = 256;      // pairs per pool tile (tensor-core B tile rows = MMA N)
constexpr int kCellTile = 128;      // cells per tensor-core A tile (TMEM lanes)
constexpr float kBandR = 5e-6f;     // FP32 form: |d| band, d = fma-chain(-R_c, b a^T, 1 - 2 tau) ~ 2 (v - tau)
constexpr int kSelChunk = 4096;     // cells per top-K phase-1 block
constexpr int kSimtItemCells = 1024; // cells per CUDA-core vote work item (any cells-per-thread variant)

// Per-cell record of a level table (structure of arrays).
//   q     FP64 centre quaternion (w, x, y, z)
//   chord FP64 covering chord (r = 2 asin(chord / 2))
//   trig  FP64 (cos r, sin r), so tau = sin^2(delta + r) costs no sqrt/div
//   idx   linear cell index (iz*n + iy)*n + ix at the table's level
//   m32   monomials [w2 x2 y2 z2 2wx 2wy 2wz 2xy 2xz 2yz] rounded to f32, + 2 pad (48 B)
//   R32   rotation matrix of q rounded to f32, row-major, + 3 pad (48 B)
struct CellSoA {
    double4_32a *q;
    double *chord;
    double2 *trig;
    int64_t *idx;
    float4 *m32;  // 3 float4 per cell
    float4 *R32;  // 3 float4 per cell
};

// One (problem, level) of a solve.
struct LevelRef {
    CellSoA cells;
    const int32_t *ncells;  // device count of cells at this level
    int32_t *counts;        // [cap] vote counts (zeroed before the vote)
    int32_t cap;            // capacity of the table
    int32_t n_side;         // grid side at this level
    int32_t chart;          // 0 orthographic, 1 stereographic (Sec. 4.3.1)
    int32_t pad;
};

// One problem of a solve.
struct ProbRef {
    const float *a;      // caller / staged input, [n][3]
    const float *b;
    int64_t n;
    int64_t pool_off;    // first pair in the pair pool (multiple of kPairTile)
    double sin_d, cos_d; // of delta
    float delta;
    int32_t levels;      // last level index (0 = coarse only)
    int32_t grid_n;
};

// Per-problem device outputs / statistics.
struct ProbStats {
    unsigned long long tests;
    unsigned long long rechecked;
    unsigned long long ambiguous;
    unsigned long long resolved;  // tests decided by the FP64 evaluation
    int32_t invalid;     // input validation failed
    int32_t pad;
};

// A vote work item: cells [cell_begin, cell_begin + cells) of (prob, level)
// against pairs [pair_begin, pair_end) of the problem.
struct VoteItem {
    int32_t prob;
    int32_t cell_begin;
    int32_t pair_begin;
    int32_t pair_end;
};

// Top-K candidate.
struct Cand {
    double score;
    int64_t idx;
    int32_t pos;  // position in the level table; -1 = none
    int32_t pad;
};

// Pair pool: one record per pair, padded to kPairTile per problem.
//   p32  [P][3] float4: P = b a^T row-major [b0a0 b0a1 b0a2 b1a0 b1a1 b1a2 b2a0 b2a1 b2a2] + 3 pad
//        (padding pairs: 0), the FP32 form's operand (q^T S q = (1 - b^T R(q) a) / 2, App. A)
//   pr   [P][2] float4: a0 a1 a2 b0 | b1 b2 c 0, c = (|a|^2 + |b|^2 - 2)/4
//   tcb  tensor-core operand tiles (16-bit S entries), layout described in k_vote_tc.cu
struct PairPool {
    float4 *p32;
    float4 *pr;
    void *tcb;
    int tc_k;  // 16 or 32 (0 if absent)
    // [P/2][5] float4, pairs (i, i+1) interleaved for the packed FP32 vote: float4 k < 4 of
    // pair-pair j = (P_2k(2j), P_2k(2j+1), P_2k+1(2j), P_2k+1(2j+1)), float4 4 = (P_8(2j),
    // P_8(2j+1), 0, 0); null if absent
    float4 *p2x = nullptr;
};

// A (cell, pair) test whose FP32 re-check lands within kBand64 of the
// threshold, deferred to the FP64 resolution pass: problem, position in the
// level table, pool index of the pair.  The vote kernels leave such a test
// uncounted; resolve64 counts it.
struct Amb64 {
    int32_t prob;
    int32_t pos;
    int64_t gp;
};

// The deferred tests of one level: q[0 .. min(*count, cap)).  q == nullptr (or
// a full queue): the vote kernel decides the test in FP64 itself.
struct AmbQueue {
    Amb64 *q = nullptr;
    int *count = nullptr;  // zeroed before the level's vote
    int *ovf = nullptr;    // set when a test found the queue full (zeroed before the vote)
    int cap = 0;
    int pad = 0;
};

// Set in a cell's count when one of its tests found the FP64 queue full: the
// resolution pass then recounts that cell from all of its pairs.  Counts stay
// below 2^30 (problems hold fewer than 2^30 pairs).
constexpr int32_t kOvfBit = 1 << 30;

// ---- launchers (each returns cudaGetLastError() of its launch) ----

// Coarse table of an n^3 grid from its non-empty rows {first table position, ix_lo, ix_hi, iz*n + iy}.
cudaError_t launch_build_level0(const int4 *rows, int nrows, int n, int chart, int64_t ncells, CellSoA out, cudaStream_t s);

// Pair step over a list of {problem, pair tile}: validates inputs and fills the pair pool.
cudaError_t launch_pair_prep(const ProbRef *probs, const int2 *tiles, int ntiles, PairPool pool, int tc_prec,
                             ProbStats *stats, cudaStream_t s);

// Vote, CUDA-core FP32 form.  variant: cells per thread (4 or 8) of the scalar
// kernel, or 100 + cells per thread (2 or 4) of the packed f32x2 kernel (needs pool.p2x),
// + 10 / + 20 for 5 / 6 resident CTAs per SM (codes 114, 124).
// item_counter: a zeroed int through which CTAs take work items dynamically; null =
// items in grid-stride order.
cudaError_t launch_vote_simt(const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                             int level_stride, int level, PairPool pool, ProbStats *stats, int variant,
                             int grid_blocks, int *item_counter, AmbQueue amb, cudaStream_t s);

// Vote, tcgen05 tensor-core form. prec: ROT_PREC_FP16 .. BF16X2; variant = epilogue
// warpgroups (2 or 4), plus 10 for 16-column instead of 32-column TMEM chunks, plus
// 100 for 128-pair MMA units in four accumulator stages (else 256 pairs, two stages).
// Every device wait is bounded (2 s); on expiry *err_flag is set and the kernel
// returns.  test_stall != 0 (fault-injection tests only): the producer issues no
// copies and each wait is bounded by 1 ms, so the kernel must report through
// *err_flag and leave the context usable.
cudaError_t launch_vote_tc(const VoteItem *items, int n_items, const ProbRef *probs, const LevelRef *lref,
                           int level_stride, int level, PairPool pool, ProbStats *stats, int prec, float band_req,
                           int variant, int grid_blocks, int *err_flag, int test_stall, AmbQueue amb,
                           cudaStream_t s);

// Once per process/device, outside stream capture: kernel attributes of the tensor-core vote.
cudaError_t prepare_vote_tc();

// Top-K phase 1 (per chunk of cells) and phase 2 (per problem merge) + children.
cudaError_t launch_topk(const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride, int level,
                        int top_k, int rank_mode, int max_cells, Cand *cand, int chunks_per_prob,
                        int32_t *kept_pos, int32_t *nkept, ProbStats *stats, cudaStream_t s);

// Phase 2 also writes the next level's children (the 8 octants of each kept cell
// that meet the ball) when the problem has a next level.

// Refinement levels (at most kSelChunk cells per problem): top-K and children in
// one block per problem.
cudaError_t launch_select_small(const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride, int level,
                                int top_k, int rank_mode, int32_t *kept_pos, int32_t *nkept, ProbStats *stats,
                                cudaStream_t s);

// Vote of a refinement level, pair-major (one block per 256-pair tile of the
// pair step's tile list); FP32 chain + FP32 re-check, exact counts in every form.
cudaError_t launch_vote_small(const ProbRef *probs, const int2 *tiles, int ntiles, const LevelRef *lref,
                              int level_stride, int level, PairPool pool, ProbStats *stats, AmbQueue amb,
                              cudaStream_t s);

// The FP64 resolution pass of one level's deferred tests (after its vote): each
// test decided by the FP64 evaluation, its vote added to the cell's count, the
// problem's ambiguous and resolved statistics updated; cells flagged with
// kOvfBit (the queue was full) recounted from all of their pairs.
// grid_blocks blocks stride over the queue (its length is read on the device)
// and over the nprob problems' cells of the level.
cudaError_t launch_resolve64(AmbQueue amb, const ProbRef *probs, int nprob, const LevelRef *lref, int level_stride,
                             int level, PairPool pool, ProbStats *stats, int grid_blocks, cudaStream_t s);

// Fit state of a large problem between its passes.
struct FitState {
    double q[4];
    int32_t done, status, nin, refits;
};

// Fit: winner voters, FP64 sum of S_i, eigen-solve, refit loop; writes results.
// Problems with n <= kFitSmallMax (small_list) get one CTA each.  The others
// (big_list) are fitted together on the whole GPU, one launch per iteration
// over every slice of every large problem (slice_part holds 11 doubles per
// 4096-pair slice, problem p's slices from slice_off[p]; big_soff[k] is the
// first of the k-th large problem's slices in a flat list of big_slices); the
// block finishing a problem's slices (done_cnt[k], nbig counters) does its
// reduction and eigen-solve, keeping q in state[k].  The path depends only on
// the problem's own size.
constexpr int64_t kFitSmallMax = 32768;
int fit_slices(int64_t n);
cudaError_t launch_fit(const ProbRef *probs, const LevelRef *lref, int level_stride, const int32_t *kept_pos,
                       int top_k, int refit_iters, PairPool pool, uint8_t *member, double *slice_part,
                       const int64_t *slice_off, const int32_t *small_list, int nsmall, const int32_t *big_list,
                       int nbig, const int64_t *big_soff, int64_t big_slices, FitState *state, int *done_cnt,
                       int sms, const ProbStats *stats, rot_vote_result *results, cudaStream_t s);

}  // namespace rv
