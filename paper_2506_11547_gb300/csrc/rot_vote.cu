// rot_vote.cu -- host runtime behind include/rot_vote.h.
//
// A solve of P problems is planned on the host (work-item lists, table and
// buffer layout inside one device workspace), its descriptors are uploaded
// with one copy, and the device pipeline runs on one stream:
//
//   pair step -> for each level: vote, top-K (+ the next level's children) -> fit -> results
//
// The pipeline of a given shape is captured once in a CUDA graph and
// replayed by later solves of the same shape (only the descriptors change).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rot_vote.h"
#include "rv_internal.h"
#include "rv_runtime.h"

using namespace rv;

namespace rv {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Coarse grid tables (cached per context, shared by all problems and waves).
// ---------------------------------------------------------------------------
static int du(int i, int n) {  // distance from 0 to box i, in units of 1/n
    const int lo = 2 * i - n, hi = 2 * i + 2 - n;
    if (lo > 0) return lo;
    if (hi < 0) return -hi;
    return 0;
}

int Context::grid_table(int n, const GridTable **out) {
    for (auto &g : grids)
        if (g.n == n) {
            *out = &g;
            return ROT_VOTE_OK;
        }
    // non-empty rows (iy, iz) and the ix interval of each, by exact integer test
    std::vector<int4> rows;
    int64_t total = 0;
    for (int iz = 0; iz < n; ++iz)
        for (int iy = 0; iy < n; ++iy) {
            const int64_t r = (int64_t)n * n - (int64_t)du(iy, n) * du(iy, n) - (int64_t)du(iz, n) * du(iz, n);
            if (r < 0) continue;
            int lo = -1, hi = -1;
            for (int ix = 0; ix < n; ++ix)
                if ((int64_t)du(ix, n) * du(ix, n) <= r) {
                    if (lo < 0) lo = ix;
                    hi = ix;
                }
            if (lo < 0) continue;
            rows.push_back(make_int4((int)total, lo, hi, iz * n + iy));
            total += hi - lo + 1;
        }
    GridTable g;
    g.n = n;
    g.ncells = total;
    const size_t bytes = align_up(sizeof(double4_32a) * total, 256) + align_up(sizeof(double) * total, 256) +
                         align_up(sizeof(double2) * total, 256) +
                         align_up(sizeof(int64_t) * total, 256) + 2 * align_up(sizeof(float4) * 3 * total, 256) +
                         256 + align_up(sizeof(int4) * rows.size(), 256);
    if (bytes_held + bytes > budget) return fail(ROT_VOTE_ENOMEM, "grid table exceeds the device memory budget");
    if (cudaMalloc(&g.mem, bytes) != cudaSuccess) return fail(ROT_VOTE_ENOMEM, "cudaMalloc of grid table failed");
    bytes_held += bytes;
    char *p = (char *)g.mem;
    auto take = [&](size_t b) {
        char *r = p;
        p += align_up(b, 256);
        return r;
    };
    g.cells.q = (double4_32a *)take(sizeof(double4_32a) * total);
    g.cells.chord = (double *)take(sizeof(double) * total);
    g.cells.trig = (double2 *)take(sizeof(double2) * total);
    g.cells.idx = (int64_t *)take(sizeof(int64_t) * total);
    g.cells.m32 = (float4 *)take(sizeof(float4) * 3 * total);
    g.cells.R32 = (float4 *)take(sizeof(float4) * 3 * total);
    g.ncells_dev = (int32_t *)take(256);
    int4 *rows_d = (int4 *)take(sizeof(int4) * rows.size());
    const int32_t nc32 = (int32_t)total;
    cudaError_t e = cudaMemcpyAsync(rows_d, rows.data(), sizeof(int4) * rows.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.ncells_dev, &nc32, sizeof(int32_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = launch_build_level0(rows_d, (int)rows.size(), n, cfg.chart, total, g.cells, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(g.mem);
        bytes_held -= bytes;
        return cuda_fail(e, "building the grid table");
    }
    g.bytes = bytes;
    grids.push_back(g);
    *out = &grids.back();
    return ROT_VOTE_OK;
}

int Context::fail(int code, const std::string &msg) {
    last_error = msg;
    return code;
}

int Context::cuda_fail(cudaError_t e, const char *what) {
    last_error = std::string("CUDA error while ") + what + ": " + cudaGetErrorString(e);
    return ROT_VOTE_ECUDA;
}

// ---------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------
static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// The tensor-core vote takes items in grid-stride order (item i on CTA i mod
// grid), so when the item count is not a multiple of the grid, the CTAs of the
// last, partial round run one more item while the others idle.  This splits
// the items of that round by pair range into pieces that spread its work over
// every CTA: for k = 1..4 target pieces per CTA, each item becomes
// round(tiles / piece) pieces (at least one, at least 4 pair tiles each), and
// the split whose busiest CTA ends first is kept (the unsplit round included).
static void split_last_round(std::vector<VoteItem> &items, int grid) {
    const int64_t n = (int64_t)items.size();
    if (grid <= 0 || n <= grid || n % grid == 0) return;
    const int64_t full = n / grid * grid;
    const std::vector<VoteItem> tail(items.begin() + full, items.end());
    auto tiles = [](const VoteItem &it) { return (int64_t)(it.pair_end - it.pair_begin) / kPairTile; };
    int64_t wr = 0;
    for (const VoteItem &it : tail) wr += tiles(it);
    auto split = [&](int k) {
        std::vector<VoteItem> out;
        const int64_t piece = std::max<int64_t>(4, (wr + (int64_t)k * grid - 1) / ((int64_t)k * grid));
        for (const VoteItem &it : tail) {
            const int64_t t = tiles(it);
            const int64_t np = std::max<int64_t>(1, std::min<int64_t>((t + piece / 2) / piece, t / 4));
            for (int64_t z = 0; z < np; ++z) {
                VoteItem x = it;
                x.pair_begin = it.pair_begin + (int32_t)(t * z / np * kPairTile);
                x.pair_end = it.pair_begin + (int32_t)(t * (z + 1) / np * kPairTile);
                out.push_back(x);
            }
        }
        return out;
    };
    auto makespan = [&](const std::vector<VoteItem> &pieces) {  // the busiest CTA's tiles in the round
        std::vector<int64_t> load((size_t)grid, 0);
        for (size_t i = 0; i < pieces.size(); ++i) load[i % (size_t)grid] += tiles(pieces[i]);
        return *std::max_element(load.begin(), load.end());
    };
    std::vector<VoteItem> best = tail;
    int64_t best_ms = makespan(tail);
    for (int k = 1; k <= 4; ++k) {
        std::vector<VoteItem> cand = split(k);
        const int64_t ms = makespan(cand);
        if (ms < best_ms) {
            best_ms = ms;
            best = std::move(cand);
        }
    }
    items.resize((size_t)full);
    items.insert(items.end(), best.begin(), best.end());
}

// Host-side argument check of one problem; returns OK or EINVAL with a reason.
int check_problem(const rot_vote_problem &p, int grid_n, int levels, std::string *why) {
    if (!p.a || !p.b) { *why = "null input pointer"; return ROT_VOTE_EINVAL; }
    if (p.n < 2) { *why = "n < 2"; return ROT_VOTE_EINVAL; }
    if (p.n > (int64_t)1 << 30) { *why = "n > 2^30"; return ROT_VOTE_EINVAL; }
    if (!(p.delta > 0.f) || !(p.delta < 1.5707963f)) { *why = "delta outside (0, pi/2)"; return ROT_VOTE_EINVAL; }
    if (!is_pow2(grid_n) || grid_n < 2 || grid_n > 256) { *why = "grid_n not a power of two in [2, 256]"; return ROT_VOTE_EINVAL; }
    if (levels < 0 || levels > kMaxLevels || ((int64_t)grid_n << levels) > ((int64_t)1 << 20)) {
        *why = "levels out of range (grid side at the last level must be <= 2^20)";
        return ROT_VOTE_EINVAL;
    }
    return ROT_VOTE_OK;
}

static int mem_kind(const void *ptr) {  // 1 = device-accessible device memory, 0 = host
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

static int pinned_kind(const void *ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeHost;
}

int Context::tc_k_of(int prec) const {
    if (prec == ROT_PREC_FP16 || prec == ROT_PREC_BF16) return 16;
    if (prec == ROT_PREC_FP16X2 || prec == ROT_PREC_BF16X2) return 32;
    return 0;
}

// Builds the plan for the valid problems `sel` (indices into p[]).
int Context::plan_batch(Wave &w, const rot_vote_problem *p, const std::vector<int> &sel) {
    Plan &pl = w.plan;
    const int P = (int)sel.size();
    std::vector<int> gridn(P), levs(P);
    bool all_dev = true;
    for (int k = 0; k < P; ++k) {
        const rot_vote_problem &q = p[sel[k]];
        gridn[k] = q.grid_n > 0 ? q.grid_n : cfg.grid_n;
        levs[k] = q.levels > 0 ? q.levels : (q.levels < 0 ? 0 : cfg.levels);
        all_dev = all_dev && mem_kind(q.a) && mem_kind(q.b);
    }
    // same shapes as the wave's current plan, on the same workspace: keep its layout, items and
    // tables, and refresh the inputs and tolerances of the problem table
    if (pl.ws_base != nullptr && pl.ws_base == w.base && pl.nprob == P && pl.shape_dev == all_dev &&
        pl.shape_amb_hook == test_amb_cap && (int)pl.shape_n.size() == P) {
        bool same = true;
        for (int k = 0; k < P && same; ++k)
            same = pl.shape_n[k] == p[sel[k]].n && pl.shape_gl[k] == (((int64_t)gridn[k] << 32) | levs[k]);
        if (same) {
            for (int k = 0; k < P; ++k) {
                const rot_vote_problem &q = p[sel[k]];
                ProbRef &r = pl.probs_h[k];
                const double d = (double)q.delta;
                r.sin_d = std::sin(d);
                r.cos_d = std::cos(d);
                r.delta = q.delta;
                if (all_dev) {
                    r.a = q.a;
                    r.b = q.b;
                }
            }
            pl.reused = true;
            return ROT_VOTE_OK;
        }
    }
    pl = Plan();
    pl.nprob = P;
    pl.prec = cfg.precision;
    pl.top_k = cfg.top_k;
    pl.stride = 0;
    int max_levels = 0;
    for (int k = 0; k < P; ++k) max_levels = std::max(max_levels, levs[k]);
    pl.max_level = max_levels;
    pl.stride = max_levels + 1;
    const int S = pl.stride;
    const int K = pl.top_k;
    const int child_cap = 8 * K;

    // coarse tables
    std::vector<const GridTable *> gt(P);
    for (int k = 0; k < P; ++k) {
        int rc = grid_table(gridn[k], &gt[k]);
        if (rc != ROT_VOTE_OK) return rc;
    }

    // pair pool layout and input residency
    pl.probs_h.resize(P);
    int64_t pool = 0, in_floats = 0;
    for (int k = 0; k < P; ++k) {
        const rot_vote_problem &q = p[sel[k]];
        ProbRef &r = pl.probs_h[k];
        r.n = q.n;
        r.pool_off = pool;
        pool += align_up((size_t)q.n, kPairTile);
        const double d = (double)q.delta;
        r.sin_d = std::sin(d);
        r.cos_d = std::cos(d);
        r.delta = q.delta;
        r.levels = levs[k];
        r.grid_n = gridn[k];
        in_floats += 3 * q.n;
    }
    pl.pool_pairs = pool;
    pl.inputs_on_device = all_dev;
    pl.in_floats = all_dev ? 0 : in_floats;

    // level items
    const int tck = tc_k_of(pl.prec);
    const int cells_per_item = tck ? kCellTile : kSimtItemCells;
    const int blocks_per_sm = tck ? 1 : 4;
    const int slots = sm_count * blocks_per_sm;
    pl.grid_blocks = slots;
    pl.items_h.assign(S, {});
    for (int lev = 0; lev <= max_levels; ++lev) {
        // total work in (cell tile x pair tile) units, to size the pair chunks
        int64_t work = 0;
        for (int k = 0; k < P; ++k) {
            if (lev > levs[k]) continue;
            const int64_t nc = lev == 0 ? gt[k]->ncells : child_cap;
            const int64_t ct = (nc + cells_per_item - 1) / cells_per_item;
            work += ct * (int64_t)(align_up((size_t)pl.probs_h[k].n, kPairTile) / kPairTile);
        }
        // tensor-core form: ~16 items per persistent CTA, taken in grid-stride order;
        // CUDA-core form: ~16 items per resident CTA, handed out by an atomic counter
        const int64_t target = 16LL * slots;
        const int64_t chunk = std::max<int64_t>(4, (work + target - 1) / target);  // pair tiles per item
        auto &items = pl.items_h[lev];
        for (int k = 0; k < P; ++k) {
            if (lev > levs[k]) continue;
            const int64_t nc = lev == 0 ? gt[k]->ncells : child_cap;
            const int64_t ptiles = align_up((size_t)pl.probs_h[k].n, kPairTile) / kPairTile;
            const int64_t nch = (ptiles + chunk - 1) / chunk;  // balanced: chunk sizes differ by <= 1 tile
            for (int64_t c0 = 0; c0 < nc; c0 += cells_per_item)
                for (int64_t q = 0; q < nch; ++q) {
                    VoteItem it;
                    it.prob = k;
                    it.cell_begin = (int32_t)c0;
                    it.pair_begin = (int32_t)(ptiles * q / nch * kPairTile);
                    it.pair_end = (int32_t)(ptiles * (q + 1) / nch * kPairTile);
                    items.push_back(it);
                }
        }
        if (tck) split_last_round(items, slots);
    }
    // top-K chunks per problem
    int64_t maxc = child_cap;
    for (int k = 0; k < P; ++k) maxc = std::max<int64_t>(maxc, gt[k]->ncells);
    pl.chunks_per_prob = (int)((maxc + kSelChunk - 1) / kSelChunk);

    // ---- workspace layout ----
    size_t off = 0;
    auto reserve = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t r = off;
        off += bytes;
        return r;
    };
    struct Slot { size_t off; };
    const size_t o_probs = reserve(sizeof(ProbRef) * P);
    const size_t o_lref = reserve(sizeof(LevelRef) * (size_t)P * S);
    std::vector<size_t> o_items(S);
    for (int lev = 0; lev < S; ++lev) o_items[lev] = reserve(sizeof(VoteItem) * std::max<size_t>(1, pl.items_h[lev].size()));
    const size_t o_in = reserve(sizeof(float) * (size_t)pl.in_floats * 2);
    const size_t o_p32 = reserve(sizeof(float4) * 3 * (size_t)pool);
    const size_t o_pr = reserve(sizeof(float4) * 2 * (size_t)pool);
    const size_t o_tcb = tck ? reserve((size_t)pool * tck * 2) : 0;
    const size_t o_p2x = tck ? 0 : reserve(sizeof(float4) * 5 * (size_t)(pool / 2));
    const size_t o_member = reserve((size_t)pool);
    const size_t o_tiles = reserve(sizeof(int2) * (size_t)(pool / kPairTile + 1));
    // zeroed region: counts, child counts, stats, nkept
    const size_t z0 = align_up(off, 256);
    int64_t counts0 = 0;
    std::vector<int64_t> c0off(P);
    for (int k = 0; k < P; ++k) {
        c0off[k] = counts0;
        counts0 += gt[k]->ncells;
    }
    const size_t o_counts0 = reserve(sizeof(int32_t) * (size_t)counts0);
    const size_t o_countsL = reserve(sizeof(int32_t) * (size_t)P * std::max(1, max_levels) * child_cap);
    const size_t o_nc = reserve(sizeof(int32_t) * (size_t)P * S);
    const size_t o_stats = reserve(sizeof(ProbStats) * P);
    const size_t o_nkept = reserve(sizeof(int32_t) * (size_t)P * S);
    const size_t o_err = reserve(sizeof(int) * 4);
    const size_t o_ictr = reserve(sizeof(int) * (size_t)S);  // per-level work-item counters (CUDA-core vote)
    const size_t o_ambcnt = reserve(sizeof(int) * 2 * (size_t)S);  // per level: FP64-queue length, full flag
    const size_t z1 = align_up(off, 256);
    // FP64 resolution queue: room for 8e-6 of the largest level's tests (uniform outliers put
    // 4e-6 of them within the band) + 64k; a full queue makes the vote decide the rest itself
    int64_t lev_tests = 0, tests_l0 = 0, pairs_all = 0;
    for (int k = 0; k < P; ++k) {
        tests_l0 += (int64_t)pl.probs_h[k].n * gt[k]->ncells;
        pairs_all += pl.probs_h[k].n;
    }
    lev_tests = std::max<int64_t>(tests_l0, pairs_all * (int64_t)child_cap);
    pl.amb_cap = (int)std::min<int64_t>((int64_t)1 << 25, (int64_t)(8e-6 * (double)lev_tests) + 65536);
    if (test_amb_cap >= 0) pl.amb_cap = test_amb_cap;
    const size_t o_amb = reserve(sizeof(Amb64) * (size_t)pl.amb_cap);
    const size_t o_kept = reserve(sizeof(int32_t) * (size_t)P * S * K);
    const size_t o_cand = reserve(sizeof(Cand) * ((size_t)P * pl.chunks_per_prob * K + (size_t)P * K));
    const size_t o_res = reserve(sizeof(rot_vote_result) * P);
    // fit: per-slice partial sums (11 doubles per 4096-pair slice) and slice offsets
    pl.slice_off_h.assign(P, 0);
    int64_t nsl = 0;
    for (int k = 0; k < P; ++k) {
        pl.slice_off_h[k] = nsl;
        nsl += fit_slices(pl.probs_h[k].n);
    }
    const size_t o_slice = reserve(sizeof(double) * 11 * (size_t)std::max<int64_t>(1, nsl));
    const size_t o_sloff = reserve(sizeof(int64_t) * P);
    // fit paths: one CTA per small problem; the large ones in whole-GPU passes
    // over the flat list of their slices
    pl.fit_list_h.clear();
    pl.fit_bsoff_h.assign(1, 0);
    for (int k = 0; k < P; ++k)
        if (pl.probs_h[k].n <= kFitSmallMax) pl.fit_list_h.push_back(k);
    pl.fit_nsmall = (int)pl.fit_list_h.size();
    for (int k = 0; k < P; ++k)
        if (pl.probs_h[k].n > kFitSmallMax) {
            pl.fit_list_h.push_back(k);
            pl.fit_bsoff_h.push_back(pl.fit_bsoff_h.back() + fit_slices(pl.probs_h[k].n));
        }
    const size_t o_flist = reserve(sizeof(int32_t) * P);
    const size_t o_bsoff = reserve(sizeof(int64_t) * (P + 1));
    const size_t o_fstate = reserve(sizeof(FitState) * P);
    const size_t o_fcnt = reserve(sizeof(int) * P);
    // child tables: P x max_levels x child_cap cells
    const size_t nchild = (size_t)P * std::max(1, max_levels) * child_cap;
    const size_t o_cq = reserve(sizeof(double4_32a) * nchild);
    const size_t o_cch = reserve(sizeof(double) * nchild);
    const size_t o_ctr = reserve(sizeof(double2) * nchild);
    const size_t o_cidx = reserve(sizeof(int64_t) * nchild);
    const size_t o_cm = reserve(sizeof(float4) * 3 * nchild);
    const size_t o_cR = reserve(sizeof(float4) * 3 * nchild);
    const size_t need = align_up(off, 256);
    int rc = w.ensure(need, *this);
    if (rc != ROT_VOTE_OK) return rc;
    char *B = (char *)w.base;
    pl.d_probs = (ProbRef *)(B + o_probs);
    pl.d_lref = (LevelRef *)(B + o_lref);
    pl.d_items.resize(S);
    for (int lev = 0; lev < S; ++lev) pl.d_items[lev] = (VoteItem *)(B + o_items[lev]);
    pl.d_in = (float *)(B + o_in);
    pl.pool.p32 = (float4 *)(B + o_p32);
    pl.pool.pr = (float4 *)(B + o_pr);
    pl.pool.tcb = tck ? (void *)(B + o_tcb) : nullptr;
    pl.pool.tc_k = tck;
    pl.pool.p2x = tck ? nullptr : (float4 *)(B + o_p2x);
    pl.d_member = (uint8_t *)(B + o_member);
    pl.d_tiles = (int2 *)(B + o_tiles);
    pl.zero_off = z0;
    pl.zero_bytes = z1 - z0;
    pl.d_counts0 = (int32_t *)(B + o_counts0);
    pl.d_countsL = (int32_t *)(B + o_countsL);
    pl.d_nc = (int32_t *)(B + o_nc);
    pl.d_stats = (ProbStats *)(B + o_stats);
    pl.d_nkept = (int32_t *)(B + o_nkept);
    pl.d_kept = (int32_t *)(B + o_kept);
    pl.d_cand = (Cand *)(B + o_cand);
    pl.d_res = (rot_vote_result *)(B + o_res);
    pl.d_slice = (double *)(B + o_slice);
    pl.d_sloff = (int64_t *)(B + o_sloff);
    pl.d_flist = (int32_t *)(B + o_flist);
    pl.d_bsoff = (int64_t *)(B + o_bsoff);
    pl.d_fstate = (FitState *)(B + o_fstate);
    pl.d_fcnt = (int *)(B + o_fcnt);
    pl.d_err = (int *)(B + o_err);
    pl.d_ictr = (int *)(B + o_ictr);
    pl.d_ambcnt = (int *)(B + o_ambcnt);
    pl.d_amb = (Amb64 *)(B + o_amb);

    // pair-prep tiles
    pl.tiles_h.clear();
    for (int k = 0; k < P; ++k) {
        const int64_t nt = align_up((size_t)pl.probs_h[k].n, kPairTile) / kPairTile;
        for (int64_t t = 0; t < nt; ++t) pl.tiles_h.push_back(make_int2(k, (int)t));
    }

    // inputs: device pointers as given, else staged into d_in
    pl.in_off.assign(P, 0);
    int64_t fo = 0;
    for (int k = 0; k < P; ++k) {
        const rot_vote_problem &q = p[sel[k]];
        ProbRef &r = pl.probs_h[k];
        if (all_dev) {
            r.a = q.a;
            r.b = q.b;
        } else {
            pl.in_off[k] = fo;
            r.a = pl.d_in + fo;
            r.b = pl.d_in + pl.in_floats + fo;
            fo += 3 * q.n;
        }
    }

    // level refs
    pl.lref_h.assign((size_t)P * S, LevelRef{});
    CellSoA ch;
    ch.q = (double4_32a *)(B + o_cq);
    ch.chord = (double *)(B + o_cch);
    ch.trig = (double2 *)(B + o_ctr);
    ch.idx = (int64_t *)(B + o_cidx);
    ch.m32 = (float4 *)(B + o_cm);
    ch.R32 = (float4 *)(B + o_cR);
    for (int k = 0; k < P; ++k) {
        for (int lev = 0; lev <= levs[k]; ++lev) {
            LevelRef &L = pl.lref_h[(size_t)k * S + lev];
            L.chart = cfg.chart;
            L.pad = 0;
            if (lev == 0) {
                L.cells = gt[k]->cells;
                L.ncells = gt[k]->ncells_dev;
                L.counts = pl.d_counts0 + c0off[k];
                L.cap = (int32_t)gt[k]->ncells;
                L.n_side = gridn[k];
            } else {
                const size_t base = ((size_t)k * std::max(1, max_levels) + (lev - 1)) * child_cap;
                L.cells.q = ch.q + base;
                L.cells.chord = ch.chord + base;
                L.cells.trig = ch.trig + base;
                L.cells.idx = ch.idx + base;
                L.cells.m32 = ch.m32 + 3 * base;
                L.cells.R32 = ch.R32 + 3 * base;
                L.ncells = pl.d_nc + (size_t)k * S + lev;
                L.counts = pl.d_countsL + base;
                L.cap = child_cap;
                L.n_side = gridn[k] << lev;
            }
        }
    }
    // signature: shapes only (sizes, levels, grids, precision, residency)
    std::string sig;
    sig.reserve(64 + 24 * P);
    char buf[96];
    snprintf(buf, sizeof buf, "%d|%d|%d|%d|%d|%d|", P, pl.prec, K, cfg.rank_mode, cfg.refit_iters, (int)all_dev);
    sig += buf;
    for (int k = 0; k < P; ++k) {
        snprintf(buf, sizeof buf, "%lld,%d,%d;", (long long)pl.probs_h[k].n, gridn[k], levs[k]);
        sig += buf;
    }
    pl.signature = sig;
    pl.shape_n.resize(P);
    pl.shape_gl.resize(P);
    for (int k = 0; k < P; ++k) {
        pl.shape_n[k] = pl.probs_h[k].n;
        pl.shape_gl[k] = ((int64_t)gridn[k] << 32) | levs[k];
    }
    pl.shape_dev = all_dev;
    pl.shape_amb_hook = test_amb_cap;
    pl.ws_base = w.base;
    pl.reused = false;
    return ROT_VOTE_OK;
}

// Uploads descriptors (one H2D copy of a packed host block) and inputs.
int Context::upload(Wave &w, const rot_vote_problem *p, const std::vector<int> &sel) {
    Plan &pl = w.plan;
    const int P = pl.nprob, S = pl.stride;
    // descriptor block: probs, lref, items, tiles -> contiguous in the workspace?  They are
    // separate ranges; pack them into one pinned staging block and copy each range.
    size_t hb = sizeof(ProbRef) * P + sizeof(LevelRef) * (size_t)P * S + sizeof(int2) * pl.tiles_h.size() +
                sizeof(int64_t) * P + sizeof(int32_t) * P + sizeof(int64_t) * (P + 1) + 16 * 9;
    for (int lev = 0; lev < S; ++lev) hb += sizeof(VoteItem) * pl.items_h[lev].size();
    int rc = w.ensure_pinned(hb + 4096);
    if (rc != ROT_VOTE_OK) return fail(rc, "pinned staging allocation failed");
    char *h = (char *)w.pinned;
    size_t o = 0;
    auto put = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        if (o + bytes > w.pinned_cap) return cudaErrorInvalidValue;  // staging sized above: never taken
        memcpy(h + o, src, bytes);
        cudaError_t e = cudaMemcpyAsync(dst, h + o, bytes, cudaMemcpyHostToDevice, w.stream);
        o += align_up(bytes, 16);
        return e;
    };
    cudaError_t e = put(pl.d_probs, pl.probs_h.data(), sizeof(ProbRef) * P);
    if (!pl.reused) {  // a reused plan's tables are already in the workspace
        if (e == cudaSuccess) e = put(pl.d_lref, pl.lref_h.data(), sizeof(LevelRef) * (size_t)P * S);
        for (int lev = 0; lev < S && e == cudaSuccess; ++lev)
            e = put(pl.d_items[lev], pl.items_h[lev].data(), sizeof(VoteItem) * pl.items_h[lev].size());
        if (e == cudaSuccess) e = put(pl.d_tiles, pl.tiles_h.data(), sizeof(int2) * pl.tiles_h.size());
        if (e == cudaSuccess) e = put(pl.d_sloff, pl.slice_off_h.data(), sizeof(int64_t) * pl.slice_off_h.size());
        if (e == cudaSuccess) e = put(pl.d_flist, pl.fit_list_h.data(), sizeof(int32_t) * pl.fit_list_h.size());
        if (e == cudaSuccess) e = put(pl.d_bsoff, pl.fit_bsoff_h.data(), sizeof(int64_t) * pl.fit_bsoff_h.size());
    }
    if (e != cudaSuccess) return cuda_fail(e, "uploading descriptors");
    if (!pl.inputs_on_device) {
        // host inputs: direct copies from pinned caller memory when few problems, else pack
        bool direct = P <= 64;
        for (int k = 0; k < P && direct; ++k) direct = pinned_kind(p[sel[k]].a) && pinned_kind(p[sel[k]].b);
        if (direct) {
            for (int k = 0; k < P && e == cudaSuccess; ++k) {
                const size_t bytes = sizeof(float) * 3 * p[sel[k]].n;
                e = cudaMemcpyAsync(pl.d_in + pl.in_off[k], p[sel[k]].a, bytes, cudaMemcpyHostToDevice, w.stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(pl.d_in + pl.in_floats + pl.in_off[k], p[sel[k]].b, bytes,
                                        cudaMemcpyHostToDevice, w.stream);
            }
        } else {
            const size_t bytes = sizeof(float) * 2 * pl.in_floats;
            rc = w.ensure_stage(bytes);
            if (rc != ROT_VOTE_OK) return fail(rc, "pinned input staging allocation failed");
            float *st = (float *)w.stage;
            for (int k = 0; k < P; ++k) {
                memcpy(st + pl.in_off[k], p[sel[k]].a, sizeof(float) * 3 * p[sel[k]].n);
                memcpy(st + pl.in_floats + pl.in_off[k], p[sel[k]].b, sizeof(float) * 3 * p[sel[k]].n);
            }
            e = cudaMemcpyAsync(pl.d_in, st, bytes, cudaMemcpyHostToDevice, w.stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "copying host inputs");
    }
    return ROT_VOTE_OK;
}

// Enqueues the device pipeline of the planned batch on w.stream.
int Context::enqueue_pipeline(Wave &w) {
    Plan &pl = w.plan;
    const int P = pl.nprob, S = pl.stride, K = pl.top_k;
    char *B = (char *)w.base;
    const bool profile = cfg.keep_trace >= 2 && &w == &main_wave;
    size_t nev = 0;
    if (profile) prof.clear();
    auto mark = [&](int kind, int level, int kernels) {  // event pair around the next stage's launches
        if (!profile) return;
        while (prof_ev.size() < nev + 2) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            prof_ev.push_back(ev);
        }
        cudaEventRecord(prof_ev[nev], w.stream);
        prof.push_back(rot_vote_stage{kind, level, 0.f, kernels});
        nev += 2;
    };
    auto done = [&]() {
        if (profile) cudaEventRecord(prof_ev[nev - 1], w.stream);
    };
    cudaError_t e = cudaMemsetAsync(B + pl.zero_off, 0, pl.zero_bytes, w.stream);
    mark(0, -1, 1);
    if (e == cudaSuccess)
        e = launch_pair_prep(pl.d_probs, pl.d_tiles, (int)pl.tiles_h.size(), pl.pool, pl.prec, pl.d_stats, w.stream);
    done();
    // coarse level: the cell-major vote and the two-phase top-K; refinement
    // levels (<= 8 top_k cells per problem): the pair-major vote and a one-block
    // top-K.  Each ranking step also writes the next level's children.
    for (int lev = 0; lev < S && e == cudaSuccess; ++lev) {
        mark(1, lev, 3);  // the vote and its FP64 resolution pass (two launches)
        if (lev == 0)
            e = launch_vote(w, lev, pl.variant);
        else
            e = launch_vote_small(pl.d_probs, pl.d_tiles, (int)pl.tiles_h.size(), pl.d_lref, S, lev, pl.pool,
                                  pl.d_stats, pl.amb(lev), w.stream);
        if (e == cudaSuccess)
            // the coarse level's queue holds millions of tests (1e6 pairs, 128^3): more blocks hide
            // the dependent loads of its FP64 evaluations; the refinement levels' queues are short
            e = launch_resolve64(pl.amb(lev), pl.d_probs, P, pl.d_lref, S, lev, pl.pool, pl.d_stats,
                                 (lev == 0 ? 16 : 4) * sm_count, w.stream);
        done();
        mark(2, lev, lev == 0 ? 2 : 1);
        if (e == cudaSuccess) {
            if (lev == 0)
                e = launch_topk(pl.d_probs, P, pl.d_lref, S, lev, K, cfg.rank_mode, 0, pl.d_cand,
                                pl.chunks_per_prob, pl.d_kept, pl.d_nkept, pl.d_stats, w.stream);
            else
                e = launch_select_small(pl.d_probs, P, pl.d_lref, S, lev, K, cfg.rank_mode, pl.d_kept, pl.d_nkept,
                                        pl.d_stats, w.stream);
        }
        done();
    }
    mark(4, -1, (pl.fit_nsmall > 0 ? 1 : 0) + (P > pl.fit_nsmall ? cfg.refit_iters + 1 : 0));
    if (e == cudaSuccess)
        e = launch_fit(pl.d_probs, pl.d_lref, S, pl.d_kept, K, cfg.refit_iters, pl.pool, pl.d_member, pl.d_slice,
                       pl.d_sloff, pl.d_flist, pl.fit_nsmall, pl.d_flist + pl.fit_nsmall, P - pl.fit_nsmall,
                       pl.d_bsoff, pl.fit_bsoff_h.back(), pl.d_fstate, pl.d_fcnt, sm_count, pl.d_stats, pl.d_res,
                       w.stream);
    done();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.results_h, pl.d_res, sizeof(rot_vote_result) * P, cudaMemcpyDeviceToHost, w.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.err_h, pl.d_err, sizeof(int), cudaMemcpyDeviceToHost, w.stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the pipeline");
    return ROT_VOTE_OK;
}

cudaError_t Context::launch_vote(Wave &w, int lev, int variant) {
    Plan &pl = w.plan;
    const int nit = (int)pl.items_h[lev].size();
    if (pl.pool.tc_k)
        return launch_vote_tc(pl.d_items[lev], nit, pl.d_probs, pl.d_lref, pl.stride, lev, pl.pool, pl.d_stats,
                              pl.prec, cfg.recheck_band, variant, pl.grid_blocks, pl.d_err, w.stall, pl.amb(lev),
                              w.stream);
    return launch_vote_simt(pl.d_items[lev], nit, pl.d_probs, pl.d_lref, pl.stride, lev, pl.pool, pl.d_stats, variant,
                            pl.grid_blocks, pl.d_ictr + lev, pl.amb(lev), w.stream);
}

// ---------------------------------------------------------------------------
// Autotuner: the vote's tile shape (CUDA-core form: cells per thread;
// tensor-core form: epilogue warpgroups) is chosen per shape class by timing
// every candidate on the level-0 vote of the first solve in that class.
// ---------------------------------------------------------------------------
static int ilog2_64(int64_t x) {
    int r = 0;
    while (x > 1) {
        x >>= 1;
        ++r;
    }
    return r;
}

std::string Context::tune_key(const Plan &pl) const {
    int64_t tests0 = 0;
    for (int k = 0; k < pl.nprob; ++k)
        tests0 += (int64_t)pl.probs_h[k].n * (pl.lref_h[(size_t)k * pl.stride].cap);
    char buf[96];
    snprintf(buf, sizeof buf, "sm%d:prec%d:tests2^%d:probs2^%d", sm_count, pl.prec, ilog2_64(tests0),
             ilog2_64(pl.nprob));
    return buf;
}

// CUDA-core form: cells per thread, +100 for the packed f32x2 kernel (+10 / +20: 5 / 6 CTAs per SM); tensor-core form: epilogue warpgroups, +10 for
// 16-column TMEM chunks, +100 for 128-pair MMA units (four accumulator stages)
static std::vector<int> candidates(int tc_k) {
    return tc_k ? std::vector<int>{2, 4, 12, 14, 102, 104, 112, 114} : std::vector<int>{124, 114, 104, 102, 4, 8};
}

// The tuned variant of the bucket nearest to `key` (same SM count and
// precision; distance in the two log2 size coordinates), or -1 if none.
int Context::nearest_tuned(const std::string &key) const {
    int sm = 0, prec = 0, te = 0, pe = 0;
    if (sscanf(key.c_str(), "sm%d:prec%d:tests2^%d:probs2^%d", &sm, &prec, &te, &pe) != 4) return -1;
    int best = -1, best_d = 1 << 30;
    for (const auto &kv : tuned) {
        int sm2 = 0, prec2 = 0, te2 = 0, pe2 = 0;
        if (sscanf(kv.first.c_str(), "sm%d:prec%d:tests2^%d:probs2^%d", &sm2, &prec2, &te2, &pe2) != 4) continue;
        if (sm2 != sm || prec2 != prec) continue;
        const int d = std::abs(te2 - te) + std::abs(pe2 - pe);
        if (d < best_d) {
            best_d = d;
            best = kv.second;
        }
    }
    return best;
}

int Context::choose_variant(Wave &w, bool serving) {
    Plan &pl = w.plan;
    const std::vector<int> cand = candidates(pl.pool.tc_k);
    pl.variant = cand[0];
    if (cfg.autotune < 0) return ROT_VOTE_OK;
    if (cfg.autotune >= 2) {  // a forced tile shape
        if (std::find(cand.begin(), cand.end(), cfg.autotune) == cand.end())
            return fail(ROT_VOTE_EINVAL, "autotune names a tile shape that does not exist for this precision");
        pl.variant = cfg.autotune;
        return ROT_VOTE_OK;
    }
    const std::string key = tune_key(pl);
    auto it = tuned.find(key);
    if (it != tuned.end()) {
        pl.variant = it->second;
        return ROT_VOTE_OK;
    }
    if (serving) {  // never stall the serving scheduler on a new size bucket once one is tuned
        const int near = nearest_tuned(key);
        if (near >= 0) {
            pl.variant = near;
            return ROT_VOTE_OK;
        }
    }
    char *B = (char *)w.base;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best = cand[0];
    for (int v : cand) {
        float tot = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaError_t e = cudaMemsetAsync(B + pl.zero_off, 0, pl.zero_bytes, w.stream);
            if (e == cudaSuccess)
                e = launch_pair_prep(pl.d_probs, pl.d_tiles, (int)pl.tiles_h.size(), pl.pool, pl.prec, pl.d_stats,
                                     w.stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, w.stream);
            if (e == cudaSuccess) e = launch_vote(w, 0, v);
            if (e == cudaSuccess) e = cudaEventRecord(e1, w.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(w.stream);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(e, "autotuning the vote");
            }
            if (rep > 0) tot += ms;
        }
        int err = 0;
        cudaMemcpy(&err, pl.d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (err) {  // a bounded device-side wait expired: report it, never choose silently
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(ROT_VOTE_ETIMEDOUT, "a bounded device-side wait gave up while autotuning the vote");
        }
        if (tot < best_ms) {
            best_ms = tot;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tuned[key] = best;
    pl.variant = best;
    save_tuning(key, best, best_ms / 2.f);
    return ROT_VOTE_OK;
}

void Context::load_tuning() {
    const char *path = getenv("ROT_VOTE_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[128];
    int v;
    float ms;
    while (fscanf(f, "%127s %d %f", key, &v, &ms) == 3) tuned[key] = v;
    fclose(f);
}

void Context::save_tuning(const std::string &key, int v, float ms) {
    const char *path = getenv("ROT_VOTE_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %.4f\n", key.c_str(), v, ms);
    fclose(f);
}

// Plans, uploads and launches a batch on wave w (asynchronous).
int Context::launch_batch(Wave &w, const rot_vote_problem *p, const std::vector<int> &sel, bool serving) {
    const std::string old_sig = w.plan.signature;
    const int old_variant = w.plan.variant;
    const bool had_graph = w.graph_exec != nullptr;
    int rc = plan_batch(w, p, sel);
    if (rc != ROT_VOTE_OK) return rc;
    rc = w.ensure_results(w.plan.nprob);
    if (rc != ROT_VOTE_OK) return fail(rc, "pinned result allocation failed");
    rc = upload(w, p, sel);
    if (rc != ROT_VOTE_OK) return rc;
    rc = choose_variant(w, serving);
    if (rc != ROT_VOTE_OK) return rc;
    w.stall = test_stall > 0 ? 1 : 0;
    if (test_stall > 0) --test_stall;
    if (w.plan.variant != old_variant) w.plan.signature += "|changed";
    cudaError_t e = cudaEventRecord(w.ev0, w.stream);
    if (e != cudaSuccess) return cuda_fail(e, "recording an event");
    const bool graphs = cfg.use_graphs > 0 && cfg.keep_trace < 2 && !w.stall;
    if (graphs) {
        if (!(had_graph && old_sig == w.plan.signature && w.graph_base == w.base)) {
            if (w.graph_exec) {
                cudaGraphExecDestroy(w.graph_exec);
                w.graph_exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(w.stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "beginning graph capture");
            rc = enqueue_pipeline(w);
            cudaError_t e2 = cudaStreamEndCapture(w.stream, &g);
            if (rc != ROT_VOTE_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e2 != cudaSuccess) return cuda_fail(e2, "ending graph capture");
            e = cudaGraphInstantiate(&w.graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                w.graph_exec = nullptr;
                return cuda_fail(e, "instantiating the graph");
            }
            w.graph_base = w.base;
        }
        e = cudaGraphLaunch(w.graph_exec, w.stream);
        if (e != cudaSuccess) return cuda_fail(e, "launching the graph");
    } else {
        rc = enqueue_pipeline(w);
        if (rc != ROT_VOTE_OK) return rc;
    }
    e = cudaEventRecord(w.ev1, w.stream);
    if (e != cudaSuccess) return cuda_fail(e, "recording an event");
    return ROT_VOTE_OK;
}

// Copies finished results of a batch into out[sel[k]].
int Context::collect(Wave &w, const std::vector<int> &sel, rot_vote_result *out) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w.ev0, w.ev1);
    if (*w.err_h != 0)
        return fail(ROT_VOTE_ETIMEDOUT, "a bounded device-side wait gave up (tensor-core pipeline)");
    for (int k = 0; k < w.plan.nprob; ++k) {
        out[sel[k]] = w.results_h[k];
        out[sel[k]].ms_gpu = ms;
    }
    return ROT_VOTE_OK;
}

// ---------------------------------------------------------------------------
// Wave (workspace + stream + pinned buffers)
// ---------------------------------------------------------------------------
int Wave::ensure(size_t bytes, Context &ctx) {
    if (bytes <= cap) return ROT_VOTE_OK;
    const size_t want = std::max(bytes, 2 * cap);  // geometric growth: few reallocations
    if (ctx.bytes_held - cap + want > ctx.budget) {
        if (ctx.bytes_held - cap + bytes > ctx.budget) {
            ctx.last_error = "workspace exceeds the device memory budget";
            return ROT_VOTE_ENOMEM;
        }
    }
    const size_t alloc = (ctx.bytes_held - cap + want > ctx.budget) ? bytes : want;
    cudaStreamSynchronize(stream);
    if (base) cudaFree(base);
    ctx.bytes_held -= cap;
    base = nullptr;
    cap = 0;
    plan.ws_base = nullptr;  // the plan's tables lived in the old workspace
    if (graph_exec) {
        cudaGraphExecDestroy(graph_exec);
        graph_exec = nullptr;
    }
    if (ctx.test_fail_alloc > 0 && --ctx.test_fail_alloc == 0) {
        ctx.last_error = "device allocation failed (injected)";
        return ROT_VOTE_ENOMEM;
    }
    if (cudaMalloc(&base, alloc) != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        ctx.last_error = "cudaMalloc of the workspace failed";
        return ROT_VOTE_ENOMEM;
    }
    cap = alloc;
    ctx.bytes_held += alloc;
    return ROT_VOTE_OK;
}

int Wave::ensure_pinned(size_t bytes) {
    if (bytes <= pinned_cap) return ROT_VOTE_OK;
    cudaStreamSynchronize(stream);
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
    pinned_cap = 0;
    if (cudaMallocHost(&pinned, bytes) != cudaSuccess) {
        cudaGetLastError();
        pinned = nullptr;
        return ROT_VOTE_ENOMEM;
    }
    pinned_cap = bytes;
    return ROT_VOTE_OK;
}

int Wave::ensure_stage(size_t bytes) {
    if (bytes <= stage_cap) return ROT_VOTE_OK;
    cudaStreamSynchronize(stream);
    if (stage) cudaFreeHost(stage);
    stage = nullptr;
    stage_cap = 0;
    if (cudaMallocHost(&stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        stage = nullptr;
        return ROT_VOTE_ENOMEM;
    }
    stage_cap = bytes;
    return ROT_VOTE_OK;
}

int Wave::ensure_results(int n) {
    if (n <= results_cap) return ROT_VOTE_OK;
    cudaStreamSynchronize(stream);
    if (results_h) cudaFreeHost(results_h);
    results_h = nullptr;
    results_cap = 0;
    if (cudaMallocHost((void **)&results_h, sizeof(rot_vote_result) * n) != cudaSuccess) {
        cudaGetLastError();
        return ROT_VOTE_ENOMEM;
    }
    results_cap = n;
    return ROT_VOTE_OK;
}

int Wave::init(cudaStream_t s, bool own) {
    stream = s;
    own_stream = own;
    if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) return ROT_VOTE_ECUDA;
    if (cudaMallocHost((void **)&err_h, sizeof(int) * 4) != cudaSuccess) return ROT_VOTE_ENOMEM;
    *err_h = 0;
    return ROT_VOTE_OK;
}

// Gives the workspace back (an idle wave only): the serving scheduler does this
// when a request does not fit the budget while every other wave is idle.
void Wave::free_workspace(Context &ctx) {
    if (!base) return;
    cudaStreamSynchronize(stream);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
    cudaFree(base);
    ctx.bytes_held -= cap;
    base = nullptr;
    cap = 0;
    plan.ws_base = nullptr;
}

void Wave::release(Context &ctx) {
    if (stream) cudaStreamSynchronize(stream);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
    if (base) {
        cudaFree(base);
        ctx.bytes_held -= cap;
    }
    base = nullptr;
    cap = 0;
    plan.ws_base = nullptr;
    if (pinned) cudaFreeHost(pinned);
    if (stage) cudaFreeHost(stage);
    if (results_h) cudaFreeHost(results_h);
    if (err_h) cudaFreeHost(err_h);
    pinned = stage = nullptr;
    results_h = nullptr;
    err_h = nullptr;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
}

// ---------------------------------------------------------------------------
// Blocking solve
// ---------------------------------------------------------------------------
int Context::solve(const rot_vote_problem *p, int n, rot_vote_result *out) {
    std::vector<int> sel;
    for (int k = 0; k < n; ++k) {
        memset(&out[k], 0, sizeof(rot_vote_result));
        std::string why;
        const int g = p[k].grid_n > 0 ? p[k].grid_n : cfg.grid_n;
        const int l = p[k].levels > 0 ? p[k].levels : (p[k].levels < 0 ? 0 : cfg.levels);
        if (check_problem(p[k], g, l, &why) != ROT_VOTE_OK) {
            out[k].status = ROT_VOTE_EINVAL;
            last_error = "problem " + std::to_string(k) + ": " + why;
            continue;
        }
        sel.push_back(k);
    }
    if (sel.empty()) return ROT_VOTE_OK;
    Wave &w = main_wave;
    int rc = launch_batch(w, p, sel);
    if (rc != ROT_VOTE_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(w.stream);
    if (e != cudaSuccess) return cuda_fail(e, "running the pipeline");
    trace_valid = cfg.keep_trace > 0;
    trace_sel = sel;
    if (cfg.keep_trace >= 2)
        for (size_t k = 0; k < prof.size(); ++k) cudaEventElapsedTime(&prof[k].ms, prof_ev[2 * k], prof_ev[2 * k + 1]);
    return collect(w, sel, out);
}

// ---------------------------------------------------------------------------
// Trace (tests / diagnostics)
// ---------------------------------------------------------------------------
int Context::level_trace(int problem, int level, int64_t *idx, int32_t *count, int64_t cap, int64_t *ncells,
                         int64_t *kept_idx, int32_t *nkept) {
    if (!trace_valid) return fail(ROT_VOTE_EINVAL, "no trace: create the context with keep_trace = 1 and solve");
    const Plan &pl = main_wave.plan;
    int k = -1;
    for (int j = 0; j < (int)trace_sel.size(); ++j)
        if (trace_sel[j] == problem) k = j;
    if (k < 0 || level < 0 || level > pl.probs_h[k].levels) return fail(ROT_VOTE_EINVAL, "trace index out of range");
    const LevelRef &L = pl.lref_h[(size_t)k * pl.stride + level];
    int32_t nc = 0;
    cudaError_t e = cudaMemcpy(&nc, L.ncells, sizeof(int32_t), cudaMemcpyDeviceToHost);
    const int64_t m = std::min<int64_t>(nc, cap);
    if (e == cudaSuccess && idx && m > 0) e = cudaMemcpy(idx, L.cells.idx, sizeof(int64_t) * m, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && count && m > 0) e = cudaMemcpy(count, L.counts, sizeof(int32_t) * m, cudaMemcpyDeviceToHost);
    int32_t nk = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&nk, pl.d_nkept + (size_t)k * pl.stride + level, sizeof(int32_t), cudaMemcpyDeviceToHost);
    std::vector<int32_t> kp(pl.top_k);
    if (e == cudaSuccess)
        e = cudaMemcpy(kp.data(), pl.d_kept + ((size_t)k * pl.stride + level) * pl.top_k, sizeof(int32_t) * pl.top_k,
                       cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && kept_idx)
        for (int r = 0; r < nk && e == cudaSuccess; ++r)
            e = cudaMemcpy(&kept_idx[r], L.cells.idx + kp[r], sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the trace");
    if (ncells) *ncells = nc;
    if (nkept) *nkept = nk;
    return ROT_VOTE_OK;
}

int Context::stage_times(rot_vote_stage *out, int cap, int *count) {
    if (cfg.keep_trace < 2) return fail(ROT_VOTE_EINVAL, "create the context with keep_trace = 2 to time stages");
    const int n = (int)prof.size();
    for (int k = 0; k < n && k < cap; ++k) out[k] = prof[k];
    if (count) *count = n;
    return ROT_VOTE_OK;
}

}  // namespace rv

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int rot_vote_create(const rot_vote_config *cfg_in, rot_vote_ctx **out) {
    if (!out) return ROT_VOTE_EINVAL;
    *out = nullptr;
    rot_vote_config c;
    memset(&c, 0, sizeof c);
    if (cfg_in) c = *cfg_in;
    if (c.grid_n == 0) c.grid_n = 32;
    if (c.top_k == 0) c.top_k = 16;
    if (c.refit_iters == 0) c.refit_iters = 8;
    if (c.refit_iters < 0) c.refit_iters = 0;
    if (c.device_mem_budget == 0) c.device_mem_budget = (size_t)16 << 30;
    if (c.max_inflight == 0) c.max_inflight = 256;
    if (c.use_graphs == 0) c.use_graphs = 1;
    if (c.autotune == 0) c.autotune = 1;
    if (c.grid_n < 2 || c.grid_n > 256 || (c.grid_n & (c.grid_n - 1)) || c.levels < 0 || c.levels > kMaxLevels ||
        c.top_k < 1 || c.top_k > kMaxTopK || c.precision < 0 || c.precision > ROT_PREC_BF16X2 || c.rank_mode < 0 ||
        c.rank_mode > 1 || c.max_inflight < 1 || !(c.recheck_band >= 0.f) || c.chart < 0 || c.chart > 1)
        return ROT_VOTE_EINVAL;
    Context *ctx = new (std::nothrow) Context();
    if (!ctx) return ROT_VOTE_ENOMEM;
    const int rc = ctx->init(c);
    if (rc != ROT_VOTE_OK) {
        delete ctx;
        return rc;
    }
    *out = reinterpret_cast<rot_vote_ctx *>(ctx);
    return ROT_VOTE_OK;
}

int rot_vote_solve(rot_vote_ctx *ctx, const rot_vote_problem *p, int n_problems, rot_vote_result *out) {
    if (!ctx || !p || !out || n_problems < 1) return ROT_VOTE_EINVAL;
    Context *c = reinterpret_cast<Context *>(ctx);
    std::lock_guard<std::mutex> g(c->launch_mu);
    return c->solve(p, n_problems, out);
}

int rot_vote_submit(rot_vote_ctx *ctx, const rot_vote_problem *p, uint64_t *ticket) {
    if (!ctx || !p || !ticket) return ROT_VOTE_EINVAL;
    return reinterpret_cast<Context *>(ctx)->submit(*p, ticket);
}

int rot_vote_poll(rot_vote_ctx *ctx, uint64_t ticket, rot_vote_result *out, int timeout_us) {
    if (!ctx || !out) return ROT_VOTE_EINVAL;
    return reinterpret_cast<Context *>(ctx)->poll(ticket, out, timeout_us);
}

int rot_vote_level_trace(rot_vote_ctx *ctx, int problem, int level, int64_t *idx, int32_t *count, int64_t cap,
                         int64_t *ncells, int64_t *kept_idx, int32_t *nkept) {
    if (!ctx) return ROT_VOTE_EINVAL;
    Context *c = reinterpret_cast<Context *>(ctx);
    std::lock_guard<std::mutex> g(c->launch_mu);
    return c->level_trace(problem, level, idx, count, cap, ncells, kept_idx, nkept);
}

int rot_vote_stage_times(rot_vote_ctx *ctx, rot_vote_stage *out, int cap, int *count) {
    if (!ctx || (!out && cap > 0)) return ROT_VOTE_EINVAL;
    Context *c = reinterpret_cast<Context *>(ctx);
    std::lock_guard<std::mutex> g(c->launch_mu);
    return c->stage_times(out, cap, count);
}

int rot_vote_serve_spans(rot_vote_ctx *ctx, rot_vote_batch_span *out, int cap, int *count) {
    if (!ctx || !count || (!out && cap > 0) || cap < 0) return ROT_VOTE_EINVAL;
    return reinterpret_cast<Context *>(ctx)->serve_spans(out, cap, count);
}

void rot_vote_destroy(rot_vote_ctx *ctx) {
    if (!ctx) return;
    Context *c = reinterpret_cast<Context *>(ctx);
    c->shutdown();
    delete c;
}

const char *rot_vote_last_error(const rot_vote_ctx *ctx) {
    if (!ctx) return "null context";
    return reinterpret_cast<const Context *>(ctx)->last_error.c_str();
}

}  // extern "C"
