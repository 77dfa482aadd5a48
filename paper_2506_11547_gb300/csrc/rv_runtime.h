// rv_runtime.h -- host-side context, waves and plans (internal).
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rot_vote.h"
#include "rv_internal.h"

namespace rv {

size_t align_up(size_t x, size_t a);
int check_problem(const rot_vote_problem &p, int grid_n, int levels, std::string *why);

struct GridTable {
    int n = 0;
    int64_t ncells = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    CellSoA cells{};
    int32_t *ncells_dev = nullptr;
};

// Host description and device layout of one planned batch.
struct Plan {
    std::string signature;
    int nprob = 0, prec = 0, top_k = 16, stride = 1, max_level = 0;
    int chunks_per_prob = 1, grid_blocks = 1;
    int variant = 0;  // vote tile shape: cells per thread (CUDA cores) or epilogue warpgroups (tensor cores)
    int64_t pool_pairs = 0, in_floats = 0;
    bool inputs_on_device = true;
    std::vector<ProbRef> probs_h;
    std::vector<LevelRef> lref_h;
    std::vector<std::vector<VoteItem>> items_h;
    std::vector<int2> tiles_h;
    std::vector<int64_t> in_off;
    std::vector<int64_t> slice_off_h;
    std::vector<int32_t> fit_list_h;  // fit order: small problems (one CTA each), then large (whole-GPU passes)
    int fit_nsmall = 0;
    std::vector<int64_t> fit_bsoff_h;  // first slice of each large problem in the flat slice list, + total
    // device pointers (inside the wave's workspace)
    ProbRef *d_probs = nullptr;
    LevelRef *d_lref = nullptr;
    std::vector<VoteItem *> d_items;
    float *d_in = nullptr;
    PairPool pool{};
    uint8_t *d_member = nullptr;
    int2 *d_tiles = nullptr;
    size_t zero_off = 0, zero_bytes = 0;
    int32_t *d_counts0 = nullptr, *d_countsL = nullptr, *d_nc = nullptr, *d_nkept = nullptr, *d_kept = nullptr;
    ProbStats *d_stats = nullptr;
    Cand *d_cand = nullptr;
    rot_vote_result *d_res = nullptr;
    double *d_slice = nullptr;
    int64_t *d_sloff = nullptr;
    int32_t *d_flist = nullptr;
    int64_t *d_bsoff = nullptr;
    FitState *d_fstate = nullptr;
    int *d_fcnt = nullptr;  // per large problem: slices of the current fit iteration written
    int *d_err = nullptr;
    int *d_ictr = nullptr;  // per-level work-item counters of the CUDA-core vote (zeroed per solve)
    Amb64 *d_amb = nullptr; // tests deferred to the FP64 resolution pass (reused level after level)
    int *d_ambcnt = nullptr;  // per level: queue length, then queue-full flag (zeroed per solve)
    int amb_cap = 0;
    // the shapes this layout was planned for: a batch with the same ones (sizes, grids, levels,
    // input residency, FP64-queue capacity hook) on the same workspace reuses the plan and
    // refreshes only the per-problem inputs
    std::vector<int64_t> shape_n;
    std::vector<int64_t> shape_gl;  // grid_n << 32 | levels, per problem
    bool shape_dev = true;
    int shape_amb_hook = -1;
    void *ws_base = nullptr;
    bool reused = false;  // this batch reused the plan: only the problem table is uploaded
    AmbQueue amb(int lev) const {
        AmbQueue q;
        q.q = d_amb;
        q.count = d_ambcnt + 2 * lev;
        q.ovf = d_ambcnt + 2 * lev + 1;
        q.cap = amb_cap;
        return q;
    }
};

class Context;

// A workspace + stream + pinned staging: one batch in flight at a time.
struct Wave {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *base = nullptr;
    size_t cap = 0;
    void *pinned = nullptr;
    size_t pinned_cap = 0;
    void *stage = nullptr;
    size_t stage_cap = 0;
    rot_vote_result *results_h = nullptr;
    int results_cap = 0;
    int *err_h = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    void *graph_base = nullptr;
    Plan plan;
    // serving bookkeeping
    bool busy = false;       // a batch is admitted to this wave (being launched, or in flight)
    bool launching = false;  // the scheduler is launching it with the context lock released
    int stall = 0;  // fault injection for this batch (see Context::test_stall)
    std::vector<uint64_t> tickets;
    std::vector<double> t_submit;

    int init(cudaStream_t s, bool own);
    int ensure(size_t bytes, Context &ctx);
    int ensure_pinned(size_t bytes);
    int ensure_stage(size_t bytes);
    int ensure_results(int n);
    void free_workspace(Context &ctx);
    void release(Context &ctx);
};

struct Pending {
    uint64_t ticket;
    rot_vote_problem prob;
    double t_submit;
};

class Context {
  public:
    rot_vote_config cfg{};
    int device = 0, sm_count = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, bytes_held = 0;
    std::unordered_map<std::string, int> tuned;  // autotuner choices per shape class
    int test_fail_alloc = 0;  // fault injection: the k-th workspace allocation fails (ROT_VOTE_TEST_FAIL_ALLOC=k)
    int test_stall = 0;       // fault injection: in the next k solves the tensor-core copies never arrive and
                              // device waits are bounded by 1 ms (ROT_VOTE_TEST_STALL=k)
    int test_amb_cap = -1;    // test hook: the FP64 queue holds k tests (ROT_VOTE_TEST_AMB_CAP=k), so that
                              // the recount of the cells it could not take is exercised
    // per-kernel profiling (keep_trace == 2)
    std::vector<cudaEvent_t> prof_ev;
    std::vector<rot_vote_stage> prof;
    std::string last_error;
    std::list<GridTable> grids;  // list: stable addresses
    Wave main_wave;
    bool trace_valid = false;
    std::vector<int> trace_sel;
    // Alg. 1 (rv_alg1.cu): header, angle tables, staged inputs and the accumulator
    void *a1_mem = nullptr;
    size_t a1_cap = 0;
    int a1_J = 0;            // J of the angle tables in a1_mem (0 = none)
    size_t a1_toff = 0;      // their offset
    bool a1_peaks_attr = false;  // dynamic shared memory of the peak kernel raised
    bool a1_wrapped = false;     // the last Alg. 1 problem had counter wraps: vote with the wrap record first
    int a1_clean_side = -1;      // n whose counter words outside the ball region are all zero (-1: not known)
    // rigid pose (rv_pose.cu): row counts and offsets, translation table, staged points, kept pairs
    void *ps_mem = nullptr;
    size_t ps_cap = 0;
    void *ps_hdr_h = nullptr;
    cudaEvent_t ps_ev[2] = {nullptr, nullptr};
    void *a1_hdr_h = nullptr;
    cudaEvent_t a1_ev[2] = {nullptr, nullptr};

    // Every launch, and the state launches share (workspaces, grid tables, tuning,
    // traces, last_error), is taken under launch_mu.  The serving state below is
    // guarded by mu, which is never held across a launch, so rot_vote_submit and
    // rot_vote_poll do not wait for the scheduler's launches.  No code holds both.
    std::mutex launch_mu;

    // serving
    std::mutex mu;          // guards everything below
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::vector<Wave> waves;
    std::unordered_map<uint64_t, rot_vote_result> done;
    uint64_t next_ticket = 1;
    int64_t inflight = 0;
    bool stop = false;
    std::thread sched;
    bool sched_started = false;
    cudaEvent_t serve_ref = nullptr;          // recorded when serving starts: the origin of batch spans
    std::vector<rot_vote_batch_span> spans;   // device-time span of every completed serving batch
    static constexpr size_t kMaxSpans = 1 << 16;

    int init(const rot_vote_config &c);
    void shutdown();
    int fail(int code, const std::string &msg);
    int cuda_fail(cudaError_t e, const char *what);
    int grid_table(int n, const GridTable **out);
    int tc_k_of(int prec) const;
    int plan_batch(Wave &w, const rot_vote_problem *p, const std::vector<int> &sel);
    int upload(Wave &w, const rot_vote_problem *p, const std::vector<int> &sel);
    int enqueue_pipeline(Wave &w);
    cudaError_t launch_vote(Wave &w, int lev, int variant);
    std::string tune_key(const Plan &pl) const;
    int choose_variant(Wave &w, bool serving);
    int nearest_tuned(const std::string &key) const;
    void load_tuning();
    void save_tuning(const std::string &key, int v, float ms);
    int launch_batch(Wave &w, const rot_vote_problem *p, const std::vector<int> &sel, bool serving = false);
    int collect(Wave &w, const std::vector<int> &sel, rot_vote_result *out);
    int solve(const rot_vote_problem *p, int n, rot_vote_result *out);
    int level_trace(int problem, int level, int64_t *idx, int32_t *count, int64_t cap, int64_t *ncells,
                    int64_t *kept_idx, int32_t *nkept);
    int stage_times(rot_vote_stage *out, int cap, int *count);
    int alg1(const rot_vote_alg1_problem *p, int n, rot_vote_alg1_result *out);
    void alg1_release();
    int pose(const rot_vote_pose_problem *p, int n, rot_vote_pose_result *out);
    int pose_ensure(size_t need);
    void pose_release();
    int submit(const rot_vote_problem &p, uint64_t *ticket);
    int poll(uint64_t ticket, rot_vote_result *out, int timeout_us);
    void sched_loop();
    int serve_spans(rot_vote_batch_span *out, int cap, int *count);
};

double now_s();

}  // namespace rv
