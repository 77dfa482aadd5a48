// rv_serve.cu -- context set-up and the serving scheduler (continuous batching).
//
// rot_vote_submit appends a problem to an admission queue.  A scheduler
// thread owns a few waves (workspace + stream each).  Whenever a wave is free
// and problems are waiting, it takes as many as the in-flight limit allows off
// the queue, plans them as one batch and launches it on that wave's stream
// without waiting for the other waves, so batches admitted at different times
// run concurrently on the device.  Admission is by device memory: a batch that
// does not fit the context's budget is halved; a single problem that does not
// fit while other waves hold memory goes back to the head of the queue until
// a wave completes, and fails (ENOMEM) only when it does not fit with every
// other wave idle and their workspaces given back.  Completion is detected by
// polling the wave's end event (never by spinning on the GPU); each result is
// moved to a completed map that rot_vote_poll reads.  The context lock is not
// held across launches (they run under the launch lock), so submit and poll
// never wait for the scheduler's launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "rv_runtime.h"

namespace rv {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static constexpr int kServeWaves = 4;
static constexpr int kQueueFactor = 8;  // admission queue holds max_inflight * this

int Context::init(const rot_vote_config &c) {
    cfg = c;
    budget = c.device_mem_budget;
    if (cudaGetDevice(&device) != cudaSuccess) return ROT_VOTE_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return ROT_VOTE_ECUDA;
    sm_count = prop.multiProcessorCount;
    if (prop.major >= 10) {
        const cudaError_t e = prepare_vote_tc();
        if (e != cudaSuccess) {
            last_error = std::string("setting tensor-core kernel attributes: ") + cudaGetErrorString(e);
            return ROT_VOTE_ECUDA;
        }
    }
    if (c.cuda_stream) {
        stream = (cudaStream_t)c.cuda_stream;
        own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return ROT_VOTE_ECUDA;
        own_stream = true;
    }
    if (main_wave.init(stream, false) != ROT_VOTE_OK) return ROT_VOTE_ECUDA;
    load_tuning();
    // fault-injection hooks for the failure tests (never set in normal use)
    if (const char *e = getenv("ROT_VOTE_TEST_FAIL_ALLOC")) test_fail_alloc = atoi(e);
    if (const char *e = getenv("ROT_VOTE_TEST_STALL")) test_stall = atoi(e);
    if (const char *e = getenv("ROT_VOTE_TEST_AMB_CAP")) test_amb_cap = atoi(e);
    return ROT_VOTE_OK;
}

void Context::shutdown() {
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv.notify_all();
    if (sched_started && sched.joinable()) sched.join();
    for (auto &w : waves) w.release(*this);
    waves.clear();
    if (serve_ref) cudaEventDestroy(serve_ref);
    serve_ref = nullptr;
    main_wave.release(*this);
    alg1_release();
    pose_release();
    for (auto ev : prof_ev) cudaEventDestroy(ev);
    prof_ev.clear();
    for (auto &g : grids)
        if (g.mem) cudaFree(g.mem);
    grids.clear();
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
}

int Context::submit(const rot_vote_problem &p, uint64_t *ticket) {
    std::string why;
    const int g = p.grid_n > 0 ? p.grid_n : cfg.grid_n;
    const int l = p.levels > 0 ? p.levels : (p.levels < 0 ? 0 : cfg.levels);
    int rc = ROT_VOTE_OK;
    {
        std::unique_lock<std::mutex> lk(mu);
        if (check_problem(p, g, l, &why) != ROT_VOTE_OK) {
            rc = ROT_VOTE_EINVAL;
        } else if ((int64_t)queue.size() >= (int64_t)cfg.max_inflight * kQueueFactor) {
            rc = ROT_VOTE_EAGAIN;
            why = "admission queue full";
        } else if (!sched_started) {
            waves.resize(kServeWaves);
            for (auto &w : waves) {
                cudaStream_t s;
                if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                    rc = ROT_VOTE_ECUDA;
                    why = "creating a serving stream";
                    break;
                }
                if (w.init(s, true) != ROT_VOTE_OK) {
                    rc = ROT_VOTE_ECUDA;
                    why = "initialising a serving wave";
                    break;
                }
            }
            if (rc == ROT_VOTE_OK &&
                (cudaEventCreate(&serve_ref) != cudaSuccess || cudaEventRecord(serve_ref, waves[0].stream) != cudaSuccess)) {
                rc = ROT_VOTE_ECUDA;
                why = "recording the serving start event";
            }
            if (rc == ROT_VOTE_OK) {
                stop = false;
                sched = std::thread([this] { sched_loop(); });
                sched_started = true;
            }
        }
        if (rc == ROT_VOTE_OK) {
            Pending pd;
            pd.ticket = next_ticket++;
            pd.prob = p;
            pd.t_submit = now_s();
            queue.push_back(pd);
            *ticket = pd.ticket;
        }
    }
    if (rc != ROT_VOTE_OK) {  // last_error is launch state: written under the launch lock
        std::lock_guard<std::mutex> g(launch_mu);
        return fail(rc, why);
    }
    cv.notify_all();
    return ROT_VOTE_OK;
}

int Context::poll(uint64_t ticket, rot_vote_result *out, int timeout_us) {
    std::unique_lock<std::mutex> lk(mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
    for (;;) {
        auto it = done.find(ticket);
        if (it != done.end()) {
            *out = it->second;
            done.erase(it);
            return ROT_VOTE_OK;
        }
        if (ticket == 0 || ticket >= next_ticket) return ROT_VOTE_ENOTFOUND;
        bool known = false;
        for (auto &q : queue)
            if (q.ticket == ticket) known = true;
        for (auto &w : waves)
            for (auto t : w.tickets)
                if (t == ticket) known = true;
        if (!known) return ROT_VOTE_ENOTFOUND;
        if (timeout_us <= 0 || std::chrono::steady_clock::now() >= deadline) return ROT_VOTE_PENDING;
        cv.wait_until(lk, deadline);
    }
}

// Scheduler: harvest finished waves, then admit and launch on free waves.
// Runs with mu held except around launches and result copies, which take
// launch_mu instead.
void Context::sched_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    bool mem_wait = false;  // the head problem did not fit while other waves held memory
    while (!stop) {
        bool progressed = false;
        // 1. harvest
        for (size_t wi = 0; wi < waves.size(); ++wi) {
            Wave &w = waves[wi];
            if (!w.busy || w.launching) continue;
            const cudaError_t q = cudaEventQuery(w.ev1);
            if (q == cudaErrorNotReady) continue;
            const size_t nb = w.tickets.size();
            std::vector<int> sel(nb);
            std::vector<rot_vote_result> res(nb);
            for (size_t k = 0; k < nb; ++k) sel[k] = (int)k;
            float t0 = 0.f, t1 = 0.f;
            lk.unlock();
            int rc;
            {
                std::lock_guard<std::mutex> g(launch_mu);
                rc = q == cudaSuccess ? collect(w, sel, res.data()) : cuda_fail(q, "serving batch");
                if (q == cudaSuccess) {
                    cudaEventElapsedTime(&t0, serve_ref, w.ev0);
                    cudaEventElapsedTime(&t1, serve_ref, w.ev1);
                }
            }
            lk.lock();
            const double t = now_s();
            for (size_t k = 0; k < nb; ++k) {
                rot_vote_result r = res[k];
                if (rc != ROT_VOTE_OK) {
                    memset(&r, 0, sizeof r);
                    r.status = rc;
                }
                r.latency_ms = (float)((t - w.t_submit[k]) * 1e3);
                done[w.tickets[k]] = r;
            }
            if (spans.size() >= kMaxSpans) spans.erase(spans.begin(), spans.begin() + kMaxSpans / 2);
            spans.push_back(rot_vote_batch_span{t0, t1, (int32_t)wi, (int32_t)nb});
            inflight -= (int64_t)nb;
            w.tickets.clear();
            w.t_submit.clear();
            w.busy = false;
            progressed = true;
            mem_wait = false;
        }
        if (progressed) cv.notify_all();
        // 2. admit onto free waves
        for (size_t wi = 0; wi < waves.size() && !mem_wait && !stop; ++wi) {
            Wave &w = waves[wi];
            if (w.busy || queue.empty()) continue;
            const int64_t room = (int64_t)cfg.max_inflight - inflight;
            if (room <= 0) break;
            int take = (int)std::min<int64_t>(room, (int64_t)queue.size());
            std::vector<Pending> batch(queue.begin(), queue.begin() + take);
            queue.erase(queue.begin(), queue.begin() + take);
            // reserved: its tickets stay visible to rot_vote_poll while it is launched
            w.busy = w.launching = true;
            w.tickets.clear();
            w.t_submit.clear();
            for (auto &b : batch) {
                w.tickets.push_back(b.ticket);
                w.t_submit.push_back(b.t_submit);
            }
            bool others_busy = false;
            for (size_t k = 0; k < waves.size(); ++k)
                if (k != wi && waves[k].busy) others_busy = true;
            lk.unlock();
            int rc = ROT_VOTE_ENOMEM;
            {
                std::lock_guard<std::mutex> g(launch_mu);
                auto try_launch = [&](int n) {
                    std::vector<rot_vote_problem> probs(n);
                    std::vector<int> sel(n);
                    for (int k = 0; k < n; ++k) {
                        probs[k] = batch[k].prob;
                        sel[k] = k;
                    }
                    const int saved_graphs = cfg.use_graphs;
                    cfg.use_graphs = -1;  // every serving batch has its own shape: launch directly
                    const int r = launch_batch(w, probs.data(), sel, true);
                    cfg.use_graphs = saved_graphs;
                    return r;
                };
                while (take > 0) {
                    rc = try_launch(take);
                    if (rc != ROT_VOTE_ENOMEM || take == 1) break;
                    take /= 2;  // memory-based admission: admit fewer and retry
                }
                if (rc == ROT_VOTE_ENOMEM && !others_busy) {
                    // every other wave is idle: give their workspaces back and try the head alone
                    for (size_t k = 0; k < waves.size(); ++k)
                        if (k != wi) waves[k].free_workspace(*this);
                    main_wave.free_workspace(*this);
                    take = 1;
                    rc = try_launch(1);
                }
            }
            lk.lock();
            w.launching = false;
            const int admitted = rc == ROT_VOTE_OK ? take : 0;
            if (rc != ROT_VOTE_OK && !(rc == ROT_VOTE_ENOMEM && others_busy)) {
                // the head problem cannot run at all: fail it so the queue moves on
                rot_vote_result r;
                memset(&r, 0, sizeof r);
                r.status = rc;
                r.latency_ms = (float)((now_s() - batch[0].t_submit) * 1e3);
                done[batch[0].ticket] = r;
                batch.erase(batch.begin());
                cv.notify_all();
                progressed = true;
            } else if (rc != ROT_VOTE_OK) {
                mem_wait = true;  // wait for a wave to complete and free memory
            }
            // the problems not admitted go back to the head of the queue, in order
            queue.insert(queue.begin(), batch.begin() + admitted, batch.end());
            if (admitted > 0) {
                w.tickets.resize(admitted);
                w.t_submit.resize(admitted);
                inflight += admitted;
                progressed = true;
            } else {
                w.tickets.clear();
                w.t_submit.clear();
                w.busy = false;
            }
        }
        if (!progressed) cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

int Context::serve_spans(rot_vote_batch_span *out, int cap, int *count) {
    std::lock_guard<std::mutex> lk(mu);
    const int n = (int)spans.size();
    for (int k = 0; k < n && k < cap; ++k) out[k] = spans[k];
    *count = n;
    return ROT_VOTE_OK;
}

}  // namespace rv
