// rv_serve.cu -- context set-up and the serving scheduler (continuous batching).
//
// rot_vote_submit appends a problem to an admission queue.  A scheduler
// thread owns a few waves (workspace + stream each).  Whenever a wave is free
// and problems are waiting, it admits as many as the in-flight limit and the
// device-memory budget allow, plans them as one batch and launches it on that
// wave's stream without waiting for the other waves, so batches admitted at
// different times run concurrently on the device.  Completion is detected by
// polling the wave's end event (never by spinning on the GPU); each result is
// moved to a completed map that rot_vote_poll reads.
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
    std::unique_lock<std::mutex> lk(mu);
    if (check_problem(p, g, l, &why) != ROT_VOTE_OK) return fail(ROT_VOTE_EINVAL, why);
    if ((int64_t)queue.size() >= (int64_t)cfg.max_inflight * kQueueFactor)
        return fail(ROT_VOTE_EAGAIN, "admission queue full");
    if (!sched_started) {
        waves.resize(kServeWaves);
        for (auto &w : waves) {
            cudaStream_t s;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
                return fail(ROT_VOTE_ECUDA, "creating a serving stream");
            if (w.init(s, true) != ROT_VOTE_OK) return fail(ROT_VOTE_ECUDA, "initialising a serving wave");
        }
        stop = false;
        sched = std::thread([this] { sched_loop(); });
        sched_started = true;
    }
    Pending pd;
    pd.ticket = next_ticket++;
    pd.prob = p;
    pd.t_submit = now_s();
    queue.push_back(pd);
    *ticket = pd.ticket;
    lk.unlock();
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
void Context::sched_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        bool progressed = false;
        // 1. harvest
        for (auto &w : waves) {
            if (!w.busy) continue;
            const cudaError_t q = cudaEventQuery(w.ev1);
            if (q == cudaErrorNotReady) continue;
            const double t = now_s();
            std::vector<int> sel(w.tickets.size());
            std::vector<rot_vote_result> res(w.tickets.size());
            for (size_t k = 0; k < sel.size(); ++k) sel[k] = (int)k;
            int rc = q == cudaSuccess ? collect(w, sel, res.data()) : cuda_fail(q, "serving batch");
            for (size_t k = 0; k < w.tickets.size(); ++k) {
                rot_vote_result r = res[k];
                if (rc != ROT_VOTE_OK) {
                    memset(&r, 0, sizeof r);
                    r.status = rc;
                }
                r.latency_ms = (float)((t - w.t_submit[k]) * 1e3);
                done[w.tickets[k]] = r;
            }
            inflight -= (int64_t)w.tickets.size();
            w.tickets.clear();
            w.t_submit.clear();
            w.busy = false;
            progressed = true;
        }
        if (progressed) cv.notify_all();
        // 2. admit onto free waves
        for (auto &w : waves) {
            if (w.busy || queue.empty()) continue;
            const int64_t room = (int64_t)cfg.max_inflight - inflight;
            if (room <= 0) break;
            int take = (int)std::min<int64_t>(room, (int64_t)queue.size());
            std::vector<rot_vote_problem> probs;
            std::vector<Pending> batch;
            int rc = ROT_VOTE_ENOMEM;
            while (take > 0) {
                batch.assign(queue.begin(), queue.begin() + take);
                probs.resize(take);
                for (int k = 0; k < take; ++k) probs[k] = batch[k].prob;
                std::vector<int> sel(take);
                for (int k = 0; k < take; ++k) sel[k] = k;
                const int saved_graphs = cfg.use_graphs;
                cfg.use_graphs = -1;  // every serving batch has its own shape: launch directly
                rc = launch_batch(w, probs.data(), sel, true);
                cfg.use_graphs = saved_graphs;
                if (rc != ROT_VOTE_ENOMEM) break;
                take /= 2;  // memory-based admission: admit fewer and retry
            }
            if (rc != ROT_VOTE_OK) {
                // the head problem cannot run at all: fail it so the queue moves on
                Pending head = queue.front();
                queue.pop_front();
                rot_vote_result r;
                memset(&r, 0, sizeof r);
                r.status = rc;
                r.latency_ms = (float)((now_s() - head.t_submit) * 1e3);
                done[head.ticket] = r;
                cv.notify_all();
                continue;
            }
            for (int k = 0; k < take; ++k) queue.pop_front();
            w.busy = true;
            w.tickets.clear();
            w.t_submit.clear();
            for (auto &b : batch) {
                w.tickets.push_back(b.ticket);
                w.t_submit.push_back(b.t_submit);
            }
            inflight += take;
            progressed = true;
        }
        if (!progressed) cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace rv
