// server.cpp -- simulation-job server with continuous batching (sim_server_* in sim.h).
//
// Jobs (netlist, instance count, seed, cycle budget) arrive at any time.  A
// server thread keeps one instance pool per netlist on the device (pool.hpp);
// a job is admitted when its pool has a free run of slots, creating the pool
// if the device-memory footprint of all pools stays under the cap.  Every
// pool is stepped on its own stream, by one persistent launch per step whose
// grid covers only the pool's instance groups in use (or, as configured, by
// per-cycle launches replayed from a graph), so pools of different netlists
// run concurrently on the GPU, and each step advances
// every job in the pool by the same number of cycles (never past the
// earliest-finishing job's budget).  A finished job's digests are read, its
// slots freed, and queued jobs take them at the next step boundary.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sim.h"
#include "pool.hpp"

namespace rtl {
int set_error(int code, const std::string& msg);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id;
    sim_job spec;
    int32_t state = SIM_JOB_QUEUED;
    uint64_t cycles_done = 0;
    double t_arrive = 0, t_start = 0, t_done = 0;
    uint32_t slot_lo = 0;
    std::vector<uint64_t> digests;
    std::string error;
};

struct Pool {
    sim_netlist* nl = nullptr;
    sim_batch* batch = nullptr;
    uint32_t capacity = 0;
    size_t bytes = 0;
    std::vector<uint64_t> slot_job;      // 0 = free
    std::vector<uint64_t> active;        // job ids
    bool inflight = false;
    uint64_t step_n = 0;
    cudaEvent_t done_ev = nullptr;
    double idle_since = 0;
    bool failed = false;
};

}  // namespace

struct sim_server {
    sim_server_config cfg{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    std::deque<uint64_t> queue;
    uint64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::vector<std::unique_ptr<Pool>> pools;   // owned by the worker thread
    size_t bytes_in_use = 0;
    // written by the worker, read by sim_server_stats on other threads
    std::atomic<uint64_t> instance_cycles{0};
    std::atomic<uint64_t> kernels{0};

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void run();
    bool try_admit(Job& j);
    void finish_step(Pool& p);
    void fail_pool_jobs(Pool& p, const std::string& msg);
    void drop_failed_pools();
};

namespace {

// First free run of n slots, or -1.
int64_t find_slots(const Pool& p, uint32_t n) {
    uint32_t run = 0;
    for (uint32_t s = 0; s < p.capacity; s++) {
        run = p.slot_job[s] ? 0 : run + 1;
        if (run == n) return int64_t(s + 1 - n);
    }
    return -1;
}

}  // namespace

bool sim_server::try_admit(Job& j) {
    // slots of a pool change only between its steps: wait while a pool of this
    // netlist is stepping, then take free slots in it or open another pool
    Pool* pool = nullptr;
    for (auto& p : pools) {
        if (p->nl != j.spec.netlist) continue;
        if (p->inflight) return false;
        if (find_slots(*p, j.spec.n_inst) >= 0) {
            pool = p.get();
            break;
        }
    }
    if (!pool) {
        uint32_t cap = std::max(cfg.pool_slots, j.spec.n_inst);
        size_t bytes = rtl::pool_footprint(j.spec.netlist, cap);
        if (bytes_in_use + bytes > cfg.hbm_cap_bytes) {
            // release idle pools (no jobs, no step in flight) to make room
            for (auto it = pools.begin(); it != pools.end() && bytes_in_use + bytes > cfg.hbm_cap_bytes;) {
                if ((*it)->active.empty() && !(*it)->inflight) {
                    bytes_in_use -= (*it)->bytes;
                    cudaEventDestroy((*it)->done_ev);
                    sim_batch_destroy((*it)->batch);
                    it = pools.erase(it);
                } else {
                    ++it;
                }
            }
            if (bytes_in_use + bytes > cfg.hbm_cap_bytes) return false;
        }
        std::unique_ptr<Pool> p(new Pool());
        p->nl = j.spec.netlist;
        p->capacity = cap;
        p->bytes = bytes;
        p->slot_job.assign(cap, 0);
        int rc = rtl::pool_create(j.spec.netlist, cap, cfg.persistent != 0, &p->batch);
        if (rc) {
            j.state = SIM_JOB_FAILED;
            j.error = sim_last_error();
            return true;
        }
        cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming);
        bytes_in_use += bytes;
        pool = p.get();
        pools.push_back(std::move(p));
    }
    int64_t lo = find_slots(*pool, j.spec.n_inst);
    if (lo < 0) return false;
    int rc = rtl::pool_admit(pool->batch, uint32_t(lo), j.spec.n_inst, j.spec.seed);
    if (rc) {
        j.state = SIM_JOB_FAILED;
        j.error = sim_last_error();
        return true;
    }
    for (uint32_t s = 0; s < j.spec.n_inst; s++) pool->slot_job[lo + s] = j.id;
    pool->active.push_back(j.id);
    j.slot_lo = uint32_t(lo);
    j.state = SIM_JOB_RUNNING;
    j.t_start = now();
    return true;
}

void sim_server::fail_pool_jobs(Pool& p, const std::string& msg) {
    std::lock_guard<std::mutex> g(mu);
    p.failed = true;
    for (uint64_t id : p.active) {
        Job& j = *jobs[id];
        j.state = SIM_JOB_FAILED;
        j.error = msg;
        j.t_done = now();
        for (uint32_t s = 0; s < j.spec.n_inst; s++) p.slot_job[j.slot_lo + s] = 0;
    }
    p.active.clear();
    cv.notify_all();
}

// A pool whose step failed holds state part-way through a cycle: its jobs
// have been failed, and the pool is released instead of taking new jobs.
void sim_server::drop_failed_pools() {
    for (auto it = pools.begin(); it != pools.end();) {
        Pool& p = **it;
        if (!p.failed) {
            ++it;
            continue;
        }
        cudaStreamSynchronize(rtl::pool_stream(p.batch));
        {
            std::lock_guard<std::mutex> g(mu);
            bytes_in_use -= p.bytes;
        }
        cudaEventDestroy(p.done_ev);
        sim_batch_destroy(p.batch);
        it = pools.erase(it);
    }
}

void sim_server::finish_step(Pool& p) {
    p.inflight = false;
    std::vector<uint64_t> still;
    for (uint64_t id : p.active) {
        Job* j;
        {
            std::lock_guard<std::mutex> g(mu);
            j = jobs[id].get();
            j->cycles_done += p.step_n;
        }
        instance_cycles += p.step_n * j->spec.n_inst;
        if (j->cycles_done < j->spec.n_cycles) {
            still.push_back(id);
            continue;
        }
        std::vector<uint64_t> d(j->spec.n_inst);
        int rc = rtl::pool_digests(p.batch, j->slot_lo, j->spec.n_inst, d.data());
        std::lock_guard<std::mutex> g(mu);
        if (rc) {
            j->state = SIM_JOB_FAILED;
            j->error = sim_last_error();
        } else {
            j->digests.swap(d);
            j->state = SIM_JOB_DONE;
        }
        j->t_done = now();
        for (uint32_t s = 0; s < j->spec.n_inst; s++) p.slot_job[j->slot_lo + s] = 0;
        cv.notify_all();
    }
    p.active.swap(still);
    if (p.active.empty()) p.idle_since = now();
}

void sim_server::run() {
    while (!stop.load()) {
        // admit queued jobs in arrival order (a job that does not fit yet does
        // not block later jobs of other netlists); job fields change under the lock
        {
            std::lock_guard<std::mutex> g(mu);
            std::deque<uint64_t> waiting;
            for (uint64_t id : queue) {
                Job& j = *jobs[id];
                if (!try_admit(j)) {
                    waiting.push_back(id);
                } else if (j.state == SIM_JOB_FAILED) {
                    j.t_done = now();
                    cv.notify_all();
                }
            }
            queue.swap(waiting);
        }
        // start a step on every idle pool with jobs; persistent steps of the
        // pools with jobs split the GPU between them
        bool any_inflight = false;
        uint32_t busy = 0;
        for (auto& pp : pools) busy += !pp->active.empty();
        for (auto& pp : pools) {
            Pool& p = *pp;
            if (!p.inflight && !p.active.empty()) {
                uint64_t n = cfg.chunk_cycles;
                uint32_t hi = 0;       // slots in use end here (first-fit keeps them at the front)
                {
                    std::lock_guard<std::mutex> g(mu);
                    for (uint64_t id : p.active) {
                        n = std::min(n, jobs[id]->spec.n_cycles - jobs[id]->cycles_done);
                        hi = std::max(hi, jobs[id]->slot_lo + jobs[id]->spec.n_inst);
                    }
                }
                uint64_t launched = 0;
                int rc = rtl::pool_set_active(p.batch, (hi + 31) / 32, busy);
                if (!rc) rc = rtl::pool_step(p.batch, n, &launched);
                if (!rc && cudaEventRecord(p.done_ev, rtl::pool_stream(p.batch)) != cudaSuccess) rc = SIM_ERR_CUDA;
                if (rc) {
                    fail_pool_jobs(p, sim_last_error());
                    continue;
                }
                p.step_n = n;
                p.inflight = true;
                kernels += launched;
            }
            any_inflight |= p.inflight;
        }
        // collect finished steps
        bool progressed = false;
        for (auto& pp : pools) {
            Pool& p = *pp;
            if (!p.inflight) continue;
            cudaError_t e = cudaEventQuery(p.done_ev);
            if (e == cudaErrorNotReady) continue;
            progressed = true;
            int rc = sim_sync(p.batch);     // surfaces launch or device errors
            if (e != cudaSuccess || rc) {
                p.inflight = false;
                fail_pool_jobs(p, rc ? sim_last_error() : cudaGetErrorString(e));
                continue;
            }
            finish_step(p);
        }
        drop_failed_pools();
        if (!progressed) {
            std::unique_lock<std::mutex> lk(mu);
            if (!any_inflight && queue.empty())
                cv.wait_for(lk, std::chrono::milliseconds(2));
            else if (!any_inflight)
                cv.wait_for(lk, std::chrono::microseconds(200));
            else
                lk.unlock(), std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    for (auto& p : pools) {
        cudaStreamSynchronize(rtl::pool_stream(p->batch));
        cudaEventDestroy(p->done_ev);
        sim_batch_destroy(p->batch);
    }
    pools.clear();
}

extern "C" {

void sim_server_config_default(sim_server_config* c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->struct_size = sizeof(sim_server_config);
    c->hbm_cap_bytes = 150ULL << 30;
    c->pool_slots = 1024;
    c->chunk_cycles = 1000;
    c->persistent = 1;
}

int sim_server_create(const sim_server_config* cfg, sim_server** out) {
    if (!out) return rtl::set_error(SIM_ERR_BADARG, "null argument");
    std::unique_ptr<sim_server> s(new sim_server());
    sim_server_config_default(&s->cfg);
    if (cfg) {
        if (cfg->struct_size != sizeof(sim_server_config))
            return rtl::set_error(SIM_ERR_BADARG, "sim_server_config.struct_size mismatch");
        s->cfg = *cfg;
    }
    if (!s->cfg.pool_slots || !s->cfg.chunk_cycles) return rtl::set_error(SIM_ERR_BADARG, "pool_slots and chunk_cycles must be > 0");
    int dev = 0;
    cudaGetDevice(&dev);
    s->t0 = Clock::now();
    sim_server* raw = s.get();
    s->worker = std::thread([raw, dev] {
        cudaSetDevice(dev);
        raw->run();
    });
    *out = s.release();
    return SIM_OK;
}

int sim_submit(sim_server* s, const sim_job* job, uint64_t* job_id) {
    if (!s || !job || !job_id || !job->netlist || job->n_inst == 0)
        return rtl::set_error(SIM_ERR_BADARG, "bad job");
    if (rtl::pool_footprint(job->netlist, std::max(job->n_inst, 32u)) > s->cfg.hbm_cap_bytes)
        return rtl::set_error(SIM_ERR_ADMISSION, "job needs more device memory than the server's cap");
    std::unique_ptr<Job> j(new Job());
    j->spec = *job;
    std::lock_guard<std::mutex> g(s->mu);
    j->id = s->next_id++;
    j->t_arrive = s->now();
    *job_id = j->id;
    if (job->n_cycles == 0) {
        j->state = SIM_JOB_DONE;
        j->t_start = j->t_done = j->t_arrive;
    } else {
        s->queue.push_back(j->id);
    }
    s->jobs[j->id] = std::move(j);
    s->cv.notify_all();
    return SIM_OK;
}

int sim_poll(sim_server* s, uint64_t job_id, sim_job_status* st) {
    if (!s || !st) return rtl::set_error(SIM_ERR_BADARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return rtl::set_error(SIM_ERR_BADARG, "unknown job");
    const Job& j = *it->second;
    memset(st, 0, sizeof *st);
    st->state = j.state;
    st->n_inst = j.spec.n_inst;
    st->cycles_done = j.cycles_done;
    st->t_arrive = j.t_arrive;
    st->t_start = j.t_start;
    st->t_done = j.t_done;
    if (j.state == SIM_JOB_FAILED) return rtl::set_error(SIM_ERR_STATE, "job failed: " + j.error);
    return SIM_OK;
}

int sim_job_digests(sim_server* s, uint64_t job_id, uint64_t* out) {
    if (!s || !out) return rtl::set_error(SIM_ERR_BADARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return rtl::set_error(SIM_ERR_BADARG, "unknown job");
    if (it->second->state != SIM_JOB_DONE) return rtl::set_error(SIM_ERR_STATE, "job is not done");
    std::copy(it->second->digests.begin(), it->second->digests.end(), out);
    return SIM_OK;
}

int sim_server_wait(sim_server* s, uint64_t job_id, uint32_t timeout_ms) {
    if (!s) return rtl::set_error(SIM_ERR_BADARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] {
        auto it = s->jobs.find(job_id);
        return it == s->jobs.end() || it->second->state >= SIM_JOB_DONE;
    };
    if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return rtl::set_error(SIM_ERR_TIMEOUT, "job not finished within the wait");
    return SIM_OK;
}

int sim_server_stats(sim_server* s, uint64_t* instance_cycles, uint64_t* kernels, uint64_t* bytes_in_use) {
    if (!s) return rtl::set_error(SIM_ERR_BADARG, "null server");
    std::lock_guard<std::mutex> g(s->mu);
    if (instance_cycles) *instance_cycles = s->instance_cycles.load();
    if (kernels) *kernels = s->kernels.load();
    if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
    return SIM_OK;
}

size_t sim_server_footprint(const sim_netlist* nl, uint32_t slots) {
    return nl ? rtl::pool_footprint(nl, slots) : 0;
}

void sim_server_destroy(sim_server* s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

}  // extern "C"
