// sfft_server.cu -- continuous batching of independent sparse FFTs behind sfft_submit / sfft_poll /
// sfft_wait (declared in include/sfft.h, "Serving").  Host code only: one dispatcher thread per server
// owns every CUDA call the server makes; submitting and waiting threads touch only the job table
// under the server's mutex.
//
// Job life: submitted (inbox) -> admission queue (FIFO; a host-memory signal waits there until its
// device copy fits in the memory budget, then its copy starts on the copy stream) -> ready queue of
// its parameter set -> a batch on an idle plan instance (sfft::execute_batch with a request table, so
// each job draws with its own seed and id) -> results copied to the job's host arrays -> done.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sfft_internal.h"

using namespace sfft;

namespace {

using Clock = std::chrono::steady_clock;

double micros(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// The parameter set a job belongs to: a field-by-field copy with the padding zeroed, compared bytewise.
struct ParamKey {
    unsigned char bytes[sizeof(sfft_params)];
    bool operator<(const ParamKey& o) const { return std::memcmp(bytes, o.bytes, sizeof bytes) < 0; }
};

ParamKey make_key(const sfft_params& p, sfft_params* canon) {
    sfft_params q;
    std::memset(&q, 0, sizeof q);
    q.n = p.n;
    q.k = p.k;
    q.mode = p.mode;
    q.precision = p.precision;
    q.delta = p.delta;
    q.alpha0 = p.alpha0;
    q.bins_per_k = p.bins_per_k;
    q.B_min = p.B_min;
    q.extra_rounds = p.extra_rounds;
    q.thr = p.thr;
    q.tau_dec = p.tau_dec;
    q.iso_tol = p.iso_tol;
    q.gmin = p.gmin;
    q.prune = p.prune;
    q.ref_lo = p.ref_lo;
    q.ref_hi = p.ref_hi;
    q.ref_tol = p.ref_tol;
    q.z_cap = p.z_cap;
    q.eps = p.eps;
    q.t_regions = p.t_regions;
    q.R_loc = p.R_loc;
    q.R_est = p.R_est;
    q.s = p.s;
    q.est_gmin = p.est_gmin;
    q.streams = p.streams;
    q.gain = p.gain;
    q.chunk_taps = p.chunk_taps;
    ParamKey k;
    std::memcpy(k.bytes, &q, sizeof q);
    if (canon) *canon = q;
    return k;
}

enum class JobState { Queued, Ready, Running, Done, Failed };

struct Job {
    uint64_t ticket = 0;
    sfft_params p{};
    ParamKey key{};
    sfft_job desc{};
    size_t x_bytes = 0;
    JobState state = JobState::Queued;
    sfft_status status = SFFT_OK;
    sfft_job_result res{};
    Clock::time_point t_submit, t_launch;
    void* d_stage = nullptr;       // device copy of a host-memory signal
    cudaEvent_t staged = nullptr;  // recorded on the copy stream after that copy
};

// One plan with its stream, completion event and output buffers: one batch in flight at a time.
struct Instance {
    sfft_plan plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Job*> jobs;        // slot r of the running batch
    ReqDesc* h_table = nullptr;    // page-locked request table (rewritten only while idle)
    uint32_t* h_idx = nullptr;     // page-locked copies of the outputs
    double* h_val = nullptr;
    uint32_t* h_count = nullptr;
    int32_t* h_flag = nullptr;
    uint32_t* d_idx = nullptr;
    double* d_val = nullptr;
    uint32_t* d_count = nullptr;
    int32_t* d_flag = nullptr;
    size_t bytes = 0;              // device bytes (plan + outputs)
    // general-mode plans: one CUDA graph per batch size, made on first use, that replays the whole
    // transform of the plan's request table into this instance's outputs (a general batch is tens of
    // launches; the dispatcher then issues one)
    std::map<uint32_t, sfft_graph> graphs;
};

struct ParamSet {
    sfft_params p{};
    std::vector<std::unique_ptr<Instance>> inst;
    std::deque<Job*> ready;
    uint64_t last_use = 0;
    uint32_t pending = 0;          // instances being built by the builder thread
    sfft_status build_error = SFFT_OK;  // why the set's first instance could not be built
};

// A plan instance the builder thread is asked for, and what it hands back.
struct BuildOrder {
    ParamKey key;
    sfft_params p;
    const sfft_plan_s* tables;     // an instance of the same set to copy the host tables from, or null
    size_t reserved;               // device bytes already counted for it (a copy's size is known)
};
struct BuildResult {
    ParamKey key;
    std::unique_ptr<Instance> inst;
    sfft_status status;
    size_t reserved;
};

void destroy_instance(Instance* in) {
    if (!in) return;
    for (auto& g : in->graphs) sfft_graph_destroy(g.second);
    in->graphs.clear();
    if (in->plan) sfft_plan_destroy(in->plan);
    if (in->stream) cudaStreamDestroy(in->stream);
    if (in->done) cudaEventDestroy(in->done);
    cudaFreeHost(in->h_table);
    cudaFreeHost(in->h_idx);
    cudaFreeHost(in->h_val);
    cudaFreeHost(in->h_count);
    cudaFreeHost(in->h_flag);
    cudaFree(in->d_idx);
    cudaFree(in->d_val);
    cudaFree(in->d_count);
    cudaFree(in->d_flag);
}

}  // namespace

struct sfft_server_s {
    int device = 0;
    sfft_server_config cfg{};
    std::thread thread;

    // shared with submitting / waiting threads (guarded by mu)
    std::mutex mu;
    std::condition_variable cv_work;  // wakes the dispatcher
    std::condition_variable cv_done;  // wakes waiters
    std::deque<Job*> inbox;
    std::unordered_map<uint64_t, Job*> jobs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    bool gpu_event = false;           // a batch finished (set from a stream callback)
    uint64_t submitted = 0, completed = 0, failed = 0, launches = 0, launched_jobs = 0, n_inst = 0;
    size_t bytes_in_use = 0, bytes_peak = 0;
    std::vector<double> latencies;
    std::thread builder;
    std::condition_variable cv_build;  // wakes the builder
    std::deque<BuildOrder> orders;
    std::vector<BuildResult> built;
    bool builder_stop = false;

    // dispatcher-only state
    std::deque<Job*> admit_q;
    std::map<ParamKey, std::unique_ptr<ParamSet>> sets;
    std::multimap<size_t, void*> free_bufs;  // cached staging buffers by size (counted in bytes_in_use)
    std::vector<cudaEvent_t> event_pool;
    cudaStream_t copy_stream = nullptr;
    uint64_t tick = 0;
    size_t held = 0;                         // dispatcher's count of device bytes held
};

namespace {

void account(sfft_server_s* S, long long delta) {
    S->held = (size_t)((long long)S->held + delta);
    std::lock_guard<std::mutex> lk(S->mu);
    S->bytes_in_use = S->held;
    S->bytes_peak = std::max(S->bytes_peak, S->held);
}

void CUDART_CB on_batch_done(void* arg) {
    auto* S = static_cast<sfft_server_s*>(arg);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->gpu_event = true;
    }
    S->cv_work.notify_one();
}

cudaEvent_t take_event(sfft_server_s* S) {
    if (!S->event_pool.empty()) {
        cudaEvent_t e = S->event_pool.back();
        S->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

bool set_idle(const ParamSet& ps) {
    if (!ps.ready.empty() || ps.pending) return false;
    for (const auto& in : ps.inst)
        if (in->busy) return false;
    return true;
}

void drop_set(sfft_server_s* S, std::map<ParamKey, std::unique_ptr<ParamSet>>::iterator it) {
    long long freed = 0;
    for (auto& in : it->second->inst) {
        freed += (long long)in->bytes;
        destroy_instance(in.get());
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->n_inst -= it->second->inst.size();
    }
    S->sets.erase(it);
    account(S, -freed);
}

// Frees cached buffers, then idle parameter sets (least recently used first), until `need` more bytes
// fit in the budget.  Returns whether they fit.
bool make_room(sfft_server_s* S, size_t need, const ParamKey* keep) {
    while (S->held + need > S->cfg.mem_budget && !S->free_bufs.empty()) {
        auto it = S->free_bufs.begin();
        cudaFree(it->second);
        const size_t b = it->first;
        S->free_bufs.erase(it);
        account(S, -(long long)b);
    }
    while (S->held + need > S->cfg.mem_budget) {
        auto victim = S->sets.end();
        for (auto it = S->sets.begin(); it != S->sets.end(); ++it) {
            if (keep && !(it->first < *keep) && !(*keep < it->first)) continue;
            if (it->second->inst.empty() || !set_idle(*it->second)) continue;
            if (victim == S->sets.end() || it->second->last_use < victim->second->last_use) victim = it;
        }
        if (victim == S->sets.end()) return false;
        drop_set(S, victim);
    }
    return true;
}

void* take_buffer(sfft_server_s* S, size_t bytes, const ParamKey& key) {
    auto it = S->free_bufs.find(bytes);
    if (it != S->free_bufs.end()) {
        void* p = it->second;
        S->free_bufs.erase(it);
        return p;
    }
    if (!make_room(S, bytes, &key)) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    account(S, (long long)bytes);
    return p;
}

void finish_jobs(sfft_server_s* S, const std::vector<Job*>& js) {
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Job* j : js) {
            if (j->status == SFFT_OK) {
                j->state = JobState::Done;
                j->res.latency_us = micros(j->t_submit, now);
                S->latencies.push_back(j->res.latency_us);
                ++S->completed;
            } else {
                j->state = JobState::Failed;
                ++S->failed;
            }
        }
    }
    S->cv_done.notify_all();
}

void release_stage(sfft_server_s* S, Job* j) {
    if (j->d_stage) {
        S->free_bufs.emplace(j->x_bytes, j->d_stage);
        j->d_stage = nullptr;
    }
    if (j->staged) {
        S->event_pool.push_back(j->staged);
        j->staged = nullptr;
    }
}

void fail_job(sfft_server_s* S, Job* j, sfft_status st) {
    release_stage(S, j);
    j->status = st;
    finish_jobs(S, {j});
}

// Builds a plan instance (builder thread; touches no server state).
std::unique_ptr<Instance> build_instance(const sfft_params& p, uint32_t mb, const sfft_plan_s* tables,
                                         sfft_status* err) {
    auto in = std::make_unique<Instance>();
    const uint32_t zc = p.z_cap;
    sfft_status st = plan_create(&p, mb, tables, &in->plan);
    if (st != SFFT_OK) {
        *err = st;
        return nullptr;
    }
    bool ok = cudaStreamCreateWithFlags(&in->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&in->done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost((void**)&in->h_table, (size_t)mb * sizeof(ReqDesc)) == cudaSuccess &&
              cudaMallocHost((void**)&in->h_idx, (size_t)mb * zc * 4) == cudaSuccess &&
              cudaMallocHost((void**)&in->h_val, (size_t)mb * zc * 16) == cudaSuccess &&
              cudaMallocHost((void**)&in->h_count, (size_t)mb * 4) == cudaSuccess &&
              cudaMallocHost((void**)&in->h_flag, (size_t)mb * 4) == cudaSuccess &&
              cudaMalloc((void**)&in->d_idx, (size_t)mb * zc * 4) == cudaSuccess &&
              cudaMalloc((void**)&in->d_val, (size_t)mb * zc * 16) == cudaSuccess &&
              cudaMalloc((void**)&in->d_count, (size_t)mb * 4) == cudaSuccess &&
              cudaMalloc((void**)&in->d_flag, (size_t)mb * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy_instance(in.get());
        *err = SFFT_ERR_OOM;
        return nullptr;
    }
    in->bytes = in->plan->dev_bytes + (size_t)mb * zc * 20 + (size_t)mb * 8;
    *err = SFFT_OK;
    return in;
}

// The builder thread: plans are built here so that the dispatcher keeps serving other parameter sets
// (building computes window tables on the host and synchronises the device).
void builder(sfft_server_s* S) {
    cudaSetDevice(S->device);
    for (;;) {
        BuildOrder o;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_build.wait(lk, [&] { return S->builder_stop || !S->orders.empty(); });
            if (S->orders.empty()) return;
            o = S->orders.front();
            S->orders.pop_front();
        }
        sfft_status err = SFFT_OK;
        std::unique_ptr<Instance> in = build_instance(o.p, S->cfg.max_batch, o.tables, &err);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->built.push_back(BuildResult{o.key, std::move(in), err, o.reserved});
        }
        S->cv_work.notify_one();
    }
}

// Dispatcher: attach finished builds to their sets; a set whose first build failed fails its jobs.
void collect_builds(sfft_server_s* S) {
    std::vector<BuildResult> got;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        got.swap(S->built);
    }
    for (BuildResult& b : got) {
        auto it = S->sets.find(b.key);
        if (it == S->sets.end()) {  // cannot happen: a set with a pending build is never dropped
            if (b.inst) destroy_instance(b.inst.get());
            account(S, -(long long)b.reserved);
            continue;
        }
        ParamSet& ps = *it->second;
        --ps.pending;
        account(S, (b.inst ? (long long)b.inst->bytes : 0) - (long long)b.reserved);
        if (b.inst) {
            {
                std::lock_guard<std::mutex> lk(S->mu);
                ++S->n_inst;
            }
            ps.inst.push_back(std::move(b.inst));
        } else if (ps.inst.empty() && ps.pending == 0) {
            ps.build_error = b.status;
            while (!ps.ready.empty()) {
                Job* j = ps.ready.front();
                ps.ready.pop_front();
                fail_job(S, j, b.status);
            }
        }
    }
}

// Orders one more instance of a set.  The first instance of a set is always built (the set cannot run
// without it; its size is counted once known); a further one only if a copy of the first fits in the
// budget, and its size is reserved at once.
void order_build(sfft_server_s* S, const ParamKey& key, ParamSet& ps) {
    size_t reserve = 0;
    if (!ps.inst.empty()) {
        reserve = ps.inst.front()->bytes;
        if (!make_room(S, reserve, &key)) return;
        account(S, (long long)reserve);
    }
    ++ps.pending;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->orders.push_back(BuildOrder{key, ps.p, ps.inst.empty() ? nullptr : ps.inst.front()->plan, reserve});
    }
    S->cv_build.notify_one();
}

// 1. completed batches: results to the jobs' host arrays, staging memory back to the cache
void reap(sfft_server_s* S) {
    for (auto& kv : S->sets) {
        ParamSet& ps = *kv.second;
        const uint32_t zc = ps.p.z_cap;
        for (auto& inp : ps.inst) {
            Instance* in = inp.get();
            if (!in->busy) continue;
            const cudaError_t q = cudaEventQuery(in->done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) set_last_error(std::string("server batch: ") + cudaGetErrorString(q));
            in->busy = false;
            for (size_t r = 0; r < in->jobs.size(); ++r) {
                Job* j = in->jobs[r];
                if (q != cudaSuccess) {
                    j->status = SFFT_ERR_CUDA;
                } else {
                    const uint32_t cnt = in->h_count[r];
                    const uint32_t m = std::min(cnt, j->desc.cap);
                    std::memcpy(j->desc.h_idx, in->h_idx + r * zc, (size_t)m * 4);
                    std::memcpy(j->desc.h_val, in->h_val + 2 * r * zc, (size_t)m * 16);
                    j->res.count = m;
                    j->res.flag = cnt > j->desc.cap ? (int32_t)SFFT_ERR_CAPACITY : in->h_flag[r];
                    j->res.queued_us = micros(j->t_submit, j->t_launch);
                }
                release_stage(S, j);
            }
            std::vector<Job*> js;
            js.swap(in->jobs);
            finish_jobs(S, js);
        }
    }
}

// 2. admission in submission order: parameter sets are created on first use; a host-memory signal
// needs its device copy to fit in the budget (the head of the queue waits, so large jobs are not
// starved by later small ones)
void admit(sfft_server_s* S) {
    while (!S->admit_q.empty()) {
        Job* j = S->admit_q.front();
        auto it = S->sets.find(j->key);
        if (it == S->sets.end()) {
            auto ps = std::make_unique<ParamSet>();
            ps->p = j->p;
            it = S->sets.emplace(j->key, std::move(ps)).first;
            // keep at most max_plans parameter sets with resident plans
            size_t resident = 0;
            for (auto& kv : S->sets) resident += kv.second->inst.empty() ? 0 : 1;
            while (resident >= S->cfg.max_plans) {
                auto victim = S->sets.end();
                for (auto v = S->sets.begin(); v != S->sets.end(); ++v)
                    if (v != it && !v->second->inst.empty() && set_idle(*v->second) &&
                        (victim == S->sets.end() || v->second->last_use < victim->second->last_use))
                        victim = v;
                if (victim == S->sets.end()) break;
                drop_set(S, victim);
                --resident;
            }
        }
        ParamSet& ps = *it->second;
        if (ps.inst.empty()) {
            if (ps.pending == 0 && ps.build_error != SFFT_OK) {  // the set cannot be built
                S->admit_q.pop_front();
                fail_job(S, j, ps.build_error);
                continue;
            }
            if (ps.pending == 0) order_build(S, it->first, ps);
            // a host signal is staged only once its set's plan exists and is counted in the budget
            if (!j->desc.x_on_device) break;
        }
        if (!j->desc.x_on_device) {
            void* buf = take_buffer(S, j->x_bytes, j->key);
            if (!buf) {
                bool progress = false;  // memory comes back only if something runs or is queued to run
                for (auto& kv : S->sets) progress = progress || !set_idle(*kv.second);
                if (progress) break;
                S->admit_q.pop_front();
                fail_job(S, j, SFFT_ERR_OOM);
                continue;
            }
            j->d_stage = buf;
            j->staged = take_event(S);
            if (!j->staged ||
                cudaMemcpyAsync(buf, j->desc.x, j->x_bytes, cudaMemcpyHostToDevice, S->copy_stream) != cudaSuccess ||
                cudaEventRecord(j->staged, S->copy_stream) != cudaSuccess) {
                set_last_error("server: staging copy failed");
                S->admit_q.pop_front();
                fail_job(S, j, SFFT_ERR_CUDA);
                continue;
            }
        }
        S->admit_q.pop_front();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            j->state = JobState::Ready;
        }
        it->second->ready.push_back(j);
    }
}

// 3. one batch per idle (or new) instance of every parameter set with ready jobs
void launch(sfft_server_s* S) {
    for (auto& kv : S->sets) {
        ParamSet& ps = *kv.second;
        while (!ps.ready.empty()) {
            Instance* in = nullptr;
            for (auto& c : ps.inst)
                if (!c->busy) {
                    in = c.get();
                    break;
                }
            if (!in) {
                // all instances busy (or none yet): ask for one more, and serve the other sets meanwhile
                if (ps.inst.size() + ps.pending < S->cfg.instances) order_build(S, kv.first, ps);
                break;
            }
            const uint32_t batch = (uint32_t)std::min<size_t>(ps.ready.size(), S->cfg.max_batch);
            in->jobs.assign(ps.ready.begin(), ps.ready.begin() + batch);
            ps.ready.erase(ps.ready.begin(), ps.ready.begin() + batch);
            ps.last_use = ++S->tick;
            const Clock::time_point now = Clock::now();
            cudaError_t e = cudaSuccess;
            for (uint32_t r = 0; r < batch; ++r) {
                Job* j = in->jobs[r];
                j->t_launch = now;
                in->h_table[r].x = j->d_stage ? j->d_stage : j->desc.x;
                in->h_table[r].seed = j->desc.seed;
                in->h_table[r].id = j->desc.id;
                in->h_table[r].period = j->desc.period;
                if (j->staged && e == cudaSuccess) e = cudaStreamWaitEvent(in->stream, j->staged, 0);
            }
            const uint32_t zc = ps.p.z_cap;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(in->plan->d_reqs, in->h_table, (size_t)batch * sizeof(ReqDesc),
                                    cudaMemcpyHostToDevice, in->stream);
            sfft_status st = e == cudaSuccess ? SFFT_OK : SFFT_ERR_CUDA;
            sfft_graph g = nullptr;
            if (st == SFFT_OK && ps.p.mode == SFFT_GENERAL) {
                auto it = in->graphs.find(batch);
                if (it != in->graphs.end()) {
                    g = it->second;
                } else if (sfft_graph_create(in->plan, nullptr, batch, 0, in->d_idx, in->d_val, zc, in->d_count,
                                             in->d_flag, &g) == SFFT_OK) {
                    in->graphs[batch] = g;
                } else {
                    g = nullptr;  // run it as plain launches
                }
            }
            if (st == SFFT_OK && g)
                st = sfft_graph_launch(g, in->stream);
            else if (st == SFFT_OK)
                st = execute_batch(in->plan, nullptr, in->plan->d_reqs, batch, 0, in->stream, in->d_idx, in->d_val,
                                   zc, in->d_count, in->d_flag);
            if (st == SFFT_OK) {
                e = cudaMemcpyAsync(in->h_count, in->d_count, (size_t)batch * 4, cudaMemcpyDeviceToHost, in->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(in->h_flag, in->d_flag, (size_t)batch * 4, cudaMemcpyDeviceToHost, in->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(in->h_idx, in->d_idx, (size_t)batch * zc * 4, cudaMemcpyDeviceToHost,
                                        in->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(in->h_val, in->d_val, (size_t)batch * zc * 16, cudaMemcpyDeviceToHost,
                                        in->stream);
                // the callback only wakes the dispatcher; `done` is recorded after it, so a completed
                // event also means the callback has returned (nothing touches the server later)
                if (e == cudaSuccess) e = cudaLaunchHostFunc(in->stream, on_batch_done, S);
                if (e == cudaSuccess) e = cudaEventRecord(in->done, in->stream);
                if (e != cudaSuccess) {
                    set_last_error(std::string("server launch: ") + cudaGetErrorString(e));
                    st = SFFT_ERR_CUDA;
                }
            }
            if (st != SFFT_OK) {
                std::vector<Job*> js;
                js.swap(in->jobs);
                for (Job* j : js) {
                    release_stage(S, j);
                    j->status = st;
                }
                finish_jobs(S, js);
                continue;
            }
            in->busy = true;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (Job* j : in->jobs) j->state = JobState::Running;
                ++S->launches;
                S->launched_jobs += batch;
            }
        }
    }
}

bool any_busy(const sfft_server_s* S) {
    for (const auto& kv : S->sets)
        for (const auto& in : kv.second->inst)
            if (in->busy) return true;
    return false;
}

bool any_ready(const sfft_server_s* S) {
    for (const auto& kv : S->sets)
        if (!kv.second->ready.empty()) return true;
    return false;
}

bool any_pending(const sfft_server_s* S) {
    for (const auto& kv : S->sets)
        if (kv.second->pending) return true;
    return false;
}

void dispatcher(sfft_server_s* S) {
    cudaSetDevice(S->device);
    bool stop = false;
    for (;;) {
        std::vector<Job*> fresh;
        const bool busy = any_busy(S) || any_ready(S) || !S->admit_q.empty();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto wake = [&] {
                return !S->inbox.empty() || (S->stopping && !stop) || S->gpu_event || !S->built.empty();
            };
            if (!wake()) {
                if (busy)
                    S->cv_work.wait_for(lk, std::chrono::microseconds(200), wake);
                else
                    S->cv_work.wait(lk, wake);
            }
            fresh.assign(S->inbox.begin(), S->inbox.end());
            S->inbox.clear();
            S->gpu_event = false;
            stop = S->stopping;
        }
        for (Job* j : fresh) S->admit_q.push_back(j);
        collect_builds(S);
        reap(S);
        admit(S);
        launch(S);
        if (stop && S->admit_q.empty() && !any_busy(S) && !any_ready(S) && !any_pending(S)) {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->inbox.empty()) break;
        }
    }
}

}  // namespace

extern "C" {

sfft_status sfft_server_create(const sfft_server_config* cfg, sfft_server* out) {
    if (!out) return SFFT_ERR_INVALID_ARG;
    *out = nullptr;
    sfft_server_config c{};
    if (cfg) c = *cfg;
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.instances == 0) c.instances = 2;
    if (c.max_plans == 0) c.max_plans = 16;
    if (c.max_batch > 4096 || c.instances > 16) return SFFT_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("server: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return SFFT_ERR_CUDA;
    }
    if (c.mem_budget == 0) {
        size_t free_b = 0, total_b = 0;
        e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) {
            set_last_error(std::string("server: ") + cudaGetErrorString(e));
            cudaGetLastError();
            return SFFT_ERR_CUDA;
        }
        c.mem_budget = free_b / 2;
    }
    auto* S = new (std::nothrow) sfft_server_s();
    if (!S) return SFFT_ERR_OOM;
    S->device = dev;
    S->cfg = c;
    if ((e = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        set_last_error(std::string("server: ") + cudaGetErrorString(e));
        delete S;
        return SFFT_ERR_CUDA;
    }
    try {
        S->builder = std::thread(builder, S);
        S->thread = std::thread(dispatcher, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->builder_stop = true;
        }
        S->cv_build.notify_one();
        if (S->builder.joinable()) S->builder.join();
        cudaStreamDestroy(S->copy_stream);
        delete S;
        return SFFT_ERR_OOM;
    }
    *out = S;
    return SFFT_OK;
}

sfft_status sfft_server_destroy(sfft_server S) {
    if (!S) return SFFT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_one();
    if (S->thread.joinable()) S->thread.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->builder_stop = true;
    }
    S->cv_build.notify_one();
    if (S->builder.joinable()) S->builder.join();
    cudaSetDevice(S->device);
    for (BuildResult& b : S->built)
        if (b.inst) destroy_instance(b.inst.get());
    while (!S->sets.empty()) drop_set(S, S->sets.begin());
    for (auto& kv : S->free_bufs) cudaFree(kv.second);
    for (cudaEvent_t ev : S->event_pool) cudaEventDestroy(ev);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    for (auto& kv : S->jobs) delete kv.second;
    delete S;
    return SFFT_OK;
}

// A checked job of validated params p, ready to queue (nullptr and *st set on an error)
static Job* make_job(const sfft_server_s* S, const sfft_params* p, const sfft_job* job, sfft_status* st) {
    *st = SFFT_ERR_INVALID_ARG;
    if (!job->x || !job->h_idx || !job->h_val || job->cap == 0) return nullptr;
    const size_t elem = p->precision == SFFT_FP64 ? 16 : 8;
    if (job->x_on_device && ((uintptr_t)job->x % elem) != 0) return nullptr;
    if (job->period != 0 && ((job->period & (job->period - 1)) != 0 || job->period > p->n)) return nullptr;
    const size_t x_bytes = (size_t)(job->period ? job->period : p->n) * elem;
    if (!job->x_on_device && x_bytes > S->cfg.mem_budget) {
        *st = SFFT_ERR_OOM;
        return nullptr;
    }
    auto* j = new (std::nothrow) Job();
    if (!j) {
        *st = SFFT_ERR_OOM;
        return nullptr;
    }
    j->key = make_key(*p, &j->p);
    j->desc = *job;
    j->x_bytes = x_bytes;
    *st = SFFT_OK;
    return j;
}

// Queue checked jobs in order under one lock, one wake-up (BUSY, nothing queued: the server stops)
static sfft_status queue_jobs(sfft_server_s* S, Job* const* js, uint32_t count, uint64_t* tickets) {
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) return SFFT_ERR_BUSY;
        for (uint32_t i = 0; i < count; ++i) {
            Job* j = js[i];
            j->t_submit = now;
            j->ticket = S->next_ticket++;
            S->jobs.emplace(j->ticket, j);
            S->inbox.push_back(j);
            ++S->submitted;
            tickets[i] = j->ticket;
        }
    }
    S->cv_work.notify_one();
    return SFFT_OK;
}

sfft_status sfft_submit(sfft_server S, const sfft_params* p, const sfft_job* job, uint64_t* ticket) {
    if (!S || !p || !job || !ticket) return SFFT_ERR_INVALID_ARG;
    const sfft_status v = validate_params(p);
    if (v != SFFT_OK) return v;
    sfft_status st;
    Job* j = make_job(S, p, job, &st);
    if (!j) return st;
    if ((st = queue_jobs(S, &j, 1, ticket)) != SFFT_OK) delete j;
    return st;
}

sfft_status sfft_submit_many(sfft_server S, const sfft_params* p, const sfft_job* jobs, uint32_t count,
                             uint64_t* tickets) {
    if (!S || !p || !jobs || !tickets || count == 0) return SFFT_ERR_INVALID_ARG;
    const sfft_status v = validate_params(p);
    if (v != SFFT_OK) return v;
    std::vector<Job*> js;
    js.reserve(count);
    sfft_status st = SFFT_OK;
    for (uint32_t i = 0; i < count && st == SFFT_OK; ++i) {
        Job* j = make_job(S, p, jobs + i, &st);
        if (j) js.push_back(j);
    }
    if (st == SFFT_OK) st = queue_jobs(S, js.data(), count, tickets);
    if (st != SFFT_OK)
        for (Job* j : js) delete j;
    return st;
}

sfft_status sfft_poll(sfft_server S, uint64_t ticket) {
    if (!S) return SFFT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return SFFT_ERR_INVALID_ARG;
    const Job* j = it->second;
    if (j->state == JobState::Done) return SFFT_OK;
    if (j->state == JobState::Failed) return j->status;
    return SFFT_ERR_BUSY;
}

sfft_status sfft_wait(sfft_server S, uint64_t ticket, uint64_t timeout_us, sfft_job_result* res) {
    if (!S) return SFFT_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return SFFT_ERR_INVALID_ARG;
    Job* j = it->second;  // (the node stays put while the lock is released; an iterator need not)
    auto finished = [&] { return j->state == JobState::Done || j->state == JobState::Failed; };
    if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished)) return SFFT_ERR_TIMEOUT;
    const sfft_status st = j->state == JobState::Done ? SFFT_OK : j->status;
    if (res) *res = j->res;
    S->jobs.erase(ticket);  // by key: submissions during the wait may have rehashed the map
    delete j;
    return st;
}

sfft_status sfft_wait_many(sfft_server S, const uint64_t* tickets, uint32_t count, uint64_t timeout_us,
                           sfft_job_result* res, int32_t* status) {
    if (!S || !tickets || !status || count == 0) return SFFT_ERR_INVALID_ARG;
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
    sfft_status first = SFFT_OK;
    bool pending = false;
    std::unique_lock<std::mutex> lk(S->mu);
    for (uint32_t i = 0; i < count; ++i) {
        auto it = S->jobs.find(tickets[i]);
        if (it == S->jobs.end()) {
            status[i] = SFFT_ERR_INVALID_ARG;
            if (first == SFFT_OK) first = SFFT_ERR_INVALID_ARG;
            continue;
        }
        Job* j = it->second;
        auto finished = [&] { return j->state == JobState::Done || j->state == JobState::Failed; };
        if (!S->cv_done.wait_until(lk, deadline, finished)) {
            status[i] = SFFT_ERR_TIMEOUT;
            pending = true;
            continue;
        }
        const sfft_status st = j->state == JobState::Done ? SFFT_OK : j->status;
        status[i] = st;
        if (res) res[i] = j->res;
        if (st != SFFT_OK && first == SFFT_OK) first = st;
        S->jobs.erase(j->ticket);
        delete j;
    }
    if (first != SFFT_OK) return first;
    return pending ? SFFT_ERR_TIMEOUT : SFFT_OK;
}

sfft_status sfft_server_stats_get(sfft_server S, sfft_server_stats* st) {
    if (!S || !st) return SFFT_ERR_INVALID_ARG;
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        st->submitted = S->submitted;
        st->completed = S->completed;
        st->failed = S->failed;
        st->launches = S->launches;
        st->plans = S->n_inst;
        st->bytes_in_use = S->bytes_in_use;
        st->bytes_peak = S->bytes_peak;
        st->mean_batch = S->launches ? (double)S->launched_jobs / (double)S->launches : 0.0;
        lat = S->latencies;
    }
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        size_t i = (size_t)(q * (double)lat.size());
        if (i >= lat.size()) i = lat.size() - 1;
        return lat[i];
    };
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    return SFFT_OK;
}

}  // extern "C"
