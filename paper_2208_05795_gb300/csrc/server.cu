// server.cu -- the serving runtime: a job queue over resident codes with
// admission by device-memory footprint, continuous batching of enumeration
// and importance-sampling jobs over a pool of prioritized streams, and
// latency statistics.  Host code only; every step of a job runs in the
// library's kernels (enumeration: api.cu, importance sampling: isfer.cu).
//
// Scheduling.  One worker thread owns the GPU side.  It loops: (1) collect
// the jobs whose end event has completed, copy their results to the host and
// give their device memory back; (2) admit queued jobs in arrival order while
// a slot is free and the footprint fits the budget (a job that does not fit
// may be overtaken by later jobs for at most backfill_ms, then admission
// waits for it); (3) sleep until a submit or the next poll.  An admitted job
// is enqueued on its slot's high- or low-priority stream (by its size), with
// persistent grids capped to its work and the decode split into chunks, so
// that a job arriving while a large one runs gets SMs at the large job's
// next chunk boundary.  Serial mode is the plain method for comparison: one
// job at a time, arrival order, one full-GPU launch per step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

using namespace tsx;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
    uint64_t id = 0;
    int kind = TSX_JOB_ENUMERATE;
    tsx_code *code = nullptr;
    tsx_enum_params ep{};
    tsx_is_params ip{};
    std::vector<int32_t> T;
    long long bytes = 0;
    double work = 0.0;
    long long units = 0;  // candidates (bound) or samples
    int state = 0;        // 0 queued, 1 running, 2 completed
    int status = TSX_EAGAIN;
    int slot = -1;
    bool high = false;
    int grid_sms = 0;
    Clock::time_point t_submit, t_start, t_end;
    tsx_ts_list *list = nullptr;
    IsJob *is = nullptr;
    cudaEvent_t done = nullptr;
    tsx_enum_stats es{};
    tsx_is_result ir{};
};

}  // namespace

struct tsx_server {
    tsx_server_params p{};
    int device = 0, num_sms = 0;
    std::mutex mu;
    std::condition_variable wake;  // worker: submit, destroy
    std::condition_variable fin;   // waiters: a job completed
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<Job *> queue;
    std::vector<Job *> running;
    std::unordered_map<uint64_t, Job *> jobs;
    std::vector<cudaStream_t> hi, lo;
    std::vector<char> slot_busy;
    long long hbm_used = 0;
    // statistics
    std::vector<double> lat, qwait;
    long long n_submitted = 0, n_done = 0, n_failed = 0, eu = 0, dec = 0, hbm_peak = 0;
    int max_conc = 0;
    bool any = false;
    Clock::time_point t_first, t_last;
};

extern "C" void server_params_default(tsx_server_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->max_jobs = 8;
    p->serial = 0;
    p->device = -1;
    p->hbm_bytes = 0;
    p->chunk_candidates = 16384;
    p->chunk_samples = 32768;
    p->small_work = 2e10;
    p->backfill_ms = 100.0;
    p->max_large = 1;
}

namespace {

// Sizes, validates and classifies a job (no device work).
int plan_job(tsx_server *S, Job *J) {
    const DevCode &g = *code_dev(J->code);
    if (code_device(J->code) != S->device) return TSX_EINVAL;
    const bool serial = S->p.serial != 0;
    int st;
    if (J->kind == TSX_JOB_ENUMERATE) {
        st = list_bytes(J->code, &J->ep, serial ? 0 : S->p.chunk_candidates, &J->bytes, &J->units);
        if (st != TSX_OK) return st;
        // edge updates: half of the bisection's decodes, each of half the maximum iterations
        J->work = (double)J->units * 0.5 * (J->ep.amp_steps + 1) * g.E * 0.5 * std::max(1, J->ep.K);
    } else if (J->kind == TSX_JOB_IS_FER) {
        st = is_job_bytes(J->code, J->T.data(), (int32_t)J->T.size(), &J->ip, serial ? 0 : S->p.chunk_samples,
                          &J->bytes);
        if (st != TSX_OK) return st;
        J->units = J->ip.n_samples;
        // edge updates: one decode per sample, of half the maximum iterations
        J->work = (double)J->units * g.E * 0.5 * std::max(1, J->ip.K);
    } else {
        return TSX_EINVAL;
    }
    J->high = !serial && J->work <= S->p.small_work;
    // persistent grids sized to the work: about 64 candidates (or samples) per SM
    int sms = S->num_sms;
    if (!serial) {
        const long long want = (J->units + 63) / 64;
        sms = (int)std::max<long long>(1, std::min<long long>(S->num_sms, want));
    }
    J->grid_sms = sms;
    return TSX_OK;
}

// Allocates and enqueues a job on its slot's stream (worker thread, no lock).
int start_job(tsx_server *S, Job *J) {
    cudaStream_t s = J->high ? S->hi[J->slot] : S->lo[J->slot];
    const bool serial = S->p.serial != 0;
    int st;
    if (J->kind == TSX_JOB_ENUMERATE)
        st = list_start(J->code, &J->ep, s, serial ? 0 : S->p.chunk_candidates, J->grid_sms, &J->list);
    else
        st = is_job_start(J->code, J->T.data(), (int32_t)J->T.size(), &J->ip, s,
                          serial ? 0 : S->p.chunk_samples, J->grid_sms, &J->is);
    if (st != TSX_OK) return st;
    if (cudaEventCreateWithFlags(&J->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(J->done, s) != cudaSuccess)
        return TSX_ECUDA;
    return TSX_OK;
}

// Results to the host, device memory back (worker thread, no lock).
int finish_job(Job *J) {
    int st = TSX_OK;
    if (J->list) {
        st = list_finish(J->list);
        tsx_ts_view v;
        if (ts_list_view(J->list, &v) == st) J->es = v.stats;
    } else if (J->is) {
        st = is_job_finish(J->is, &J->ir, nullptr, nullptr);
        is_job_delete(J->is);
        J->is = nullptr;
    }
    if (J->done) {
        cudaEventDestroy(J->done);
        J->done = nullptr;
    }
    return st;
}

void complete(tsx_server *S, Job *J, int st) {
    J->status = st;
    J->state = 2;
    J->t_end = Clock::now();
    if (J->slot >= 0) S->slot_busy[J->slot] = 0;
    S->hbm_used -= J->bytes;
    S->n_done++;
    if (st != TSX_OK) S->n_failed++;
    S->lat.push_back(ms_between(J->t_submit, J->t_end));
    S->qwait.push_back(ms_between(J->t_submit, J->t_start));
    if (J->kind == TSX_JOB_ENUMERATE) {
        S->eu += J->es.edge_updates;
        S->dec += J->es.decodes;
    } else {
        S->eu += J->ir.edge_updates;
        S->dec += J->ir.decodes;
    }
    S->t_last = J->t_end;
}

int free_slot(tsx_server *S) {
    for (int i = 0; i < (int)S->slot_busy.size(); i++)
        if (!S->slot_busy[i]) return i;
    return -1;
}

void worker_loop(tsx_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    const long long budget = S->p.hbm_bytes;
    while (true) {
        // (1) completions
        std::vector<Job *> ended;
        for (size_t i = 0; i < S->running.size();) {
            Job *J = S->running[i];
            const cudaError_t e = cudaEventQuery(J->done);
            if (e == cudaErrorNotReady) {
                i++;
                continue;
            }
            if (e != cudaSuccess) J->status = TSX_ECUDA;
            ended.push_back(J);
            S->running[i] = S->running.back();
            S->running.pop_back();
        }
        if (!ended.empty()) {
            lk.unlock();
            std::vector<int> sts;
            for (Job *J : ended) {
                const int st = finish_job(J);
                sts.push_back(J->status == TSX_ECUDA ? TSX_ECUDA : st);
            }
            lk.lock();
            for (size_t i = 0; i < ended.size(); i++) complete(S, ended[i], sts[i]);
            S->fin.notify_all();
        }
        // (2) admission in arrival order, with bounded overtaking
        while (!S->queue.empty()) {
            const int slot = free_slot(S);
            if (slot < 0) break;
            Job *pick = nullptr;
            size_t at = 0;
            const auto now = Clock::now();
            int n_large = 0;
            for (Job *R : S->running) n_large += R->high ? 0 : 1;
            bool large_waits = false;  // large jobs start in arrival order among themselves
            for (size_t i = 0; i < S->queue.size(); i++) {
                Job *J = S->queue[i];
                if (!J->high && (large_waits || n_large >= S->p.max_large)) {
                    large_waits = true;
                    continue;
                }
                if (S->hbm_used + J->bytes <= budget) {
                    pick = J;
                    at = i;
                    break;
                }
                // a job that does not fit may be overtaken only while it has waited less than backfill_ms
                if (S->p.serial || ms_between(J->t_submit, now) >= S->p.backfill_ms) break;
                if (!J->high) large_waits = true;
            }
            if (!pick) break;
            S->queue.erase(S->queue.begin() + (long)at);
            pick->slot = slot;
            pick->state = 1;
            pick->t_start = now;
            S->slot_busy[slot] = 1;
            S->hbm_used += pick->bytes;
            S->hbm_peak = std::max(S->hbm_peak, S->hbm_used);
            lk.unlock();
            const int st = start_job(S, pick);
            lk.lock();
            if (st != TSX_OK) {
                finish_job(pick);
                if (pick->list) {
                    list_delete(pick->list);
                    pick->list = nullptr;
                }
                complete(S, pick, st);
                S->fin.notify_all();
            } else {
                S->running.push_back(pick);
                S->max_conc = std::max(S->max_conc, (int)S->running.size());
            }
        }
        // (3) sleep
        if (S->stop && S->running.empty()) break;
        if (!S->running.empty())
            S->wake.wait_for(lk, std::chrono::microseconds(50));
        else
            S->wake.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    }
}

void fill_result(const Job *J, tsx_job_result *r) {
    memset(r, 0, sizeof(*r));
    r->status = J->state == 2 ? J->status : TSX_EAGAIN;
    r->kind = J->kind;
    r->high_priority = J->high ? 1 : 0;
    r->grid_sms = J->grid_sms;
    r->device_bytes = J->bytes;
    if (J->state >= 1) r->queue_ms = ms_between(J->t_submit, J->t_start);
    if (J->state == 2) {
        r->run_ms = ms_between(J->t_start, J->t_end);
        r->latency_ms = ms_between(J->t_submit, J->t_end);
        r->enum_stats = J->es;
        r->is_result = J->ir;
    }
}

double quantile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    // nearest rank
    size_t k = (size_t)std::ceil(q * (double)v.size());
    if (k < 1) k = 1;
    if (k > v.size()) k = v.size();
    return v[k - 1];
}

}  // namespace

extern "C" int server_create(const tsx_server_params *params, tsx_server **out) {
    if (!out) return TSX_EINVAL;
    *out = nullptr;
    tsx_server_params p;
    if (params)
        p = *params;
    else
        server_params_default(&p);
    if (p.max_jobs < 1 || p.max_jobs > 64 || p.hbm_bytes < 0 || p.chunk_candidates < 0 || p.chunk_samples < 0 ||
        !(p.small_work >= 0.0) || !(p.backfill_ms >= 0.0) || p.max_large < 1)
        return TSX_EINVAL;
    if (p.serial) p.max_jobs = 1;
    tsx_server *S = new tsx_server();
    int dev = p.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete S; return TSX_ECUDA; }
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(dev) != cudaSuccess) { delete S; return TSX_EINVAL; }
    S->device = dev;
    cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (p.hbm_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaSetDevice(prev); delete S; return TSX_ECUDA; }
        p.hbm_bytes = (int64_t)(fr / 2);
    }
    S->p = p;
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    S->hi.resize(p.max_jobs);
    S->lo.resize(p.max_jobs);
    S->slot_busy.assign(p.max_jobs, 0);
    for (int i = 0; i < p.max_jobs; i++)
        if (cudaStreamCreateWithPriority(&S->hi[i], cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&S->lo[i], cudaStreamNonBlocking, least) != cudaSuccess) {
            for (cudaStream_t s : S->hi) if (s) cudaStreamDestroy(s);
            for (cudaStream_t s : S->lo) if (s) cudaStreamDestroy(s);
            cudaSetDevice(prev);
            delete S;
            return TSX_ECUDA;
        }
    cudaSetDevice(prev);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return TSX_OK;
}

extern "C" int server_submit(tsx_server *S, const tsx_job *job, uint64_t *id) {
    const auto t = Clock::now();
    if (!S || !job || !id || !job->code) return TSX_EINVAL;
    Job *J = new Job();
    J->kind = job->kind;
    J->code = job->code;
    J->ep = job->enum_params;
    J->ip = job->is_params;
    if (job->kind == TSX_JOB_IS_FER) {
        if (job->a < 0 || (job->a > 0 && !job->ts_vars)) { delete J; return TSX_EINVAL; }
        J->T.assign(job->ts_vars, job->ts_vars + job->a);
    }
    J->t_submit = t;
    const int st = plan_job(S, J);
    if (st != TSX_OK) { delete J; return st; }
    if (J->bytes > S->p.hbm_bytes) { delete J; return TSX_ENOMEM; }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { delete J; return TSX_EBUSY; }
        J->id = S->next_id++;
        S->jobs[J->id] = J;
        S->queue.push_back(J);
        S->n_submitted++;
        if (!S->any) {
            S->any = true;
            S->t_first = t;
        }
        *id = J->id;
    }
    S->wake.notify_all();
    return TSX_OK;
}

extern "C" int server_poll(tsx_server *S, uint64_t id, tsx_job_result *r) {
    if (!S || !r) return TSX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return TSX_ENOTFOUND;
    fill_result(it->second, r);
    return r->status;
}

extern "C" int server_wait(tsx_server *S, uint64_t id, double timeout_ms, tsx_job_result *r) {
    if (!S || !r) return TSX_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto done = [&] {
        auto it = S->jobs.find(id);
        return it == S->jobs.end() || it->second->state == 2;
    };
    if (timeout_ms < 0)
        S->fin.wait(lk, done);
    else
        S->fin.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), done);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return TSX_ENOTFOUND;
    fill_result(it->second, r);
    return r->status;
}

extern "C" int server_job_view(tsx_server *S, uint64_t id, tsx_ts_view *view) {
    if (!S || !view) return TSX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return TSX_ENOTFOUND;
    Job *J = it->second;
    if (J->state != 2) return TSX_EAGAIN;
    if (J->kind != TSX_JOB_ENUMERATE || !J->list) return J->status != TSX_OK ? J->status : TSX_EINVAL;
    // host results only: the list was fetched when the job completed
    return ts_list_view(J->list, view);
}

extern "C" int server_release(tsx_server *S, uint64_t id) {
    if (!S) return TSX_EINVAL;
    Job *J = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->jobs.find(id);
        if (it == S->jobs.end()) return TSX_ENOTFOUND;
        if (it->second->state != 2) return TSX_EAGAIN;
        J = it->second;
        S->jobs.erase(it);
    }
    if (J->list) list_delete(J->list);
    delete J;
    return TSX_OK;
}

extern "C" int server_drain(tsx_server *S) {
    if (!S) return TSX_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    S->fin.wait(lk, [&] { return S->queue.empty() && S->running.empty(); });
    return TSX_OK;
}

extern "C" int server_stats(tsx_server *S, tsx_server_stats *o) {
    if (!S || !o) return TSX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(o, 0, sizeof(*o));
    o->submitted = S->n_submitted;
    o->done = S->n_done;
    o->failed = S->n_failed;
    o->running = (int64_t)S->running.size();
    o->queued = (int64_t)S->queue.size();
    o->p50_ms = quantile(S->lat, 0.50);
    o->p90_ms = quantile(S->lat, 0.90);
    o->p99_ms = quantile(S->lat, 0.99);
    o->max_ms = quantile(S->lat, 1.0);
    double sl = 0.0, sq = 0.0;
    for (double x : S->lat) sl += x;
    for (double x : S->qwait) sq += x;
    o->mean_ms = S->lat.empty() ? 0.0 : sl / (double)S->lat.size();
    o->mean_queue_ms = S->qwait.empty() ? 0.0 : sq / (double)S->qwait.size();
    o->makespan_ms = S->any && S->n_done ? ms_between(S->t_first, S->t_last) : 0.0;
    o->edge_updates = S->eu;
    o->decodes = S->dec;
    o->edge_updates_per_s = o->makespan_ms > 0.0 ? (double)S->eu / (o->makespan_ms / 1e3) : 0.0;
    o->hbm_peak_bytes = S->hbm_peak;
    o->max_concurrent = S->max_conc;
    return TSX_OK;
}

extern "C" void server_reset_stats(tsx_server *S) {
    if (!S) return;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat.clear();
    S->qwait.clear();
    S->n_submitted = (long long)(S->queue.size() + S->running.size());
    S->n_done = S->n_failed = S->eu = S->dec = 0;
    S->hbm_peak = S->hbm_used;
    S->max_conc = (int)S->running.size();
    S->any = false;
}

extern "C" void server_destroy(tsx_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued jobs are dropped; the ones on the device finish
        for (Job *J : S->queue) {
            J->state = 2;
            J->status = TSX_EBUSY;
        }
        S->queue.clear();
    }
    S->wake.notify_all();
    if (S->worker.joinable()) S->worker.join();
    S->fin.notify_all();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto &kv : S->jobs) {
        if (kv.second->list) list_delete(kv.second->list);
        delete kv.second;
    }
    S->jobs.clear();
    for (cudaStream_t s : S->hi) cudaStreamSynchronize(s), cudaStreamDestroy(s);
    for (cudaStream_t s : S->lo) cudaStreamSynchronize(s), cudaStreamDestroy(s);
    cudaSetDevice(prev);
    delete S;
}
