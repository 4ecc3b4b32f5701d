// Serving: a request loop with continuous batching.  Jobs (one graph each)
// are submitted at any time; worker threads admit them while a slot is free
// and the device memory estimated for the admitted jobs stays within the
// budget, keep each job's CSR and community state resident for the whole
// run, and run the jobs side by side on their own streams, so that the
// iterations of different jobs overlap on the device.  A job's result does
// not depend on what runs beside it (each job is an independent graph
// handle; every kernel is deterministic).
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

#include "lf_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    std::vector<int32_t> src, dst;
    int32_t queue_size = 1, max_iters = 0;
    double threshold = 0.0;
    int64_t est_bytes = 0;
    // result
    bool done = false;
    lf_job_result res{};
    std::string error;
    std::vector<int64_t> offsets;
    std::vector<int32_t> members;
};

}  // namespace

struct lf_server {
    lf_server_options opt{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> pending;
    std::map<int64_t, std::shared_ptr<Job>> jobs;
    int64_t next_id = 1;
    int64_t reserved = 0;   // estimated bytes of the jobs admitted and not finished
    int active = 0;
    int waiters = 0;        // threads inside lf_server_wait
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

double ms_since(const lf_server *s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

// Device memory a job will hold, from its edge count: the input copy and the
// CSR (12 bytes per input edge), orientation and triangle work (~24 per
// edge), per-node arrays and membership rows (~96 per node, with nodes
// bounded by twice the edges), plus a fixed amount for scratch.
int64_t estimate_bytes(int64_t edges) { return 36 * edges + 96 * 2 * edges + (64ll << 20); }

void worker(lf_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admit the oldest pending job once it fits the budget (a job larger
            // than the whole budget runs alone)
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->pending.empty()) return false;
                const int64_t need = s->pending.front()->est_bytes;
                return s->active == 0 || s->reserved + need <= s->opt.hbm_budget_bytes;
            });
            if (s->stop && s->pending.empty()) break;
            if (s->stop) break;
            job = s->pending.front();
            s->pending.pop_front();
            s->reserved += job->est_bytes;
            ++s->active;
            job->res.t_admit_ms = ms_since(s);
        }
        lf_options o{};
        o.stream = st;
        lf_graph *g = nullptr;
        lf_status rc = lf_graph_create(job->src.data(), job->dst.data(), (int64_t)job->src.size(), &o, &g);
        lf_run_stats stats{};
        std::vector<double> hist((size_t)std::max(1, job->max_iters));
        stats.history_cap = job->max_iters;
        stats.wcc_history = hist.data();
        if (rc == LF_OK) rc = lf_run(g, job->queue_size, job->threshold, job->max_iters, &stats);
        int64_t nc = 0, nm = 0;
        if (rc == LF_OK) rc = lf_get_communities(g, nullptr, 0, nullptr, 0, &nc, &nm);
        if (rc == LF_OK) {
            job->offsets.resize((size_t)nc + 1);
            job->members.resize((size_t)std::max<int64_t>(nm, 1));
            rc = lf_get_communities(g, job->offsets.data(), nc + 1, job->members.data(), (int64_t)job->members.size(),
                                    &nc, &nm);
            job->members.resize((size_t)nm);
        }
        std::string err = rc == LF_OK ? std::string() : std::string(lf_last_error());
        if (g) {
            lf_get_sizes(g, &job->res.num_nodes, &job->res.num_edges);
            lf_graph_destroy(g);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            job->res.status = rc;
            job->res.iterations = stats.iterations;
            job->res.converged = stats.converged;
            job->res.wcc_initial = stats.wcc_initial;
            job->res.wcc_final = stats.iterations > 0 ? hist[(size_t)stats.iterations - 1] : stats.wcc_initial;
            job->res.num_communities = nc;
            job->res.t_done_ms = ms_since(s);
            job->res.est_bytes = job->est_bytes;
            job->error = err;
            job->done = true;
            job->src.clear();
            job->src.shrink_to_fit();
            job->dst.clear();
            job->dst.shrink_to_fit();
            s->reserved -= job->est_bytes;
            --s->active;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

lf_status lf_server_create(const lf_server_options *opt, lf_server **out) {
    if (!out) {
        lf::set_error(LF_ERR_INVALID, "out is NULL");
        return LF_ERR_INVALID;
    }
    *out = nullptr;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        lf::set_error(LF_ERR_CUDA, "no CUDA device available");
        return LF_ERR_CUDA;
    }
    auto *s = new (std::nothrow) lf_server();
    if (!s) {
        lf::set_error(LF_ERR_OOM, "out of host memory");
        return LF_ERR_OOM;
    }
    if (opt) s->opt = *opt;
    if (s->opt.max_active < 1) s->opt.max_active = 4;
    if (s->opt.hbm_budget_bytes <= 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        s->opt.hbm_budget_bytes = (int64_t)(free_b / 2);
    }
    cudaGetDevice(&s->device);
    s->t0 = Clock::now();
    for (int i = 0; i < s->opt.max_active; ++i) s->workers.emplace_back(worker, s);
    *out = s;
    return LF_OK;
}

lf_status lf_server_submit(lf_server *s, const int32_t *src, const int32_t *dst, int64_t num_edges,
                           int32_t queue_size, double wcc_threshold, int32_t max_iters, int64_t *job_id) {
    if (!s || !job_id || num_edges < 0 || (num_edges > 0 && (!src || !dst)) || queue_size < 1 || max_iters < 0) {
        lf::set_error(LF_ERR_INVALID, "invalid argument");
        return LF_ERR_INVALID;
    }
    auto job = std::make_shared<Job>();
    job->src.assign(src, src + num_edges);
    job->dst.assign(dst, dst + num_edges);
    job->queue_size = queue_size;
    job->threshold = wcc_threshold;
    job->max_iters = max_iters;
    job->est_bytes = estimate_bytes(num_edges);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            lf::set_error(LF_ERR_STATE, "server is shutting down");
            return LF_ERR_STATE;
        }
        job->id = s->next_id++;
        job->res.t_submit_ms = ms_since(s);
        s->pending.push_back(job);
        s->jobs[job->id] = job;
        *job_id = job->id;
    }
    s->cv_work.notify_all();
    return LF_OK;
}

lf_status lf_server_wait(lf_server *s, int64_t job_id, double timeout_s, lf_job_result *res) {
    if (!s) {
        lf::set_error(LF_ERR_INVALID, "server is NULL");
        return LF_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) {
        lf::set_error(LF_ERR_INVALID, "unknown job %lld", (long long)job_id);
        return LF_ERR_INVALID;
    }
    std::shared_ptr<Job> job = it->second;
    const auto pred = [&] { return job->done; };
    ++s->waiters;
    bool finished = true;
    if (timeout_s < 0)
        s->cv_done.wait(lk, pred);
    else
        finished = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
    if (--s->waiters == 0 && s->stop) s->cv_done.notify_all();   // lf_server_destroy waits for this
    if (!finished) {
        lf::set_error(LF_ERR_TIMEOUT, "job %lld not finished", (long long)job_id);
        return LF_ERR_TIMEOUT;
    }
    if (res) *res = job->res;
    if (job->res.status != LF_OK) {
        lf::set_error((lf_status)job->res.status, "job %lld: %s", (long long)job_id, job->error.c_str());
        return (lf_status)job->res.status;
    }
    return LF_OK;
}

lf_status lf_server_get_communities(lf_server *s, int64_t job_id, int64_t *offsets, int64_t offsets_cap,
                                    int32_t *members, int64_t members_cap, int64_t *num_communities,
                                    int64_t *num_members) {
    if (!s) {
        lf::set_error(LF_ERR_INVALID, "server is NULL");
        return LF_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || !it->second->done) {
        lf::set_error(LF_ERR_STATE, "job %lld unknown or not finished", (long long)job_id);
        return LF_ERR_STATE;
    }
    const Job &j = *it->second;
    const int64_t nc = j.offsets.empty() ? 0 : (int64_t)j.offsets.size() - 1, nm = (int64_t)j.members.size();
    if (num_communities) *num_communities = nc;
    if (num_members) *num_members = nm;
    if (!offsets || !members) return LF_OK;
    if (offsets_cap < nc + 1 || members_cap < nm) {
        lf::set_error(LF_ERR_CAPACITY, "output buffers too small");
        return LF_ERR_CAPACITY;
    }
    if (nc + 1 > 0 && !j.offsets.empty()) std::memcpy(offsets, j.offsets.data(), (size_t)(nc + 1) * 8);
    if (nm > 0) std::memcpy(members, j.members.data(), (size_t)nm * 4);
    return LF_OK;
}

lf_status lf_server_release(lf_server *s, int64_t job_id) {
    if (!s) {
        lf::set_error(LF_ERR_INVALID, "server is NULL");
        return LF_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || !it->second->done) {
        lf::set_error(LF_ERR_STATE, "job %lld unknown or not finished", (long long)job_id);
        return LF_ERR_STATE;
    }
    s->jobs.erase(it);
    return LF_OK;
}

void lf_server_destroy(lf_server *s) {
    if (!s) return;
    {
        // jobs not yet admitted are dropped: each finishes with LF_ERR_STATE,
        // so that a thread waiting on one wakes up instead of waiting forever
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &job : s->pending) {
            job->res.status = LF_ERR_STATE;
            job->res.t_done_ms = ms_since(s);
            job->error = "cancelled: the server was destroyed before the job was admitted";
            job->done = true;
        }
        s->pending.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &t : s->workers) t.join();
    {
        // every job is finished now; let the threads inside lf_server_wait leave
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->waiters == 0; });
    }
    delete s;
}

}  // extern "C"
