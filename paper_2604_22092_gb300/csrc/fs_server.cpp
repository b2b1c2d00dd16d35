// fs_server.cpp -- continuous batching of forecast ensembles (include/fs.h,
// "Serving"). A host thread owns one batch (the device segment table) and
// runs it in quanta of K launches; between quanta it admits queued requests
// first come, first served while their device memory fits the budget and the
// updates per launch of the running requests stay under the in-flight cap
// (each request becomes ensembles of at most 32 realisations that join the
// running batch), and retires requests whose last step has been integrated.
// Built on the public ensemble and batch entry points; no numerics of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fs.h"
#include "fs_objects.h"

using fsapi::fail;
using fsapi::g_err;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    fs_graph* g = nullptr;
    int64_t n = 0;
    std::vector<fs_sim_params> params;     // one per realisation
    std::vector<int32_t> idx;
    int64_t steps = 0;
    int64_t bytes = 0;                     // device memory estimate
    std::vector<fs_ens*> ens;
    std::vector<int> ens_first;
    std::vector<std::vector<uint32_t>> ens_out;
    int64_t g_add = 0;                     // batch launch count when its ensembles joined
    std::vector<uint32_t> counts;          // [(steps+1)][n_real][4]
    Clock::time_point t_submit, t_done;
    bool done = false;
    fs_status status = FS_OK;
    int64_t load() const { return n * (int64_t)params.size(); }   // node updates per launch
};

// device memory of one ensemble (states, ages, masks, tables, counts rows; in
// the push form also the per-replicate counts and pending tallies: 1 + 2 x 2
// bytes per thread-class node, 4 + 2 x 8 per merge-class node; with a
// shedding profile two infectivity buffers like the ages and one more table
// per realisation)
int64_t ensemble_bytes(int64_t n, int64_t n_merge, int R, int age_bytes, int64_t steps, bool push, bool shed)
{
    const int64_t Rp = R <= 8 ? 8 : R <= 16 ? 16 : 32;
    int64_t b = n * Rp * (1 + age_bytes) + 2 * (n + 1) * (Rp / 8) + (int64_t)R * (2 * 4096 * 16 + 256 * 4) +
                (steps + 1) * Rp * 16 + 4096;
    if (push)
        b += (n - n_merge) * Rp * 5 + std::max<int64_t>(n_merge, 1) * Rp * 20;
    if (shed)
        b += 2 * n * Rp * age_bytes + (int64_t)R * 4096 * 16;
    return b;
}

}  // namespace

struct fs_server {
    fs_server_cfg cfg{};
    int device = 0;
    int64_t budget = 0;
    fs_batch* batch = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> all;
    std::vector<Request*> running;          // owned by the thread
    int64_t used = 0;
    int64_t G = 0;                          // launches run by the batch
    bool stop = false;
    uint64_t next_id = 1;
    fs_server_stats st{};
    fs_status thread_status = FS_OK;
    std::string thread_error;
};

namespace {

void finish(fs_server* s, Request* q, fs_status status)
{
    for (fs_ens* e : q->ens)
        fs_ens_destroy(e);
    q->ens.clear();
    std::lock_guard<std::mutex> lock(s->mu);
    q->status = status;
    q->t_done = Clock::now();
    q->done = true;
    s->used -= q->bytes;
    s->st.completed += 1;
    s->st.running -= 1;
    if (status == FS_OK)
        s->st.node_updates += q->n * (int64_t)q->params.size() * q->steps;
    s->cv.notify_all();
}

// creates the request's ensembles and adds them to the batch
fs_status start(fs_server* s, Request* q)
{
    const int n_real = (int)q->params.size();
    for (int off = 0; off < n_real; off += 32) {
        const int R = std::min(32, n_real - off);
        fs_ens* e = nullptr;
        fs_status st = fs_ens_create(q->g, q->params.data() + off, R, q->idx.data(), (int64_t)q->idx.size(), &e);
        if (st != FS_OK)
            return st;
        q->ens.push_back(e);
        q->ens_first.push_back(off);
        q->ens_out.emplace_back((size_t)(q->steps + 1) * R * 4);
        st = fs_batch_add(s->batch, e, q->steps, q->ens_out.back().data());
        if (st != FS_OK)
            return st;
    }
    q->g_add = s->G;
    return FS_OK;
}

void collect(Request* q)
{
    const int n_real = (int)q->params.size();
    q->counts.assign((size_t)(q->steps + 1) * n_real * 4, 0u);
    for (size_t m = 0; m < q->ens.size(); ++m) {
        const int off = q->ens_first[m];
        const int R = std::min(32, n_real - off);
        for (int64_t row = 0; row <= q->steps; ++row)
            memcpy(q->counts.data() + ((size_t)row * n_real + off) * 4, q->ens_out[m].data() + (size_t)row * R * 4,
                   sizeof(uint32_t) * R * 4);
    }
}

// retires the queued requests that have waited longer than the wait limit
// (FS_ETIMEOUT); they hold no device memory yet. Called with s->mu held.
void expire_locked(fs_server* s, Clock::time_point now)
{
    if (s->cfg.wait_limit_s <= 0.0)
        return;
    const auto limit = std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(s->cfg.wait_limit_s));
    std::deque<Request*> keep;
    bool any = false;
    for (Request* q : s->queue) {
        if (now - q->t_submit > limit) {
            q->status = FS_ETIMEOUT;
            q->t_done = now;
            q->done = true;
            s->st.queued -= 1;
            s->st.completed += 1;
            any = true;
        } else {
            keep.push_back(q);
        }
    }
    s->queue.swap(keep);
    if (any)
        s->cv.notify_all();
}

void serve(fs_server* s)
{
    cudaSetDevice(s->device);
    const int K = s->cfg.quantum;
    for (;;) {
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop)
                break;
            expire_locked(s, Clock::now());
            while (!s->queue.empty()) {
                Request* q = s->queue.front();
                const int64_t need_rows = ((int64_t)q->params.size() + 31) / 32;
                if (s->used + q->bytes > s->budget)
                    break;
                int64_t rows = 0, load = 0;
                for (Request* r : s->running) {
                    rows += (int64_t)r->ens.size();
                    load += r->load();
                }
                for (Request* r : admitted) {
                    rows += ((int64_t)r->params.size() + 31) / 32;
                    load += r->load();
                }
                if (rows + need_rows > s->cfg.max_members)
                    break;
                if (s->cfg.max_inflight > 0 && load > 0 && load + q->load() > s->cfg.max_inflight)
                    break;
                s->queue.pop_front();
                s->used += q->bytes;
                s->st.queued -= 1;
                s->st.running += 1;
                admitted.push_back(q);
            }
            if (admitted.empty() && s->running.empty()) {
                s->cv.wait_for(lock, std::chrono::milliseconds(20));
                continue;
            }
        }
        for (Request* q : admitted) {
            const fs_status st = start(s, q);
            if (st == FS_OK) {
                s->running.push_back(q);
            } else {
                // a failed start leaves nothing in the batch for this request:
                // its ensembles that did join are removed with the batch run
                // below only when finished, so fail the whole server instead
                std::lock_guard<std::mutex> lock(s->mu);
                s->thread_status = st;
                s->thread_error = g_err;
                s->stop = true;
                s->cv.notify_all();
            }
        }
        if (s->stop)
            break;
        const auto t0 = Clock::now();
        const fs_status st = fs_batch_run(s->batch, K, K);
        s->G += K;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->st.launches += K;
            s->st.busy_seconds += std::chrono::duration<double>(Clock::now() - t0).count();
            if (st != FS_OK) {
                s->thread_status = st;
                s->thread_error = g_err;
                s->stop = true;
                s->cv.notify_all();
            }
        }
        if (st != FS_OK)
            break;
        std::vector<Request*> keep;
        for (Request* q : s->running) {
            if (q->g_add + q->steps + 1 <= s->G) {
                collect(q);
                finish(s, q, FS_OK);
            } else {
                keep.push_back(q);
            }
        }
        s->running.swap(keep);
    }
}

}  // namespace

extern "C" {

fs_status fs_server_create(const fs_server_cfg* cfg, fs_server** out)
{
    g_err.clear();
    if (!out)
        return fail(FS_EINVAL, "fs_server_create: NULL out");
    *out = nullptr;
    fs_server_cfg c{};
    if (cfg)
        c = *cfg;
    if (c.reserved_ != 0 || c.hbm_budget_bytes < 0 || c.max_members < 0 || c.quantum < 0 ||
        c.quantum > fs::kMaxGraphSteps || c.age_dtype < FS_AGE_F32 || c.age_dtype > FS_AGE_BF16 ||
        c.max_inflight < -1 || !(c.wait_limit_s >= 0.0))
        return fail(FS_EINVAL, "fs_server_create: bad configuration");
    if (c.max_inflight == 0)
        c.max_inflight = (int64_t)1 << 25;
    if (c.max_members == 0)
        c.max_members = 4096;
    if (c.quantum == 0)
        c.quantum = 10;
    fs_server* s = new fs_server();
    s->cfg = c;
    cudaGetDevice(&s->device);
    if (c.hbm_budget_bytes > 0) {
        s->budget = c.hbm_budget_bytes;
    } else {
        size_t free_b = 0, total_b = 0;
        cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) {
            delete s;
            return fail(FS_ECUDA, "fs_server_create: cudaMemGetInfo: %s", cudaGetErrorString(e));
        }
        s->budget = (int64_t)(0.8 * (double)free_b);
    }
    fs_status st = fs_batch_create(c.age_dtype, c.max_members, nullptr, &s->batch);
    if (st != FS_OK) {
        delete s;
        return st;
    }
    s->th = std::thread(serve, s);
    *out = s;
    return FS_OK;
}

fs_status fs_server_submit(fs_server* s, fs_graph* g, const fs_sim_params* scenarios, int32_t n_scen,
                           int32_t replicates, const int32_t* index_nodes, int64_t n_index, int64_t steps,
                           uint64_t* request_id)
{
    g_err.clear();
    if (!s || !g || !scenarios || !request_id)
        return fail(FS_EINVAL, "fs_server_submit: NULL argument");
    if (n_scen < 1 || replicates < 1 || (int64_t)n_scen * replicates > (1 << 20))
        return fail(FS_EINVAL, "fs_server_submit: bad n_scen or replicates");
    if (steps < 0 || steps >= ((int64_t)1 << 31))
        return fail(FS_EINVAL, "fs_server_submit: bad steps");
    fs_graph_info_t info{};
    fs_status st = fs_graph_info_get(g, &info);
    if (st != FS_OK)
        return st;
    if (n_index < 0 || n_index > info.n || (n_index > 0 && !index_nodes))
        return fail(FS_EINVAL, "fs_server_submit: bad index list");
    Request* q = new Request();
    q->g = g;
    q->n = info.n;
    q->steps = steps;
    q->idx.assign(index_nodes, index_nodes + n_index);
    for (int sc = 0; sc < n_scen; ++sc) {
        fs_sim_params p = scenarios[sc];
        if (p.age_dtype != s->cfg.age_dtype) {
            delete q;
            return fail(FS_EINVAL, "fs_server_submit: scenario age_dtype differs from the server's");
        }
        st = fsapi::check_params(&p);
        if (st != FS_OK) {
            delete q;
            return st;
        }
        if (sc > 0 && p.flags != scenarios[0].flags) {
            delete q;
            return fail(FS_EINVAL, "fs_server_submit: scenarios must share flags");
        }
        if ((p.flags & FS_ACTIVE_LIST) || p.theta > 0) {
            delete q;
            return fail(FS_EUNSUPPORTED, "fs_server_submit: served ensembles run the renewal engine without an "
                                         "active list");
        }
        if (p.shed_mode != FS_SHED_NONE && p.flags == FS_PRESSURE_PUSH) {
            delete q;
            return fail(FS_EUNSUPPORTED, "fs_server_submit: a shedding profile needs the gather form");
        }
        if (sc > 0 && (p.shed_mode != FS_SHED_NONE) != (scenarios[0].shed_mode != FS_SHED_NONE)) {
            delete q;
            return fail(FS_EINVAL, "fs_server_submit: every scenario has a shedding profile or none");
        }
        if (sc > 0 && (p.eps > 0) != (scenarios[0].eps > 0)) {
            delete q;
            return fail(FS_EINVAL, "fs_server_submit: every scenario takes the adaptive step (eps > 0) or none");
        }
        if (p.flags == FS_PRESSURE_PUSH && !fsapi::push_available(g)) {
            delete q;
            return fail(FS_EUNSUPPORTED, "fs_server_submit: FS_PRESSURE_PUSH is not available on this graph");
        }
        if (sc > 0 && (p.model != scenarios[0].model || p.index_state != scenarios[0].index_state)) {
            delete q;
            return fail(FS_EINVAL, "fs_server_submit: scenarios must share model and index_state");
        }
        for (int r = 0; r < replicates; ++r) {
            fs_sim_params pr = p;
            pr.replicate = p.replicate + (uint32_t)r;
            q->params.push_back(pr);
        }
    }
    const int age_bytes = s->cfg.age_dtype == FS_AGE_F32 ? 4 : 2;
    const bool shed = scenarios[0].shed_mode != FS_SHED_NONE;
    for (size_t off = 0; off < q->params.size(); off += 32) {
        const int R = (int)std::min<size_t>(32, q->params.size() - off);
        q->bytes += ensemble_bytes(q->n, g->n_m, R, age_bytes, steps, fsapi::packed_push(g, scenarios[0], R), shed);
    }
    if (q->bytes > s->budget) {
        const int64_t b = q->bytes;
        delete q;
        return fail(FS_ENOMEM, "fs_server_submit: the request needs %lld bytes, beyond the budget %lld",
                    (long long)b, (long long)s->budget);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) {
        delete q;
        return fail(s->thread_status == FS_OK ? FS_ESTATE : s->thread_status, "fs_server_submit: server stopped: %s",
                    s->thread_error.c_str());
    }
    q->id = s->next_id++;
    q->t_submit = Clock::now();
    s->all[q->id] = q;
    s->queue.push_back(q);
    s->st.submitted += 1;
    s->st.queued += 1;
    *request_id = q->id;
    s->cv.notify_all();
    return FS_OK;
}

fs_status fs_server_poll(fs_server* s, uint64_t request_id, int32_t* done, uint32_t* counts_out, double* seconds)
{
    if (!s || !done)
        return fail(FS_EINVAL, "fs_server_poll: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end())
        return fail(FS_EINVAL, "fs_server_poll: unknown request %llu", (unsigned long long)request_id);
    Request* q = it->second;
    *done = q->done ? 1 : 0;
    if (!q->done) {
        if (s->stop && s->thread_status != FS_OK)
            return fail(s->thread_status, "fs_server_poll: server stopped: %s", s->thread_error.c_str());
        return FS_OK;
    }
    if (q->status != FS_OK)
        return fail(q->status, "fs_server_poll: request %llu failed", (unsigned long long)request_id);
    if (counts_out)
        memcpy(counts_out, q->counts.data(), sizeof(uint32_t) * q->counts.size());
    if (seconds)
        *seconds = std::chrono::duration<double>(q->t_done - q->t_submit).count();
    return FS_OK;
}

fs_status fs_server_drain(fs_server* s, double timeout_s)
{
    if (!s)
        return fail(FS_EINVAL, "fs_server_drain: NULL server");
    std::unique_lock<std::mutex> lock(s->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (s->st.completed < s->st.submitted) {
        if (s->stop && s->thread_status != FS_OK)
            return fail(s->thread_status, "fs_server_drain: server stopped: %s", s->thread_error.c_str());
        if (s->cv.wait_until(lock, until) == std::cv_status::timeout && s->st.completed < s->st.submitted)
            return fail(FS_ETIMEOUT, "fs_server_drain: %lld requests still open",
                        (long long)(s->st.submitted - s->st.completed));
    }
    return FS_OK;
}

fs_status fs_server_stats_get(fs_server* s, fs_server_stats* out)
{
    if (!s || !out)
        return fail(FS_EINVAL, "fs_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    out->device_bytes = s->used;
    return FS_OK;
}

fs_status fs_server_destroy(fs_server* s)
{
    if (!s)
        return fail(FS_EINVAL, "fs_server_destroy: NULL server");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->th.joinable())
        s->th.join();
    fs_batch_destroy(s->batch);               // detaches any live members
    for (Request* q : s->running)
        for (fs_ens* e : q->ens)
            fs_ens_destroy(e);
    for (auto& kv : s->all)
        delete kv.second;
    delete s;
    return FS_OK;
}

}  // extern "C"
