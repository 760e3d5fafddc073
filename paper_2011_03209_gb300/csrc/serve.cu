// serve.cu -- request server: many mapper graphs of resident datasets
// computed concurrently, admitted by device-memory footprint.
//
// The paper recomputes a mapper graph whenever the user changes a parameter
// in the interface (§4.1) or sweeps parameter ranges from its command line
// (§4.4). Here requests (dataset, parameters) arrive at any time and run as
// soon as a worker slot is free and their estimated device-memory footprint
// fits beside the requests already running. Each slot is a host thread with
// its own library context and CUDA stream, so the device work of concurrent
// requests overlaps; results are exact whatever runs beside them.
//
// Admission: a free slot takes the oldest queued request that fits beside
// the running ones; when nothing runs, the oldest request starts whatever
// its size. A request that fits may so overtake an older one that does not,
// but only kMaxOvertakes times: after that the older request is first in
// line and the slots wait for it (aging), so large requests still start.
// Shutdown completes every request still queued with MAPPER_ECANCELED and
// returns only after every thread waiting on a request has left.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mapper.h"
#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxOvertakes = 8;      // later requests that may start before a blocked one

struct Dataset {
    const float* X;
    int64_t n;
    int32_t d;
    int64_t ld;
};

struct Request {
    int64_t id;
    Dataset dataset;
    mapper_params params;
    size_t footprint;
    Clock::time_point t_submit, t_start, t_end;
    mapper_graph_t* graph = nullptr;
    int status = MAPPER_OK;
    std::string error;
    bool done = false;
    int overtaken = 0;                // later requests admitted while this one waited
};

double secs(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double>(b - a).count();
}

}  // namespace

struct mapper_server {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    int running = 0;
    bool stopping = false;
    std::vector<Dataset> datasets;
    std::deque<std::shared_ptr<Request>> queue;              // admitted in arrival order
    std::map<int64_t, std::shared_ptr<Request>> requests;    // not yet collected
    int64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    int init_status = MAPPER_OK;
    std::string init_error;
    int ready = 0;
    int waiters = 0;                                         // threads inside mapper_server_wait
};

namespace {

// Index in S->queue of the request a free slot starts now, or -1 (caller
// holds S->mu): the oldest that fits beside the running requests, unless an
// older one that does not fit has been overtaken kMaxOvertakes times already.
int pick_request(const mapper_server* S)
{
    if (S->queue.empty()) return -1;
    if (S->running == 0) return 0;
    for (size_t i = 0; i < S->queue.size(); ++i) {
        const Request& r = *S->queue[i];
        if (S->in_use + r.footprint <= S->budget) return (int)i;
        if (r.overtaken >= kMaxOvertakes) return -1;
    }
    return -1;
}

void worker_main(mapper_server* S, int slot)
{
    (void)slot;
    cudaSetDevice(S->device);
    mapper_ctx* ctx = nullptr;
    const int rc = mapper_create(&ctx, S->device, 0, nullptr);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (rc != MAPPER_OK && S->init_status == MAPPER_OK) {
            S->init_status = rc;
            S->init_error = mapper_last_error();
        }
        ++S->ready;
    }
    S->cv_done.notify_all();
    if (rc != MAPPER_OK) return;
    while (true) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            int at = -1;
            S->cv_work.wait(lk, [&] { return S->stopping || (at = pick_request(S)) >= 0; });
            if (S->stopping) break;
            r = S->queue[at];
            for (int i = 0; i < at; ++i) ++S->queue[i]->overtaken;
            S->queue.erase(S->queue.begin() + at);
            S->in_use += r->footprint;
            ++S->running;
            r->t_start = Clock::now();
        }
        S->cv_work.notify_all();
        const Dataset ds = r->dataset;
        mapper_graph_t* g = nullptr;
        const int st = mapper_graph(ctx, ds.X, ds.n, ds.d, ds.ld, &r->params, &g);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->t_end = Clock::now();
            r->status = st;
            if (st != MAPPER_OK) r->error = mapper_last_error();
            r->graph = g;
            r->done = true;
            S->in_use -= r->footprint;
            --S->running;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    mapper_destroy(ctx);
}

int fail(int status, const std::string& msg)
{
    mgb::set_error(msg);
    return status;
}

}  // namespace

extern "C" {

int mapper_server_create(mapper_server** out, int device, int n_slots, size_t hbm_budget_bytes)
{
    if (!out) return fail(MAPPER_EINVAL, "out is null");
    *out = nullptr;
    if (n_slots < 1 || n_slots > 64) return fail(MAPPER_EINVAL, "n_slots must be in [1, 64]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(MAPPER_EINVAL, "no such device");
    auto S = std::make_unique<mapper_server>();
    S->device = device;
    if (hbm_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        cudaSetDevice(device);
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(MAPPER_ECUDA, "cudaMemGetInfo failed");
        hbm_budget_bytes = free_b / 10 * 8;
    }
    S->budget = hbm_budget_bytes;
    for (int i = 0; i < n_slots; ++i) S->workers.emplace_back(worker_main, S.get(), i);
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait(lk, [&] { return S->ready == n_slots; });
    }
    if (S->init_status != MAPPER_OK) {
        const int st = S->init_status;
        const std::string msg = S->init_error;
        mapper_server_destroy(S.release());
        return fail(st, "server slot: " + msg);
    }
    *out = S.release();
    return MAPPER_OK;
}

void mapper_server_destroy(mapper_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        // queued requests never start: complete them with an error status so
        // that their waiters return
        const Clock::time_point now = Clock::now();
        for (auto& r : S->queue) {
            r->t_start = r->t_end = now;
            r->status = MAPPER_ECANCELED;
            r->error = "request dropped: the server was destroyed before it started";
            r->done = true;
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    for (auto& t : S->workers) t.join();         // running requests finish
    {
        // every thread inside mapper_server_wait leaves before S goes away
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.notify_all();
        S->cv_done.wait(lk, [&] { return S->waiters == 0; });
    }
    for (auto& kv : S->requests)
        if (kv.second->graph) mapper_free(kv.second->graph);
    delete S;
}

int mapper_server_add_dataset(mapper_server* S, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                              int32_t* dataset_id)
{
    if (!S || !X_dev || !dataset_id) return fail(MAPPER_EINVAL, "null argument");
    if (n < 1 || d < 1 || ld < d) return fail(MAPPER_EINVAL, "bad dataset shape");
    std::lock_guard<std::mutex> lk(S->mu);
    S->datasets.push_back(Dataset{X_dev, n, d, ld});
    *dataset_id = (int32_t)S->datasets.size() - 1;
    return MAPPER_OK;
}

int mapper_server_submit(mapper_server* S, int32_t dataset_id, const mapper_params* p, int64_t* request_id)
{
    if (!S || !p || !request_id) return fail(MAPPER_EINVAL, "null argument");
    auto r = std::make_shared<Request>();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (dataset_id < 0 || dataset_id >= (int32_t)S->datasets.size()) return fail(MAPPER_EINVAL, "no such dataset");
        const Dataset& ds = S->datasets[dataset_id];
        size_t fp = 0;
        const int rc = mapper_graph_footprint(ds.n, ds.d, p, &fp);
        if (rc != MAPPER_OK) return rc;
        r->id = S->next_id++;
        r->dataset = ds;
        r->params = *p;
        r->footprint = fp;
        r->t_submit = Clock::now();
        S->requests[r->id] = r;
        S->queue.push_back(r);
        *request_id = r->id;
    }
    S->cv_work.notify_all();
    return MAPPER_OK;
}

int mapper_server_wait(mapper_server* S, int64_t request_id, double timeout_s, mapper_graph_t** out,
                       mapper_request_info* info)
{
    if (!S || !out) return fail(MAPPER_EINVAL, "null argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(request_id);
    if (it == S->requests.end()) return fail(MAPPER_EINVAL, "no such request (or already collected)");
    std::shared_ptr<Request> r = it->second;
    const auto pred = [&] { return r->done; };
    ++S->waiters;
    bool finished = true;
    if (timeout_s < 0) S->cv_done.wait(lk, pred);
    else finished = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
    --S->waiters;
    if (S->stopping && S->waiters == 0) S->cv_done.notify_all();    // destroy may be waiting for us
    if (!finished) return fail(MAPPER_ETIMEOUT, "request not finished within the timeout");
    S->requests.erase(r->id);
    if (info) {
        info->queue_s = secs(r->t_submit, r->t_start);
        info->run_s = secs(r->t_start, r->t_end);
        info->latency_s = secs(r->t_submit, r->t_end);
        info->footprint = r->footprint;
        info->status = r->status;
    }
    if (r->status != MAPPER_OK) return fail(r->status, r->error);
    *out = r->graph;
    return MAPPER_OK;
}

int mapper_server_load(mapper_server* S, int* running, int* queued, size_t* bytes_in_use)
{
    if (!S) return fail(MAPPER_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (running) *running = S->running;
    if (queued) *queued = (int)S->queue.size();
    if (bytes_in_use) *bytes_in_use = S->in_use;
    return MAPPER_OK;
}

}  // extern "C"
