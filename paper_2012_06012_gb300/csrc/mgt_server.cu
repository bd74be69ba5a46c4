// Serving loop: a host scheduler thread that admits transpose requests by
// their HBM footprint and keeps the GPU busy with several in flight at once.
//
// A request is (plan, input, output) on caller-owned device buffers.  Its
// footprint is the workspace the server allocates for it plus its input and
// output bytes; requests are admitted in arrival order while the in-flight
// footprint stays within the budget and a slot is free, so requests that
// arrive while others run start as soon as slots and memory free up
// (continuous batching).  Small queued requests with the same kernel
// formats are fused into one batched launch (one launch per phase for all
// of them).  Launches spread over the server's streams; workspaces come from
// a stream-ordered memory pool that keeps its memory resident.  Completion
// is signalled by a host function on the stream, which stamps the time:
// latency = completion - submission.
#include "mgt_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace mgt;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kFuseMaxParts = 64;  // fused members: at most this many row blocks

struct Req {
    uint64_t ticket = 0;
    mgt_plan_t *plan = nullptr;
    mgt_xcsr_in in{};
    mgt_xcsr_out out{};
    size_t footprint = 0;   // workspace + input + output bytes
    size_t ws_bytes = 0;
    long long bytes = 0;    // minimal bytes moved (input once + output once)
    double t_submit = 0;
    int slot = -1;          // index of its status word in pinned memory
    bool done = false;
    int status = MGT_OK;
    double latency_ms = 0;
};

struct Launch {
    mgt_server_t *server = nullptr;
    std::vector<uint64_t> tickets;
    size_t footprint = 0;
    int stream = 0;
    int staging = -1;       // pinned staging buffer of a fused launch
    double t_done = 0;
    std::atomic<bool> done{false};
};

}  // namespace

struct mgt_server_s {
    mgt_server_cfg cfg{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_load;
    cudaMemPool_t pool = nullptr;
    unsigned *status_pinned = nullptr;  // one word per slot
    std::vector<int> free_slots;
    std::vector<void *> staging;        // pinned tables of fused launches
    std::vector<int> free_staging;
    size_t staging_bytes = 0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;                       // waiting tickets, arrival order
    std::unordered_map<uint64_t, Req> reqs;           // every ticket not yet collected
    std::vector<Launch *> inflight;
    uint64_t next_ticket = 1;
    size_t inflight_bytes = 0;
    int inflight_reqs = 0;
    bool stop = false;
    double wake_at = 0;  // end of a pending batching window
    std::thread worker;

    // statistics
    mgt_server_stats stats{};
    std::vector<double> lat;                          // completed latencies (ms)
    double t_first = 0, t_last = 0;
};

namespace {

// Runs on CUDA's callback thread when the stream reaches the end of the
// launch: no CUDA calls and no lock here (the scheduler holds its lock
// while it enqueues work); it also polls, so a missed wake-up only delays
// admission, never the time stamp.
void CUDART_CB on_done(void *arg) {
    Launch *l = static_cast<Launch *>(arg);
    l->t_done = now_s();
    l->done.store(true, std::memory_order_release);
    l->server->cv.notify_all();
}

int pick_stream(mgt_server_t *s) {
    int best = 0;
    for (int i = 1; i < (int)s->streams.size(); ++i)
        if (s->stream_load[i] < s->stream_load[best]) best = i;
    return best;
}

// Enqueues one launch for reqs (all admitted); called with the lock held.
int start_launch(mgt_server_t *s, const std::vector<uint64_t> &tickets) {
    Launch *l = new (std::nothrow) Launch;
    if (!l) return MGT_ENOMEM;
    l->server = s;
    l->tickets = tickets;
    l->stream = pick_stream(s);
    cudaStream_t st = s->streams[l->stream];
    const int n = (int)tickets.size();
    std::vector<mgt_plan_t *> plans(n);
    std::vector<mgt_xcsr_in> ins(n);
    std::vector<mgt_xcsr_out> outs(n);
    for (int k = 0; k < n; ++k) {
        Req &r = s->reqs[tickets[k]];
        plans[k] = r.plan;
        ins[k] = r.in;
        outs[k] = r.out;
        l->footprint += r.footprint;
    }
    size_t ws_bytes = 0;
    int rc = MGT_OK;
    if (n == 1) ws_bytes = align256(plans[0]->L.total);
    else rc = mgt_batched_workspace(n, plans.data(), &ws_bytes);
    void *raw = nullptr, *ws = nullptr;
    if (rc == MGT_OK) {
        const cudaError_t e = cudaMallocFromPoolAsync(&raw, std::max<size_t>(ws_bytes, 256) + 256, s->pool, st);
        if (e != cudaSuccess) rc = note_cuda(e, "server workspace");
        else ws = reinterpret_cast<void *>(align256(reinterpret_cast<uintptr_t>(raw)));
    }
    if (rc == MGT_OK) {
        if (n == 1) {
            rc = mgt_transpose(plans[0], &ins[0], &outs[0], ws, ws_bytes, st);
        } else {
            l->staging = s->free_staging.back();
            s->free_staging.pop_back();
            rc = batched_enqueue(n, plans.data(), ins.data(), outs.data(), ws, ws_bytes, st,
                                 s->staging[l->staging], s->staging_bytes);
        }
    }
    // device status words -> pinned slots (member k's header is at the
    // start of its workspace: the whole workspace alone, else after the tables)
    if (rc == MGT_OK) {
        size_t off = n == 1 ? 0 : batched_table_bytes(n, plans.data());
        for (int k = 0; k < n && rc == MGT_OK; ++k) {
            Req &r = s->reqs[tickets[k]];
            const cudaError_t e = cudaMemcpyAsync(&s->status_pinned[r.slot], static_cast<char *>(ws) + off,
                                                  sizeof(unsigned), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) rc = note_cuda(e, "server status");
            off += align256(plans[k]->L.total);
        }
    }
    if (raw) cudaFreeAsync(raw, st);
    if (rc == MGT_OK) {
        const cudaError_t e = cudaLaunchHostFunc(st, on_done, l);
        if (e != cudaSuccess) rc = note_cuda(e, "server completion");
    }
    if (rc != MGT_OK) {
        // nothing of this launch will signal: finish its requests here
        const double t = now_s();
        for (uint64_t tk : tickets) {
            Req &r = s->reqs[tk];
            r.done = true;
            r.status = rc;
            r.latency_ms = (t - r.t_submit) * 1e3;
            s->free_slots.push_back(r.slot);
            s->inflight_reqs -= 1;
            s->stats.failed += 1;
        }
        s->inflight_bytes -= l->footprint;
        if (l->staging >= 0) s->free_staging.push_back(l->staging);
        delete l;
        return rc;
    }
    s->stream_load[l->stream] += 1;
    s->inflight.push_back(l);
    s->stats.launches += 1;
    return MGT_OK;
}

void finish_launches(mgt_server_t *s) {
    for (size_t i = 0; i < s->inflight.size();) {
        Launch *l = s->inflight[i];
        if (!l->done.load(std::memory_order_acquire)) {
            ++i;
            continue;
        }
        for (uint64_t tk : l->tickets) {
            Req &r = s->reqs[tk];
            const unsigned bits = s->status_pinned[r.slot];
            r.status = (bits & ST_BADINPUT) ? MGT_EBADINPUT
                       : (bits & (ST_OVERFLOW | ST_DEBUG_BOUNDS)) ? MGT_EOVERFLOW
                       : (bits & ST_TIMEOUT)  ? MGT_ETIMEOUT
                                              : MGT_OK;
            r.latency_ms = (l->t_done - r.t_submit) * 1e3;
            r.done = true;
            s->free_slots.push_back(r.slot);
            s->inflight_reqs -= 1;
            s->stats.completed += 1;
            if (r.status != MGT_OK) s->stats.failed += 1;
            s->stats.bytes += (uint64_t)r.bytes;
            s->lat.push_back(r.latency_ms);
            if (s->t_first == 0) s->t_first = r.t_submit;
            s->t_last = l->t_done;
        }
        s->inflight_bytes -= l->footprint;
        s->stream_load[l->stream] -= 1;
        if (l->staging >= 0) s->free_staging.push_back(l->staging);
        delete l;
        s->inflight[i] = s->inflight.back();
        s->inflight.pop_back();
    }
}

// Admits queued requests in arrival order while slots and memory allow;
// fuses runs of small ones with the same kernel formats.
void admit(mgt_server_t *s) {
    const int slots = s->cfg.max_slots;
    while (!s->queue.empty() && s->inflight_reqs < slots && !s->free_slots.empty()) {
        Req &head = s->reqs[s->queue.front()];
        if (s->inflight_bytes + head.footprint > s->cfg.hbm_budget_bytes) break;
        std::vector<uint64_t> group{s->queue.front()};
        size_t fp = head.footprint;
        const bool small = head.plan->p.C <= s->cfg.fuse_max_cells && head.plan->p.P <= kFuseMaxParts;
        if (small && s->cfg.batch_max > 1 && s->cfg.batch_window_us > 0) {
            // batching window: a small head waits (up to the window) for
            // batch_max - 1 compatible requests to queue behind it
            const unsigned long long key = batch_group_key(head.plan->p);
            int run = 1;
            for (size_t q = 1; q < s->queue.size() && run < s->cfg.batch_max; ++q, ++run) {
                const Req &r = s->reqs[s->queue[q]];
                if (r.plan->p.C > s->cfg.fuse_max_cells || r.plan->p.P > kFuseMaxParts ||
                    batch_group_key(r.plan->p) != key)
                    break;
            }
            const double due = head.t_submit + 1e-6 * s->cfg.batch_window_us;
            if (run < s->cfg.batch_max && now_s() < due) {
                s->wake_at = due;
                break;
            }
        }
        if (small && s->cfg.batch_max > 1 && !s->free_staging.empty()) {
            const unsigned long long key = batch_group_key(head.plan->p);
            for (size_t q = 1; q < s->queue.size() && (int)group.size() < s->cfg.batch_max; ++q) {
                Req &r = s->reqs[s->queue[q]];
                if (r.plan->p.C > s->cfg.fuse_max_cells || r.plan->p.P > kFuseMaxParts ||
                    batch_group_key(r.plan->p) != key)
                    break;
                if ((int)group.size() + s->inflight_reqs >= slots ||
                    group.size() >= s->free_slots.size())
                    break;
                if (s->inflight_bytes + fp + r.footprint > s->cfg.hbm_budget_bytes) break;
                group.push_back(s->queue[q]);
                fp += r.footprint;
            }
        }
        for (size_t k = 0; k < group.size(); ++k) s->queue.pop_front();
        for (uint64_t tk : group) {
            Req &r = s->reqs[tk];
            r.slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->inflight_reqs += 1;
        }
        s->inflight_bytes += fp;
        s->stats.peak_inflight_bytes = std::max<uint64_t>(s->stats.peak_inflight_bytes, s->inflight_bytes);
        s->stats.peak_inflight_requests =
            std::max<uint64_t>(s->stats.peak_inflight_requests, (uint64_t)s->inflight_reqs);
        if (group.size() > 1) s->stats.fused_requests += group.size();
        start_launch(s, group);
    }
}

void worker_main(mgt_server_t *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        finish_launches(s);
        if (s->stop && s->inflight.empty() && s->queue.empty()) break;
        s->wake_at = 0;
        admit(s);
        double wait = 5e-3;
        if (s->wake_at > 0) wait = std::max(0.0, std::min(wait, s->wake_at - now_s()));
        s->cv.wait_for(lk, std::chrono::duration<double>(wait));
    }
}

}  // namespace

extern "C" {

int mgt_server_create(const mgt_server_cfg *cfg, mgt_server_t **server) {
    if (!cfg || !server) return MGT_EINVAL;
    *server = nullptr;
    if (cfg->hbm_budget_bytes == 0 || cfg->max_slots < 1 || cfg->n_streams < 1 ||
        cfg->max_queue < 1 || cfg->batch_max < 1 || cfg->max_slots > 4096 || cfg->n_streams > 64 ||
        cfg->batch_max > 256 || cfg->batch_window_us < 0 || cfg->batch_window_us > 1000000)
        return MGT_EINVAL;
    mgt_server_t *s = new (std::nothrow) mgt_server_t;
    if (!s) return MGT_ENOMEM;
    s->cfg = *cfg;
    int rc = MGT_OK;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) rc = note_cuda(e, "server device");
    for (int i = 0; rc == MGT_OK && i < cfg->n_streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = note_cuda(e, "server stream");
        else s->streams.push_back(st);
    }
    s->stream_load.assign(s->streams.size(), 0);
    if (rc == MGT_OK) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        e = cudaMemPoolCreate(&s->pool, &props);
        if (e != cudaSuccess) rc = note_cuda(e, "server pool");
    }
    if (rc == MGT_OK) {
        unsigned long long keep = ~0ull;  // keep freed workspaces resident
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) rc = note_cuda(e, "server pool");
    }
    if (rc == MGT_OK) {
        e = cudaMallocHost((void **)&s->status_pinned, sizeof(unsigned) * cfg->max_slots);
        if (e != cudaSuccess) rc = note_cuda(e, "server status");
    }
    // pinned table staging for fused launches: one per possible launch
    if (rc == MGT_OK && cfg->batch_max > 1) {
        // bound on a fused batch's table region (see mgt_batched_workspace)
        const size_t bm = (size_t)cfg->batch_max;
        s->staging_bytes = batched_table_bound((int)bm, kFuseMaxParts);
        const int nst = std::min(cfg->max_slots, 64);
        for (int i = 0; rc == MGT_OK && i < nst; ++i) {
            void *p = nullptr;
            e = cudaMallocHost(&p, s->staging_bytes);
            if (e != cudaSuccess) rc = note_cuda(e, "server staging");
            else {
                s->staging.push_back(p);
                s->free_staging.push_back(i);
            }
        }
    }
    for (int i = cfg->max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    if (rc == MGT_OK) {
        try {
            s->worker = std::thread(worker_main, s);
        } catch (...) {
            rc = MGT_ENOMEM;
        }
    }
    if (rc != MGT_OK) {
        mgt_server_destroy(s);
        return rc;
    }
    *server = s;
    return MGT_OK;
}

int mgt_submit(mgt_server_t *s, mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out,
               uint64_t *ticket) {
    if (!s || !plan || !in || !out || !ticket) return MGT_EINVAL;
    const Params &p = plan->p;
    if (p.var) return MGT_EINVAL;  // variable-width plans are not served
    if (!in->row_ptr || !in->cell_ptr || !out->row_ptr || !out->cell_ptr) return MGT_EINVAL;
    if (p.C > 0 && (!in->col_idx || !out->col_idx)) return MGT_EINVAL;
    if (p.V > 0 && (!in->values || !out->values)) return MGT_EINVAL;
    if ((out->part_cells == nullptr) != (out->part_values == nullptr)) return MGT_EINVAL;
    Req r;
    r.plan = plan;
    r.in = *in;
    r.out = *out;
    r.ws_bytes = align256(plan->L.total);
    r.bytes = mgt_minimal_bytes(&plan->desc);
    r.footprint = r.ws_bytes + (size_t)std::max<long long>(r.bytes, 0);
    if (r.footprint > s->cfg.hbm_budget_bytes) return MGT_ENOMEM;  // could never be admitted
    r.t_submit = now_s();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return MGT_EINVAL;
        if ((int)s->queue.size() >= s->cfg.max_queue) {
            s->stats.rejected += 1;
            return MGT_EAGAIN;
        }
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->queue.push_back(r.ticket);
        s->reqs.emplace(r.ticket, r);
        s->stats.submitted += 1;
    }
    s->cv.notify_all();
    return MGT_OK;
}

int mgt_poll(mgt_server_t *s, uint64_t ticket, int *done, int *status, double *latency_ms) {
    if (!s || !done) return MGT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return MGT_ENOTFOUND;
    *done = it->second.done ? 1 : 0;
    if (it->second.done) {
        if (status) *status = it->second.status;
        if (latency_ms) *latency_ms = it->second.latency_ms;
        s->reqs.erase(it);  // collected
    }
    return MGT_OK;
}

int mgt_server_drain(mgt_server_t *s) {
    if (!s) return MGT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->queue.empty() || !s->inflight.empty()) {
        s->cv.notify_all();
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
    return MGT_OK;
}

int mgt_server_get_stats(mgt_server_t *s, mgt_server_stats *out) {
    if (!s || !out) return MGT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    out->inflight_bytes = s->inflight_bytes;
    out->queued = s->queue.size();
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        auto q = [&](double f) {
            size_t k = (size_t)(f * (double)(v.size() - 1) + 0.5);
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        double m = 0;
        for (double x : s->lat) m += x;
        out->mean_ms = m / (double)s->lat.size();
        out->span_s = s->t_last - s->t_first;
    }
    return MGT_OK;
}

int mgt_server_reset_stats(mgt_server_t *s) {
    if (!s) return MGT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    s->stats = mgt_server_stats{};
    s->lat.clear();
    s->t_first = s->t_last = 0;
    return MGT_OK;
}

void mgt_server_destroy(mgt_server_t *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->status_pinned) cudaFreeHost(s->status_pinned);
    for (void *p : s->staging) cudaFreeHost(p);
    delete s;
}

}  // extern "C"
