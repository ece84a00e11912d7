// Serving: a request loop for streamed scans with continuous batching.
//
// Clients open scans and submit per-angle chunks of histories as they are
// acquired (the online mode of Sec. 4).  A worker thread admits scans while
// their device footprint fits a memory budget, and repeatedly gathers one
// pending chunk from each of up to max_batch admitted scans into a batched
// launch (one persistent traversal over all of them, see hd_batch).  Several
// such launches are kept queued on the GPU, so chunks that arrive while
// others are running join the next launch and the device stays busy.  A
// scan's hulls are computed right after its last chunk, in the same launch.
// The server uses only the public scan and batch calls.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "hd_internal.cuh"

namespace {

double now_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Chunk {
    float *dev = nullptr;  // six arrays of n floats, back to back
    int64_t n = 0;
    cudaEvent_t ready = nullptr;  // the upload has finished
};

struct SScan {
    int64_t id = 0;
    hd_geometry geom{};
    hd_params params{};
    int32_t n_chunks = 0;
    int32_t submitted = 0;
    int32_t issued = 0;   // chunks handed to a launch
    int32_t done_chunks = 0;
    int64_t histories = 0;
    size_t footprint = 0;
    int state = 0;        // 0 waiting, 1 admitted, 2 ready, 3 failed
    hd_status status = HD_OK;
    hd_scan *scan = nullptr;
    std::deque<Chunk> pending;
    double t_open = -1, t_admit = -1, t_first = -1, t_last = -1, t_ready = -1;
};

struct Tick {
    hd_batch *batch = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int64_t> scans;     // scans that had a chunk in this launch
    std::vector<bool> finishing;    // ... and whether it was their last
    std::vector<Chunk> chunks;      // buffers to release after the launch
    bool busy = false;
};

}  // namespace

struct hd_server {
    hd_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<int64_t, SScan> scans;
    std::deque<int64_t> waiting;  // admission queue (FIFO)
    std::vector<int64_t> admitted_order;
    size_t used = 0;
    int64_t next_id = 1;
    size_t rr = 0;  // round-robin position over admitted scans
    bool stop = false;
    cudaStream_t stream = nullptr;   // launches
    cudaStream_t upload = nullptr;   // chunk uploads
    std::vector<Tick> ticks;
    std::thread worker;
    hd_server_stats stats{};
};

namespace {

size_t footprint_of(const hd_geometry &g, const hd_server_config &cfg)
{
    const size_t V = static_cast<size_t>(g.nx) * g.ny * g.nz;
    // counts (2 x uint32), three byte masks, bit views, and the per-chunk
    // scratch: records (28 B) and up to eight packed pairs (64 B each)
    return V * 11 + V / 4 + static_cast<size_t>(cfg.max_chunk) * (28 + 8 * 64) + (4u << 20);
}

void release_chunk(Chunk &c, cudaStream_t st)
{
    if (c.dev) cudaFreeAsync(c.dev, st);
    if (c.ready) cudaEventDestroy(c.ready);
    c.dev = nullptr;
    c.ready = nullptr;
}

// Called with the lock held: retire finished launches.
void retire(hd_server *sv)
{
    for (auto &t : sv->ticks) {
        if (!t.busy) continue;
        const cudaError_t q = cudaEventQuery(t.done);
        if (q == cudaErrorNotReady) continue;
        const double now = now_since(sv->t0);
        for (size_t i = 0; i < t.scans.size(); ++i) {
            auto it = sv->scans.find(t.scans[i]);
            if (it == sv->scans.end()) continue;
            SScan &s = it->second;
            s.done_chunks += 1;
            if (q != cudaSuccess) {
                s.state = 3;
                s.status = HD_ERR_CUDA;
            } else if (t.finishing[i]) {
                s.state = 2;
                s.t_ready = now;
                sv->stats.scans_done += 1;
            }
        }
        if (q != cudaSuccess) cudaGetLastError();
        t.scans.clear();
        t.finishing.clear();
        t.chunks.clear();
        t.busy = false;
    }
    sv->cv_done.notify_all();
}

// Called with the lock held: admit waiting scans, first come first served.
void admit(hd_server *sv)
{
    while (!sv->waiting.empty()) {
        auto it = sv->scans.find(sv->waiting.front());
        if (it == sv->scans.end()) {
            sv->waiting.pop_front();
            continue;
        }
        SScan &s = it->second;
        if (sv->used + s.footprint > sv->cfg.hbm_budget_bytes) break;
        hd_scan *h = nullptr;
        const hd_status r = hd_scan_create(&s.geom, &s.params, &h);
        sv->waiting.pop_front();
        if (r != HD_OK) {
            s.state = 3;
            s.status = r;
            sv->cv_done.notify_all();
            continue;
        }
        s.scan = h;
        s.state = 1;
        s.t_admit = now_since(sv->t0);
        sv->used += s.footprint;
        sv->admitted_order.push_back(s.id);
        sv->stats.scans_admitted += 1;
    }
}

void worker_main(hd_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    while (!sv->stop) {
        retire(sv);
        admit(sv);
        Tick *slot = nullptr;
        for (auto &t : sv->ticks)
            if (!t.busy) {
                slot = &t;
                break;
            }
        bool any_busy = false;
        for (auto &t : sv->ticks) any_busy = any_busy || t.busy;
        // while a launch runs, let chunks of more scans gather first (a
        // scan's last chunk never waits for company)
        if (slot && any_busy) {
            int ready = 0;
            bool last_waiting = false;
            for (const int64_t id : sv->admitted_order) {
                const SScan &s = sv->scans[id];
                if (s.state != 1 || s.pending.empty()) continue;
                ++ready;
                if (s.submitted == s.n_chunks && s.issued + static_cast<int32_t>(s.pending.size()) ==
                                                     s.n_chunks &&
                    s.pending.size() == 1)
                    last_waiting = true;
            }
            if (ready < sv->cfg.min_batch && !last_waiting) slot = nullptr;
        }
        // gather at most one chunk per admitted scan, round-robin
        std::vector<std::pair<int64_t, Chunk>> take;
        std::vector<bool> finishing;
        if (slot) {
            const size_t na = sv->admitted_order.size();
            for (size_t k = 0; k < na && static_cast<int>(take.size()) < sv->cfg.max_batch; ++k) {
                const int64_t id = sv->admitted_order[(sv->rr + k) % na];
                auto it = sv->scans.find(id);
                if (it == sv->scans.end()) continue;
                SScan &s = it->second;
                if (s.state != 1 || s.pending.empty()) continue;
                take.push_back({id, s.pending.front()});
                s.pending.pop_front();
                s.issued += 1;
                finishing.push_back(s.issued == s.n_chunks);
            }
            if (na) sv->rr = (sv->rr + 1) % na;
        }
        if (take.empty()) {
            // nothing to launch: wait for work, or poll running launches
            if (any_busy) sv->cv_work.wait_for(lock, std::chrono::microseconds(200));
            else sv->cv_work.wait(lock);
            continue;
        }
        // issue the launch outside the lock
        const auto t_issue = std::chrono::steady_clock::now();
        std::vector<hd_scan *> handles;
        for (auto &tk : take) handles.push_back(sv->scans[tk.first].scan);
        lock.unlock();
        hd_status r = HD_OK;
        for (size_t i = 0; i < take.size() && r == HD_OK; ++i) {
            Chunk &c = take[i].second;
            if (cudaStreamWaitEvent(sv->stream, c.ready, 0) != cudaSuccess) r = HD_ERR_CUDA;
            const float *p = c.dev;
            const int64_t n = c.n;
            if (r == HD_OK)
                r = hd_batch_add_item(slot->batch, handles[i], p, p + n, p + 2 * n, p + 3 * n,
                                      p + 4 * n, p + 5 * n, n,
                                      finishing[i] ? HD_BATCH_FINALIZE : 0);
        }
        if (r == HD_OK) r = hd_batch_run(slot->batch, 0, sv->stream);
        for (auto &tk : take) release_chunk(tk.second, sv->stream);
        const cudaError_t e = cudaEventRecord(slot->done, sv->stream);
        lock.lock();
        slot->busy = true;
        for (size_t i = 0; i < take.size(); ++i) {
            slot->scans.push_back(take[i].first);
            slot->finishing.push_back(finishing[i] && r == HD_OK && e == cudaSuccess);
        }
        if (r != HD_OK || e != cudaSuccess) {
            for (auto &tk : take) {
                SScan &s = sv->scans[tk.first];
                s.state = 3;
                s.status = r != HD_OK ? r : HD_ERR_CUDA;
            }
        }
        sv->stats.launches += 1;
        sv->stats.chunks_launched += static_cast<int64_t>(take.size());
        sv->stats.issue_seconds +=
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_issue).count();
    }
}

}  // namespace

extern "C" {

hd_status hd_server_config_default(hd_server_config *out)
{
    if (!out) return HD_ERR_ARG;
    out->hbm_budget_bytes = size_t(64) << 30;
    out->max_chunk = 100000;
    out->max_batch = 64;
    out->max_in_flight = 2;
    out->min_batch = 8;
    return HD_OK;
}

hd_status hd_server_create(const hd_server_config *cfg, hd_server **out)
{
    if (!cfg || !out) return HD_ERR_ARG;
    *out = nullptr;
    if (cfg->max_chunk < 1 || cfg->max_batch < 1 || cfg->max_batch > hd::kMaxBatch ||
        cfg->max_in_flight < 1 || cfg->max_in_flight > 8 || cfg->hbm_budget_bytes == 0 ||
        cfg->min_batch < 1)
        return HD_ERR_ARG;
    hd_server *sv = new (std::nothrow) hd_server();
    if (!sv) return HD_ERR_NOMEM;
    sv->cfg = *cfg;
    sv->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->upload, cudaStreamNonBlocking);
    sv->ticks.resize(static_cast<size_t>(cfg->max_in_flight));
    for (auto &t : sv->ticks) {
        if (e != cudaSuccess) break;
        e = cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming);
        if (e == cudaSuccess && hd_batch_create(hd::kMaxBatch, &t.batch) != HD_OK) e = cudaErrorUnknown;
        if (e == cudaSuccess) hd_batch_set_graph(t.batch, 0);  // a new shape every launch
    }
    if (e != cudaSuccess) {
        hd_server_destroy(sv);
        return HD_ERR_CUDA;
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return HD_OK;
}

hd_status hd_server_destroy(hd_server *sv)
{
    if (!sv) return HD_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    if (sv->stream) cudaStreamSynchronize(sv->stream);
    if (sv->upload) cudaStreamSynchronize(sv->upload);
    for (auto &kv : sv->scans) {
        for (auto &c : kv.second.pending) release_chunk(c, sv->stream);
        if (kv.second.scan) hd_scan_destroy(kv.second.scan);
    }
    for (auto &t : sv->ticks) {
        if (t.batch) hd_batch_destroy(t.batch);
        if (t.done) cudaEventDestroy(t.done);
    }
    if (sv->stream) {
        cudaStreamSynchronize(sv->stream);
        cudaStreamDestroy(sv->stream);
    }
    if (sv->upload) cudaStreamDestroy(sv->upload);
    if (prev >= 0) cudaSetDevice(prev);
    delete sv;
    return HD_OK;
}

hd_status hd_server_open_scan(hd_server *sv, const hd_geometry *geom, const hd_params *params,
                              int32_t n_chunks, int64_t *scan_id)
{
    if (!sv || !geom || !params || !scan_id || n_chunks < 1) return HD_ERR_ARG;
    SScan s;
    s.geom = *geom;
    s.params = *params;
    s.n_chunks = n_chunks;
    s.footprint = footprint_of(*geom, sv->cfg);
    if (s.footprint > sv->cfg.hbm_budget_bytes) return HD_ERR_ADMISSION;
    std::lock_guard<std::mutex> lock(sv->mu);
    s.id = sv->next_id++;
    s.t_open = now_since(sv->t0);
    *scan_id = s.id;
    sv->scans[s.id] = std::move(s);
    sv->waiting.push_back(*scan_id);
    sv->stats.scans_opened += 1;
    sv->cv_work.notify_all();
    return HD_OK;
}

hd_status hd_server_submit_chunk(hd_server *sv, int64_t scan_id, const float *angle_deg,
                                 const float *u_in, const float *v_in, const float *u_out,
                                 const float *v_out, const float *wepl, int64_t n,
                                 int32_t on_device)
{
    if (!sv || n < 1 || n > sv->cfg.max_chunk) return HD_ERR_ARG;
    if (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl) return HD_ERR_ARG;
    const auto t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->scans.find(scan_id);
        if (it == sv->scans.end()) return HD_ERR_ARG;
        if (it->second.state >= 2 || it->second.submitted >= it->second.n_chunks)
            return HD_ERR_STATE;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != sv->device) cudaSetDevice(sv->device);
    Chunk c;
    c.n = n;
    const float *src[6] = {angle_deg, u_in, v_in, u_out, v_out, wepl};
    // each client thread uploads on its own per-thread stream, so uploads
    // from several threads proceed side by side
    const cudaStream_t up = cudaStreamPerThread;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&c.dev), sizeof(float) * 6 * n, up);
    for (int a = 0; e == cudaSuccess && a < 6; ++a)
        e = cudaMemcpyAsync(c.dev + a * n, src[a], sizeof(float) * n,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c.ready, up);
    // the caller may reuse its buffers as soon as this call returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(up);
    if (prev >= 0 && prev != sv->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c.dev) cudaFreeAsync(c.dev, up);
        if (c.ready) cudaEventDestroy(c.ready);
        return HD_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->scans.find(scan_id);
    if (it == sv->scans.end()) {
        release_chunk(c, sv->upload);
        return HD_ERR_ARG;
    }
    SScan &s = it->second;
    const double now = now_since(sv->t0);
    if (s.submitted == 0) s.t_first = now;
    s.submitted += 1;
    if (s.submitted == s.n_chunks) s.t_last = now;
    s.histories += n;
    s.pending.push_back(c);
    sv->stats.chunks_submitted += 1;
    sv->stats.submit_seconds +=
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_submit).count();
    sv->cv_work.notify_all();
    return HD_OK;
}

hd_status hd_server_poll(hd_server *sv, int64_t scan_id, int32_t *done, hd_status *scan_status)
{
    if (!sv || !done) return HD_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->scans.find(scan_id);
    if (it == sv->scans.end()) return HD_ERR_ARG;
    *done = it->second.state >= 2 ? 1 : 0;
    if (scan_status) *scan_status = it->second.status;
    return HD_OK;
}

hd_status hd_server_wait(hd_server *sv, int64_t scan_id, int64_t timeout_ms)
{
    if (!sv || timeout_ms < 0) return HD_ERR_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    auto ready = [&]() {
        auto it = sv->scans.find(scan_id);
        return it == sv->scans.end() || it->second.state >= 2;
    };
    if (!sv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready))
        return HD_ERR_TIMEOUT;
    auto it = sv->scans.find(scan_id);
    if (it == sv->scans.end()) return HD_ERR_ARG;
    return it->second.state == 2 ? HD_OK : it->second.status;
}

hd_status hd_server_scan(hd_server *sv, int64_t scan_id, hd_scan **out)
{
    if (!sv || !out) return HD_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->scans.find(scan_id);
    if (it == sv->scans.end()) return HD_ERR_ARG;
    if (it->second.state != 2) return HD_ERR_STATE;
    *out = it->second.scan;
    return HD_OK;
}

hd_status hd_server_get_info(hd_server *sv, int64_t scan_id, hd_server_scan_info *out)
{
    if (!sv || !out) return HD_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->scans.find(scan_id);
    if (it == sv->scans.end()) return HD_ERR_ARG;
    const SScan &s = it->second;
    out->t_open = s.t_open;
    out->t_admit = s.t_admit;
    out->t_first_chunk = s.t_first;
    out->t_last_chunk = s.t_last;
    out->t_ready = s.t_ready;
    out->histories = s.histories;
    out->chunks_submitted = s.submitted;
    out->chunks_done = s.done_chunks;
    out->state = s.state;
    return HD_OK;
}

hd_status hd_server_get_stats(hd_server *sv, hd_server_stats *out)
{
    if (!sv || !out) return HD_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->stats;
    out->bytes_in_use = static_cast<int64_t>(sv->used);
    return HD_OK;
}

hd_status hd_server_close_scan(hd_server *sv, int64_t scan_id)
{
    if (!sv) return HD_ERR_ARG;
    hd_scan *h = nullptr;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->scans.find(scan_id);
        if (it == sv->scans.end()) return HD_ERR_ARG;
        SScan &s = it->second;
        if (s.state == 1 && s.done_chunks < s.issued) return HD_ERR_STATE;  // still running
        if (s.state == 1 && !s.pending.empty()) return HD_ERR_STATE;
        for (auto &c : s.pending) release_chunk(c, sv->upload);
        h = s.scan;
        if (s.state >= 1 && h) sv->used -= s.footprint;
        for (auto ai = sv->admitted_order.begin(); ai != sv->admitted_order.end(); ++ai)
            if (*ai == scan_id) {
                sv->admitted_order.erase(ai);
                break;
            }
        for (auto wi = sv->waiting.begin(); wi != sv->waiting.end(); ++wi)
            if (*wi == scan_id) {
                sv->waiting.erase(wi);
                break;
            }
        sv->scans.erase(it);
    }
    if (h) hd_scan_destroy(h);
    sv->cv_work.notify_all();
    return HD_OK;
}

}  // extern "C"
