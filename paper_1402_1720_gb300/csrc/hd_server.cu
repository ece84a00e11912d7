// Serving: a request loop for streamed scans with continuous batching.
//
// Clients open scans and submit per-angle chunks of histories as they are
// acquired (the online mode of Sec. 4).  A submit copies its chunk into the
// scan's open staging segment: a recycled device buffer that holds six
// structure-of-arrays columns of up to segment_histories histories, so the
// chunks of one scan that arrive while the GPU is busy sit side by side.  A
// worker thread admits scans while their device footprint fits a memory
// budget, and repeatedly takes the oldest filled segment of each of up to
// max_batch admitted scans into one batched launch (one persistent traversal
// over all of them, see hd_batch): however many chunks a scan received
// meanwhile, they go to the GPU as one item.  Several launches are kept
// queued, so the device stays busy while chunks gather for the next one.  A
// scan's hulls are computed in the launch that carries its last chunk.
// Staging memory is bounded: a submit that finds no free segment waits (for
// at most submit_timeout_ms) until a launch finishes and returns its
// segments.  The server uses only the public scan and batch calls.
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
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

// One staging segment: columns angle, u_in, v_in, u_out, v_out, wepl of cap
// floats each, back to back.  Submits reserve [reserved, reserved + n) under
// the server lock and copy outside it; the worker takes a segment only when
// no copy into it is running (writers == 0), so [0, filled) is complete.
struct Segment {
    float *dev = nullptr;
    int64_t reserved = 0;
    int64_t filled = 0;
    int32_t chunks = 0;   // chunks whose copies have finished
    int32_t writers = 0;  // copies running
    bool sealed = false;  // takes no more reservations
};

struct SScan {
    int64_t id = 0;
    hd_geometry geom{};
    hd_params params{};
    int32_t n_chunks = 0;
    int32_t reserved_chunks = 0;  // submits that got space (running or done)
    int32_t submitted = 0;        // submits whose copies have finished
    int32_t issued = 0;           // chunks handed to a launch
    int32_t done_chunks = 0;
    int64_t histories = 0;
    size_t footprint = 0;
    int state = 0;  // 0 waiting, 1 admitted, 2 ready, 3 failed
    bool admitting = false;  // its device state is being created
    hd_status status = HD_OK;
    hd_scan *scan = nullptr;
    std::deque<std::unique_ptr<Segment>> segs;  // oldest first; the back may be open
    double t_open = -1, t_admit = -1, t_first = -1, t_last = -1, t_ready = -1;
};

struct Tick {
    hd_batch *batch = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int64_t> scans;     // scans that had an item in this launch
    std::vector<int32_t> chunks;    // ... how many chunks it carried
    std::vector<bool> finishing;    // ... and whether it carried the scan's last
    std::vector<float *> bufs;      // staging segments to recycle after the launch
    bool busy = false;
};

}  // namespace

struct hd_server {
    hd_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_space, cv_keep;
    std::map<int64_t, SScan> scans;
    std::deque<int64_t> waiting;  // admission queue (FIFO)
    std::vector<int64_t> admitted_order;
    size_t used = 0;
    int64_t next_id = 1;
    size_t rr = 0;  // round-robin position over admitted scans
    bool stop = false;
    cudaStream_t stream = nullptr;  // launches
    std::vector<float *> free_bufs;  // staging segments not in use
    std::vector<float *> all_bufs;   // every staging segment allocated
    int allocating = 0;              // segments being allocated (outside the lock)
    std::vector<hd_scan *> graveyard;  // closed scans to destroy
    struct Pooled {
        hd_geometry geom;
        hd_params params;
        hd_scan *scan;
        size_t footprint;
    };
    std::deque<Pooled> pool;  // closed scans kept for reuse, oldest first
    size_t pooled = 0;        // their footprint (part of `used`)
    std::vector<Tick> ticks;
    std::thread worker;  // launches
    std::thread keeper;  // creates admitted scans and destroys closed ones
    hd_server_stats stats{};
};

namespace {

size_t segment_bytes(const hd_server_config &cfg)
{
    return sizeof(float) * 6 * static_cast<size_t>(cfg.segment_histories);
}

size_t footprint_of(const hd_geometry &g, const hd_server_config &cfg)
{
    const size_t V = static_cast<size_t>(g.nx) * g.ny * g.nz;
    // counts (2 x uint32), three byte masks, bit views, and the scratch of
    // one segment-sized item: records (28 B) and up to eight packed pairs
    // (64 B each) per history
    return V * 11 + V / 4 + static_cast<size_t>(cfg.segment_histories) * (28 + 8 * 64) +
           (4u << 20);
}

// The calling thread's upload stream on `device`: non-blocking, so uploads
// from several client threads proceed side by side and never wait for work
// on the legacy default stream.  Created on first use, destroyed when the
// thread exits.
struct UploadStreams {
    std::map<int, cudaStream_t> by_device;
    ~UploadStreams()
    {
        for (auto &kv : by_device) cudaStreamDestroy(kv.second);
    }
};

cudaStream_t upload_stream(int device)
{
    thread_local UploadStreams streams;
    auto it = streams.by_device.find(device);
    if (it != streams.by_device.end()) return it->second;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    streams.by_device[device] = st;
    return st;
}

// Called with the lock held: a staging segment from the free list, or
// nullptr.
float *pop_free_buffer(hd_server *sv)
{
    if (sv->free_bufs.empty()) return nullptr;
    float *b = sv->free_bufs.back();
    sv->free_bufs.pop_back();
    return b;
}

// Called with the lock held: return the segments of a scan that will not
// run (failed or closed) to the free list.
void recycle_segments(hd_server *sv, SScan &s)
{
    for (auto &g : s.segs)
        if (g->dev && g->writers == 0) sv->free_bufs.push_back(g->dev);
    s.segs.clear();
    sv->cv_space.notify_all();
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
            s.done_chunks += t.chunks[i];
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
        for (float *b : t.bufs) sv->free_bufs.push_back(b);
        t.scans.clear();
        t.chunks.clear();
        t.finishing.clear();
        t.bufs.clear();
        t.busy = false;
    }
    sv->cv_done.notify_all();
    sv->cv_space.notify_all();
}

bool same_config(const hd_geometry &a, const hd_geometry &b, const hd_params &p,
                 const hd_params &q)
{
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.sx == b.sx && a.sy == b.sy &&
           a.sz == b.sz && a.tracker_half_sep_mm == b.tracker_half_sep_mm &&
           p.wepl_miss_lt == q.wepl_miss_lt && p.wepl_hit_gt == q.wepl_hit_gt &&
           p.msc_nt == q.msc_nt && p.msc_nbhd == q.msc_nbhd && p.sm_ge == q.sm_ge &&
           p.sm_per_slice == q.sm_per_slice && p.methods == q.methods;
}

// Admission and clean-up, on their own thread so that allocating or
// freeing a scan's device memory (which may wait for the GPU) stalls
// neither the launches nor the submits: scans are admitted first come,
// first served while their footprint fits the budget.
void keeper_main(hd_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    while (!sv->stop) {
        if (!sv->graveyard.empty()) {
            std::vector<hd_scan *> dead;
            dead.swap(sv->graveyard);
            lock.unlock();
            for (hd_scan *h : dead) hd_scan_destroy(h);
            lock.lock();
            continue;
        }
        // the first waiting scan: a pooled scan of the same geometry and
        // parameters is reset and reused; otherwise a new one is created once
        // its footprint fits (evicting pooled scans, oldest first, if needed)
        int64_t id = -1;
        hd_scan *reuse = nullptr;
        while (!sv->waiting.empty()) {
            auto it = sv->scans.find(sv->waiting.front());
            if (it == sv->scans.end()) {
                sv->waiting.pop_front();
                continue;
            }
            SScan &s = it->second;
            for (auto pi = sv->pool.begin(); pi != sv->pool.end(); ++pi)
                if (same_config(pi->geom, s.geom, pi->params, s.params)) {
                    reuse = pi->scan;
                    sv->pooled -= pi->footprint;  // stays in `used`, now for this scan
                    sv->pool.erase(pi);
                    break;
                }
            if (!reuse && sv->used + s.footprint > sv->cfg.hbm_budget_bytes && !sv->pool.empty()) {
                const auto victim = sv->pool.front();
                sv->pool.pop_front();
                sv->pooled -= victim.footprint;
                sv->used -= victim.footprint;
                sv->graveyard.push_back(victim.scan);
                continue;
            }
            if (reuse || sv->used + s.footprint <= sv->cfg.hbm_budget_bytes) {
                id = s.id;
                sv->waiting.pop_front();
                s.admitting = true;
                if (!reuse) sv->used += s.footprint;
            }
            break;
        }
        if (id < 0) {
            if (!sv->graveyard.empty()) continue;  // evicted scans to destroy first
            sv->cv_keep.wait(lock);
            continue;
        }
        const hd_geometry geom = sv->scans[id].geom;
        const hd_params params = sv->scans[id].params;
        lock.unlock();
        hd_scan *h = reuse;
        hd_status r = HD_OK;
        const cudaStream_t ks = upload_stream(sv->device);
        if (reuse) {
            r = hd_scan_reset(h, ks);
            if (r == HD_OK && cudaStreamSynchronize(ks) != cudaSuccess) r = HD_ERR_CUDA;
        } else {
            r = hd_scan_create(&geom, &params, &h);
            // scratch for a full segment now, so launches never grow it
            if (r == HD_OK) r = hd_scan_reserve(h, sv->cfg.segment_histories, ks);
        }
        lock.lock();
        SScan &s = sv->scans[id];  // not closed while admitting
        s.admitting = false;
        if (r != HD_OK) {
            if (h) sv->graveyard.push_back(h);
            sv->used -= s.footprint;
            s.state = 3;
            s.status = r;
            sv->cv_done.notify_all();
            continue;
        }
        s.scan = h;
        s.state = 1;
        s.t_admit = now_since(sv->t0);
        sv->admitted_order.push_back(id);
        sv->stats.scans_admitted += 1;
        if (reuse) sv->stats.scans_reused += 1;
        sv->cv_work.notify_all();
    }
}

// A segment the worker may launch now.
bool takeable(const SScan &s)
{
    if (s.state != 1 || s.segs.empty()) return false;
    const Segment &g = *s.segs.front();
    return g.writers == 0 && g.filled > 0;
}

void worker_main(hd_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    const int64_t cap = sv->cfg.segment_histories;
    while (!sv->stop) {
        retire(sv);
        Tick *slot = nullptr;
        for (auto &t : sv->ticks)
            if (!t.busy) {
                slot = &t;
                break;
            }
        bool any_busy = false;
        for (auto &t : sv->ticks) any_busy = any_busy || t.busy;
        // while a launch runs, let work of more scans gather first (a scan
        // whose last chunk has landed never waits for company)
        if (slot && any_busy) {
            int ready = 0;
            bool last_waiting = false;
            for (const int64_t id : sv->admitted_order) {
                const SScan &s = sv->scans[id];
                if (!takeable(s)) continue;
                ++ready;
                if (s.submitted == s.n_chunks) last_waiting = true;
            }
            if (ready < sv->cfg.min_batch && !last_waiting) slot = nullptr;
        }
        // take the oldest filled segment of each admitted scan, round-robin
        struct Take {
            int64_t id;
            hd_scan *handle;
            float *dev;
            int64_t n;
            int32_t chunks;
            bool finishing;
        };
        std::vector<Take> take;
        if (slot) {
            const size_t na = sv->admitted_order.size();
            for (size_t k = 0; k < na && static_cast<int>(take.size()) < sv->cfg.max_batch; ++k) {
                const int64_t id = sv->admitted_order[(sv->rr + k) % na];
                auto it = sv->scans.find(id);
                if (it == sv->scans.end()) continue;
                SScan &s = it->second;
                if (!takeable(s)) continue;
                std::unique_ptr<Segment> g = std::move(s.segs.front());
                s.segs.pop_front();
                s.issued += g->chunks;
                take.push_back({id, s.scan, g->dev, g->filled, g->chunks, s.issued == s.n_chunks});
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
        lock.unlock();
        hd_status r = HD_OK;
        for (size_t i = 0; i < take.size() && r == HD_OK; ++i) {
            const float *p = take[i].dev;
            r = hd_batch_add_item(slot->batch, take[i].handle, p, p + cap, p + 2 * cap,
                                  p + 3 * cap, p + 4 * cap, p + 5 * cap, take[i].n,
                                  take[i].finishing ? HD_BATCH_FINALIZE : 0);
        }
        if (r == HD_OK) r = hd_batch_run(slot->batch, 0, sv->stream);
        const cudaError_t e = cudaEventRecord(slot->done, sv->stream);
        lock.lock();
        slot->busy = true;
        int64_t chunks = 0;
        for (const Take &tk : take) {
            slot->scans.push_back(tk.id);
            slot->chunks.push_back(tk.chunks);
            slot->finishing.push_back(tk.finishing && r == HD_OK && e == cudaSuccess);
            slot->bufs.push_back(tk.dev);
            chunks += tk.chunks;
            if (r != HD_OK || e != cudaSuccess) {
                SScan &s = sv->scans[tk.id];
                s.state = 3;
                s.status = r != HD_OK ? r : HD_ERR_CUDA;
            }
        }
        if (r != HD_OK || e != cudaSuccess) sv->cv_done.notify_all();
        sv->stats.launches += 1;
        sv->stats.items_launched += static_cast<int64_t>(take.size());
        sv->stats.chunks_launched += chunks;
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
    out->segment_histories = 1 << 19;
    out->staging_bytes = size_t(4) << 30;
    out->submit_timeout_ms = 60000;
    return HD_OK;
}

hd_status hd_server_create(const hd_server_config *cfg, hd_server **out)
{
    if (!cfg || !out) return HD_ERR_ARG;
    *out = nullptr;
    if (cfg->max_chunk < 1 || cfg->max_batch < 1 || cfg->max_batch > hd::kMaxBatch ||
        cfg->max_in_flight < 1 || cfg->max_in_flight > 8 || cfg->hbm_budget_bytes == 0 ||
        cfg->min_batch < 1 || cfg->segment_histories < cfg->max_chunk ||
        cfg->segment_histories > (int64_t(1) << 25) || cfg->submit_timeout_ms < 0 ||
        cfg->staging_bytes < sizeof(float) * 6 * static_cast<size_t>(cfg->segment_histories))
        return HD_ERR_ARG;
    hd_server *sv = new (std::nothrow) hd_server();
    if (!sv) return HD_ERR_NOMEM;
    sv->cfg = *cfg;
    sv->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
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
    sv->keeper = std::thread(keeper_main, sv);
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
    sv->cv_space.notify_all();
    sv->cv_keep.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->keeper.joinable()) sv->keeper.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    if (sv->stream) cudaStreamSynchronize(sv->stream);
    for (auto &kv : sv->scans)
        if (kv.second.scan) hd_scan_destroy(kv.second.scan);
    for (hd_scan *h : sv->graveyard) hd_scan_destroy(h);
    for (auto &p : sv->pool) hd_scan_destroy(p.scan);
    for (auto &t : sv->ticks) {
        if (t.batch) hd_batch_destroy(t.batch);
        if (t.done) cudaEventDestroy(t.done);
    }
    for (float *b : sv->all_bufs) cudaFree(b);
    if (sv->stream) cudaStreamDestroy(sv->stream);
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
    sv->cv_keep.notify_all();
    return HD_OK;
}

}  // extern "C"

namespace {

// A submit: reserve staging space, copy the chunk in (per column, or one
// strided copy when pitch > 0: column a at angle_deg + a pitch), account.
hd_status submit(hd_server *sv, int64_t scan_id, const float *angle_deg, const float *u_in,
                 const float *v_in, const float *u_out, const float *v_out, const float *wepl,
                 int64_t n, int64_t pitch, int32_t on_device)
{
    if (!sv || n < 1 || n > sv->cfg.max_chunk) return HD_ERR_ARG;
    if (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl) return HD_ERR_ARG;
    const auto t_submit = std::chrono::steady_clock::now();
    const auto deadline = t_submit + std::chrono::milliseconds(sv->cfg.submit_timeout_ms);
    const int64_t cap = sv->cfg.segment_histories;
    Segment *seg = nullptr;
    int64_t off = 0;
    {
        // reserve room in the scan's open segment (a new one when it is
        // full); device memory for a new segment is allocated outside the lock
        std::unique_lock<std::mutex> lock(sv->mu);
        float *held = nullptr;  // a segment buffer this call owns
        auto give_back = [&]() {
            if (held) sv->free_bufs.push_back(held);
            held = nullptr;
            sv->cv_space.notify_all();
        };
        for (;;) {
            auto it = sv->scans.find(scan_id);
            if (it == sv->scans.end()) {
                give_back();
                return HD_ERR_ARG;
            }
            SScan &s = it->second;
            if (s.state >= 2 || s.reserved_chunks >= s.n_chunks) {
                give_back();
                return HD_ERR_STATE;
            }
            if (!s.segs.empty() && !s.segs.back()->sealed && s.segs.back()->reserved + n <= cap) {
                seg = s.segs.back().get();
                give_back();
                break;
            }
            if (!held) held = pop_free_buffer(sv);
            if (held) {
                if (!s.segs.empty()) s.segs.back()->sealed = true;
                s.segs.emplace_back(new Segment());
                s.segs.back()->dev = held;
                held = nullptr;
                seg = s.segs.back().get();
                break;
            }
            const size_t nbufs = sv->all_bufs.size() + static_cast<size_t>(sv->allocating);
            if ((nbufs + 1) * segment_bytes(sv->cfg) <= sv->cfg.staging_bytes) {
                sv->allocating += 1;
                lock.unlock();
                const auto t_alloc = std::chrono::steady_clock::now();
                float *b = nullptr;
                const cudaError_t ea =
                    cudaMalloc(reinterpret_cast<void **>(&b), segment_bytes(sv->cfg));
                if (ea != cudaSuccess) cudaGetLastError();
                lock.lock();
                sv->allocating -= 1;
                sv->stats.alloc_seconds +=
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t_alloc).count();
                if (ea != cudaSuccess) return HD_ERR_NOMEM;
                sv->all_bufs.push_back(b);
                held = b;
                continue;  // the scan may have changed meanwhile
            }
            // staging is full: wait for a launch to return its segments
            if (sv->stop ||
                sv->cv_space.wait_until(lock, deadline) == std::cv_status::timeout)
                return HD_ERR_TIMEOUT;
        }
        off = seg->reserved;
        seg->reserved += n;
        seg->writers += 1;
        sv->scans[scan_id].reserved_chunks += 1;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != sv->device) cudaSetDevice(sv->device);
    const auto t_copy = std::chrono::steady_clock::now();
    const cudaStream_t up = upload_stream(sv->device);
    const float *src[6] = {angle_deg, u_in, v_in, u_out, v_out, wepl};
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = up ? cudaSuccess : cudaErrorUnknown;
    if (e == cudaSuccess && pitch > 0) {
        // the six columns are rows of one array: one strided copy
        e = cudaMemcpy2DAsync(seg->dev + off, sizeof(float) * static_cast<size_t>(cap), src[0],
                              sizeof(float) * static_cast<size_t>(pitch),
                              sizeof(float) * static_cast<size_t>(n), 6, kind, up);
    } else {
        for (int a = 0; e == cudaSuccess && a < 6; ++a)
            e = cudaMemcpyAsync(seg->dev + a * cap + off, src[a], sizeof(float) * n, kind, up);
    }
    // the caller may reuse its buffers as soon as this call returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(up);
    if (e != cudaSuccess) cudaGetLastError();
    if (prev >= 0 && prev != sv->device) cudaSetDevice(prev);
    const double copy_s =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_copy).count();
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stats.copy_seconds += copy_s;
    SScan &s = sv->scans[scan_id];  // cannot be closed while a copy runs
    seg->writers -= 1;
    if (e != cudaSuccess) {
        // the segment has a hole: the scan cannot be completed
        s.state = 3;
        s.status = HD_ERR_CUDA;
        sv->cv_done.notify_all();
        return HD_ERR_CUDA;
    }
    seg->filled += n;
    seg->chunks += 1;
    const double now = now_since(sv->t0);
    if (s.submitted == 0) s.t_first = now;
    s.submitted += 1;
    if (s.submitted == s.n_chunks) s.t_last = now;
    s.histories += n;
    sv->stats.chunks_submitted += 1;
    sv->stats.submit_seconds +=
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_submit).count();
    sv->cv_work.notify_all();
    return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_server_submit_chunk(hd_server *sv, int64_t scan_id, const float *angle_deg,
                                 const float *u_in, const float *v_in, const float *u_out,
                                 const float *v_out, const float *wepl, int64_t n,
                                 int32_t on_device)
{
    return submit(sv, scan_id, angle_deg, u_in, v_in, u_out, v_out, wepl, n, 0, on_device);
}

hd_status hd_server_submit_rows(hd_server *sv, int64_t scan_id, const float *rows, int64_t pitch,
                                int64_t n, int32_t on_device)
{
    if (!rows || pitch < n) return HD_ERR_ARG;
    return submit(sv, scan_id, rows, rows + pitch, rows + 2 * pitch, rows + 3 * pitch,
                  rows + 4 * pitch, rows + 5 * pitch, n, pitch, on_device);
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
    out->bytes_in_use = static_cast<int64_t>(sv->used - sv->pooled);
    out->bytes_pooled = static_cast<int64_t>(sv->pooled);
    return HD_OK;
}

hd_status hd_server_close_scan(hd_server *sv, int64_t scan_id)
{
    if (!sv) return HD_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->scans.find(scan_id);
    if (it == sv->scans.end()) return HD_ERR_ARG;
    SScan &s = it->second;
    if (s.admitting) return HD_ERR_STATE;                                // being created
    if (s.state == 1 && s.done_chunks < s.issued) return HD_ERR_STATE;  // still running
    if (s.state == 1 && !s.segs.empty()) return HD_ERR_STATE;
    for (const auto &g : s.segs)
        if (g->writers) return HD_ERR_STATE;  // a submit is copying into it
    if (s.state == 3 && s.done_chunks < s.issued) return HD_ERR_STATE;
    recycle_segments(sv, s);
    if (s.state == 2 && s.scan) {
        // kept for a later scan of the same geometry and parameters
        sv->pool.push_back({s.geom, s.params, s.scan, s.footprint});
        sv->pooled += s.footprint;
    } else if (s.scan) {
        if (s.state >= 1) sv->used -= s.footprint;
        sv->graveyard.push_back(s.scan);  // destroyed by the keeper thread
    }
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
    sv->cv_keep.notify_all();
    return HD_OK;
}

}  // extern "C"
