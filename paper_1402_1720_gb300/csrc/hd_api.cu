// C ABI of libhulld: scan objects, validation, memory and launch order.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "hd_geom.cuh"
#include "hd_rows.cuh"
#include "hd_thick.cuh"

namespace {

thread_local char g_last_cuda[256] = "";

void note_cuda(cudaError_t e, const char *where)
{
    std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s (%d)", where, cudaGetErrorString(e),
                  static_cast<int>(e));
}

#define HD_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            note_cuda(e_, #call);                      \
            return HD_ERR_CUDA;                        \
        }                                              \
    } while (0)

// Makes `dev` current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

constexpr int64_t kChunk = int64_t(1) << 25;  // histories per internal launch sequence
// a block's slot offsets (below the chunk size) fit a pair-list entry
static_assert(kChunk <= (int64_t(1) << (32 - hd::kRecordTileBits)), "pair-list entry width");
constexpr int64_t kMaxScanHistories = 4294967295LL;

// theta_i = round(atan(2^-i) * 180/pi * 2^30), K = round(2^30 prod (1 + 2^-2i)^-1/2),
// evaluated in double; the rounding is accepted only when the value is well
// away from a half-integer, so the integers do not depend on the libm.
bool make_cordic(hd::Cordic &c)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < 32; ++i) {
        const double v = std::atan(std::ldexp(1.0, -i)) * (180.0 / pi) * 1073741824.0;
        const double f = v - std::floor(v);
        if (std::fabs(f - 0.5) < 5e-5) return false;
        c.theta[i] = static_cast<long long>(std::floor(v + 0.5));
    }
    double k = 1073741824.0;
    for (int i = 0; i < 32; ++i) k /= std::sqrt(1.0 + std::ldexp(1.0, -2 * i));
    const double f = k - std::floor(k);
    if (std::fabs(f - 0.5) < 1e-3) return false;
    c.K = static_cast<long long>(std::floor(k + 0.5));
    return true;
}


}  // namespace

namespace hd {

bool make_cordic_table(Cordic &c) { return make_cordic(c); }

void note_cuda_error(cudaError_t e, const char *where) { note_cuda(e, where); }

hd_status check_geometry(const hd_geometry *g)
{
    if (!g) return HD_ERR_ARG;
    const int32_t n[3] = {g->nx, g->ny, g->nz};
    const float s[3] = {g->sx, g->sy, g->sz};
    int64_t V = 1;
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || n[a] > kMaxN) return HD_ERR_RANGE;
        if (!(s[a] >= 1.0f / 64.0f && s[a] <= 64.0f)) return HD_ERR_RANGE;
        if (static_cast<double>(n[a]) * s[a] > 8192.0) return HD_ERR_RANGE;
        V *= n[a];
    }
    if (V > (int64_t(1) << 31) - (int64_t(1) << 26)) return HD_ERR_RANGE;
    if (!(g->tracker_half_sep_mm > 0.0f && g->tracker_half_sep_mm < 4096.0f)) return HD_ERR_RANGE;
    return HD_OK;
}

}  // namespace hd

struct hd_scan {
    int device = 0;
    int sm_count = 0;
    hd_geometry geom{};
    hd_params params{};
    hd::GeomQ gq{};
    hd::Cordic cordic{};
    int64_t V = 0;
    int64_t words = 0;
    uint32_t *N = nullptr, *M = nullptr;
    uint8_t *H1 = nullptr, *H2 = nullptr, *H3 = nullptr;
    uint32_t *bits_out = nullptr;
    unsigned long long *slice_key = nullptr;
    uint32_t *mt = nullptr, *slope = nullptr;
    long long *index = nullptr;
    hd::Ctrl *ctrl = nullptr;
    // scratch: traversal records, (record, tile) pairs, jobs, host staging
    hd::TilePlan tp{};
    hd_tuning tuning{1024, 12, 32767, 0};
    int trace_grid = 0;
    int32_t *rec_buf = nullptr;   // 8 int32 arrays of rec_cap (coordinates, status, global list)
    int64_t rec_cap = 0;
    uint32_t *pair_buf = nullptr;  // lean walks (kLeanWords per pair), then the fallback list
    hd::TileJob *jobs = nullptr;
    int64_t job_cap = 0;
    hd::ScanDesc *desc_dev = nullptr;  // this scan's traversal descriptor
    hd::ScanDesc desc_host{};
    bool desc_dirty = true;
    // 2 * ntiles tile totals, then the ingest blocks' pair counts per tile
    // (tile_count_words)
    uint32_t *tile_count = nullptr;
    uint32_t *tile_cursor = nullptr;  // 2 * ntiles
    int64_t *rows_scratch = nullptr;  // tile sums of the system-row offset scan
    int64_t rows_scratch_cap = 0;
    uint32_t *rows_bits = nullptr;    // the hull packed for the row passes
    int32_t thick_k = 0;             // thick rays: in-plane dilation (0 = thin paths)
    float euclid_d0 = 0.0f;          // thick rays by Euclidean distance, mm (0 = off)
    void *thick_ws = nullptr;        // their difference arrays
    bool inputs_on_host = false;  // the chunk being added is read in place from host memory
    float *staging = nullptr;  // copied host inputs: 6 columns of staging_half floats
    int64_t staging_half = 0;
    uint32_t *compact_blocks = nullptr;
    unsigned long long *d_count = nullptr;
    int32_t *compact_out = nullptr;
    uint64_t n_total = 0;
    bool finalized = false;
    // profiling: (phase, start, stop) event triples awaiting readout
    bool profiling = false;
    struct Pending { int phase; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double ms[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t launches = 0;
    int64_t trace_launches = 0;
};

namespace {

cudaEvent_t take_event(hd_scan *s)
{
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Records a start event for `phase` on st when profiling; returns the event.
cudaEvent_t prof_begin(hd_scan *s, cudaStream_t st)
{
    if (!s->profiling) return nullptr;
    cudaEvent_t e = take_event(s);
    if (e) cudaEventRecord(e, st);
    return e;
}

void prof_end(hd_scan *s, int phase, cudaEvent_t a, cudaStream_t st)
{
    if (!s->profiling || !a) return;
    cudaEvent_t b = take_event(s);
    if (!b) return;
    cudaEventRecord(b, st);
    s->pending.push_back({phase, a, b});
}

void drain_profile(hd_scan *s)
{
    for (auto &p : s->pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            s->ms[p.phase] += ms;
        cudaGetLastError();
        s->event_pool.push_back(p.a);
        s->event_pool.push_back(p.b);
    }
    s->pending.clear();
}

void free_scan(hd_scan *s)
{
    drain_profile(s);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);

    void *ptrs[] = {s->N, s->M, s->H1, s->H2, s->H3, s->bits_out, s->slice_key,
                    s->mt, s->slope, s->index, s->ctrl, s->rec_buf, s->staging,
                    s->compact_blocks, s->d_count, s->compact_out, s->pair_buf, s->jobs,
                    s->rows_scratch, s->rows_bits, s->thick_ws,
                    s->tile_count, s->tile_cursor, s->desc_dev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete s;
}

hd_status validate(const hd_geometry *g, const hd_params *p)
{
    if (!g || !p) return HD_ERR_ARG;
    const hd_status gs = hd::check_geometry(g);
    if (gs != HD_OK) return gs;
    if (std::isnan(p->wepl_miss_lt) || std::isnan(p->wepl_hit_gt)) return HD_ERR_ARG;
    if (p->wepl_miss_lt > p->wepl_hit_gt) return HD_ERR_ARG;
    if (p->msc_nbhd != 4 && p->msc_nbhd != 6) return HD_ERR_ARG;
    if (p->sm_ge != 0 && p->sm_ge != 1) return HD_ERR_ARG;
    if (p->sm_per_slice != 0 && p->sm_per_slice != 1) return HD_ERR_ARG;
    if (p->methods == 0 || (p->methods & ~uint32_t(HD_SC | HD_MSC | HD_SM))) return HD_ERR_ARG;
    return HD_OK;
}

// Pairs of a chunk of n records: a path nearly parallel to the slices
// touches one or two slabs per x-y tile it crosses (its bounding box is what
// is counted); a record that does not fit the pair budget takes the
// global-memory path.
int64_t pairs_per_record(const hd::TilePlan &tp)
{
    int64_t k = 2 * static_cast<int64_t>(tp.ntx) * tp.nty;
    return k < tp.max_tiles ? k : tp.max_tiles;
}

hd_status ensure_records(hd_scan *s, int64_t n, cudaStream_t st)
{
    if (n <= s->rec_cap) return HD_OK;
    HD_CUDA(cudaStreamSynchronize(st));
    if (s->rec_buf) cudaFree(s->rec_buf);
    if (s->pair_buf) cudaFree(s->pair_buf);
    if (s->jobs) cudaFree(s->jobs);
    s->rec_buf = nullptr;
    s->pair_buf = nullptr;
    s->jobs = nullptr;
    s->rec_cap = 0;
    bool ok = cudaMalloc(&s->rec_buf, sizeof(int32_t) * 8 *
                                          static_cast<size_t>(hd::records_stride(n))) == cudaSuccess;
    if (ok && s->tp.ntiles > 0) {
        const int64_t pair_cap = pairs_per_record(s->tp) * n;
        const int64_t min_job = s->tp.job_size < hd::kMinJob ? s->tp.job_size : hd::kMinJob;
        const int64_t job_cap = pair_cap / min_job + 2 * s->tp.ntiles + 1;
        ok = cudaMalloc(&s->pair_buf, sizeof(uint32_t) * (hd::kLeanWords + 3) *
                                          static_cast<size_t>(pair_cap)) == cudaSuccess &&
             cudaMalloc(&s->jobs, sizeof(hd::TileJob) * static_cast<size_t>(job_cap)) == cudaSuccess;
        s->tp.pair_cap = pair_cap;
        s->job_cap = job_cap;
    }
    if (!ok) {
        cudaGetLastError();
        if (s->rec_buf) cudaFree(s->rec_buf);
        if (s->pair_buf) cudaFree(s->pair_buf);
        s->rec_buf = nullptr;
        s->pair_buf = nullptr;
        return HD_ERR_NOMEM;
    }
    s->rec_cap = n;
    s->desc_dirty = true;
    return HD_OK;
}


// Staging for host inputs that the device cannot read in place: six
// columns of `cap` histories.
hd_status ensure_staging(hd_scan *s, int64_t cap, cudaStream_t st)
{
    if (cap <= s->staging_half) return HD_OK;
    HD_CUDA(cudaStreamSynchronize(st));
    if (s->staging) {
        cudaFree(s->staging);
        s->staging = nullptr;
        s->staging_half = 0;
    }
    if (cudaMalloc(&s->staging, sizeof(float) * 6 * static_cast<size_t>(cap)) != cudaSuccess) {
        cudaGetLastError();
        s->staging = nullptr;
        return HD_ERR_NOMEM;
    }
    s->staging_half = cap;
    return HD_OK;
}

// Whether the device can read all six host arrays in place: page-locked
// memory mapped at the same address and allocated or registered with this
// device current (other host memory, including page-locked memory of another
// device's context, is copied instead).  Called with `device` current.
bool all_mapped_host(const float *const src[6], int device)
{
    for (int a = 0; a < 6; ++a) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, src[a]) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer != src[a] || at.device != device)
            return false;
    }
    return true;
}

// The records of a chunk of n histories: seven arrays of n slots and the
// global path's list, each starting on a 16-byte boundary.
hd::Records records_of(const hd_scan *s, int64_t n)
{
    hd::Records r;
    const size_t stride = static_cast<size_t>(hd::records_stride(n));
    for (int a = 0; a < 6; ++a) r.g[a] = s->rec_buf + a * stride;
    r.status = s->rec_buf + 6 * stride;
    r.glist = s->rec_buf + 7 * stride;
    r.cap = n;
    return r;
}

// Most ingest blocks a chunk can use.
size_t ingest_blocks_max(const hd_scan *s)
{
    return static_cast<size_t>(s->sm_count > 0 ? s->sm_count : 1) *
           static_cast<size_t>(hd::kIngestBlocksPerSm);
}

// Words of tile_count: the 2 * ntiles totals, a column of pair counts per
// tile and class for the most ingest blocks, then each block's pairs in all.
size_t tile_count_words(const hd_scan *s)
{
    const size_t cols = 2 * static_cast<size_t>(s->tp.ntiles);
    return cols * (1 + ingest_blocks_max(s)) + ingest_blocks_max(s);
}

hd::Pairs pairs_of(const hd_scan *s)
{
    hd::Pairs p;
    // the lean walks (kLeanWords words per pair), then the fallback list (two
    // words per pair), then the ingest blocks' pair lists (one word per pair)
    uint32_t *base = reinterpret_cast<uint32_t *>(s->pair_buf);
    const size_t cap = static_cast<size_t>(s->tp.pair_cap);
    p.v = reinterpret_cast<uint4 *>(base);
    p.fb = base ? reinterpret_cast<uint2 *>(base + hd::kLeanWords * cap) : nullptr;
    p.stage = base ? base + (hd::kLeanWords + 2) * cap : nullptr;
    return p;
}

// Tiles: one or more z-slices of the full x-y plane when they fit in the
// shared-memory budget, otherwise x-y strips of one slice.
void make_tile_plan(hd_scan *s)
{
    hd::TilePlan &tp = s->tp;
    const int nx = s->geom.nx, ny = s->geom.ny, nz = s->geom.nz;
    // one word per voxel of a tile box padded by a column and a row
    const int budget = hd::kTileSmemBytes / 4;
    tp.nx = nx;
    tp.ny = ny;
    tp.nz = nz;
    const int64_t plane = int64_t(nx + 1) * (ny + 1);
    if (plane <= budget) {
        // slabs of one z-slice by default: walks inside them never cross z, so
        // nearly all of them have the closed-form (lean) runs; deeper slabs
        // (slab_depth > 1) cut the pairs per history but send the walks that
        // cross z inside a slab to the general walk in global memory
        tp.tx = nx;
        tp.ty = ny;
        tp.tz = static_cast<int>(budget / plane);
        const int depth = s->tuning.slab_depth > 0 ? s->tuning.slab_depth : 1;
        if (depth < tp.tz) tp.tz = depth;
        if (tp.tz > nz) tp.tz = nz;
        const int ntz = (nz + tp.tz - 1) / tp.tz;
        tp.tz = (nz + ntz - 1) / ntz;
    } else {
        tp.tx = nx;
        tp.ty = budget / (nx + 1) - 1;
        const int nty = (ny + tp.ty - 1) / tp.ty;
        tp.ty = (ny + nty - 1) / nty;
        tp.tz = 1;
    }
    tp.ntx = (nx + tp.tx - 1) / tp.tx;
    tp.nty = (ny + tp.ty - 1) / tp.ty;
    tp.ntz = (nz + tp.tz - 1) / tp.tz;
    tp.ntiles = tp.ntx * tp.nty * tp.ntz;
    if (tp.ntiles > hd::kMaxTiles) tp.ntiles = 0;
    tp.max_tiles = hd::kMaxRecordTiles;
    tp.pairs_per_record = static_cast<int>(pairs_per_record(tp));
    tp.job_size = s->tuning.job_size;  // <= 32767: int16 differences in the tiled traversal
    tp.refill = s->tuning.refill;
    tp.threads = s->tuning.threads;
    // one 32-bit word per voxel (x-run and y-run difference counts in its
    // two halves), plus a padding column and row for the ends of runs
    tp.tile_words = (tp.tx + 1) * (tp.ty + 1) * tp.tz;
    auto magic = [](int t) {
        return t == 1 ? 0u : static_cast<unsigned>((1ull << 32) / static_cast<unsigned>(t)) + 1u;
    };
    tp.mtx = magic(tp.tx);
    tp.mty = magic(tp.ty);
    tp.mtz = magic(tp.tz);
    tp.pair_cap = 0;
}

hd::ScanDesc make_desc(const hd_scan *s)
{
    hd::ScanDesc d{};
    d.tp = s->tp;
    d.pairs = pairs_of(s);
    d.jobs = s->jobs;
    d.ctrl = s->ctrl;
    d.N = s->N;
    d.M = s->M;
    return d;
}

hd_status upload_desc(hd_scan *s, cudaStream_t st)
{
    if (!s->desc_dirty) return HD_OK;
    s->desc_host = make_desc(s);
    HD_CUDA(cudaMemcpyAsync(s->desc_dev, &s->desc_host, sizeof(hd::ScanDesc),
                            cudaMemcpyHostToDevice, st));
    HD_CUDA(cudaStreamSynchronize(st));  // desc_host may change before the copy ran
    s->desc_dirty = false;
    return HD_OK;
}

// Classification, geometry and bucketing of one chunk (everything before
// the traversal).
hd_status stage_prepare(hd_scan *s, const hd::Inputs &in, int64_t n, cudaStream_t st)
{
    const uint32_t m = s->params.methods;
    const int use_miss = (m & (HD_SC | HD_MSC)) ? 1 : 0;
    const int use_hit = (m & HD_SM) ? 1 : 0;
    const hd::Records rec = records_of(s, n);
    hd::TilePlan tp = s->tp;
    if (s->trace_grid <= 0) tp.ntiles = 0;
    HD_CUDA(cudaMemsetAsync(&s->ctrl->njobs, 0, sizeof(hd::Ctrl) - offsetof(hd::Ctrl, njobs), st));
    const size_t cols = 2 * static_cast<size_t>(s->tp.ntiles);
    uint32_t *block_count = s->tile_count + cols;
    uint32_t *block_pairs = block_count + cols * ingest_blocks_max(s);
    const hd::Pairs pairs = pairs_of(s);
    HD_CUDA(hd::launch_ingest(in, n, s->gq, s->cordic, s->params.wepl_miss_lt,
                              s->params.wepl_hit_gt, use_miss, use_hit, tp, rec, s->ctrl,
                              tp.ntiles > 0 ? block_count : nullptr, block_pairs, pairs.stage,
                              s->inputs_on_host ? 1 : 0, s->sm_count, st));
    s->launches += 1;
    if (tp.ntiles > 0) {
        HD_CUDA(hd::launch_plan(tp, n, block_count, s->tile_count, s->tile_cursor, s->jobs, s->ctrl,
                                s->sm_count, st));
        HD_CUDA(hd::launch_scatter(tp, rec, n, s->ctrl, s->tile_cursor, block_count, block_pairs,
                                   pairs, s->sm_count, st));
        s->launches += 3;
    }
    return HD_OK;
}

// Records outside the tiled path, walked with global-memory updates.
hd_status stage_global(hd_scan *s, int64_t n, cudaStream_t st)
{
    HD_CUDA(hd::launch_trace_global(records_of(s, n), s->ctrl, n, s->gq, s->N, s->M, 0,
                                    s->sm_count, st));
    s->launches += 1;
    return HD_OK;
}

hd_status stage_reset(hd_scan *scan, cudaStream_t st)
{
    const size_t V = static_cast<size_t>(scan->V);
    if (scan->N) HD_CUDA(cudaMemsetAsync(scan->N, 0, sizeof(uint32_t) * V, st));
    if (scan->M) HD_CUDA(cudaMemsetAsync(scan->M, 0, sizeof(uint32_t) * V, st));
    HD_CUDA(cudaMemsetAsync(scan->ctrl, 0, sizeof(hd::Ctrl), st));
    return HD_OK;
}

hd_status stage_finalize(hd_scan *scan, cudaStream_t st)
{
    hd::DecideArgs a{};
    a.nx = scan->geom.nx;
    a.ny = scan->geom.ny;
    a.nz = scan->geom.nz;
    a.methods = static_cast<int32_t>(scan->params.methods);
    a.nt = scan->params.msc_nt;
    a.nbhd = scan->params.msc_nbhd;
    a.sm_ge = scan->params.sm_ge;
    a.sm_per_slice = scan->params.sm_per_slice;
    a.N = scan->N;
    a.M = scan->M;
    a.slice_key = scan->slice_key;
    a.mt = scan->mt;
    a.slope = scan->slope;
    a.index = scan->index;
    a.H1 = scan->H1;
    a.H2 = scan->H2;
    a.H3 = scan->H3;
    HD_CUDA(hd::launch_finalize(a, scan->sm_count, st));
    return HD_OK;
}

int finalize_launches(const hd_scan *scan) { return (scan->params.methods & HD_SM) ? 3 : 1; }

// One chunk through the whole path on st.
hd_status run_chunk(hd_scan *s, const hd::Inputs &in, int64_t n, cudaStream_t st)
{
    if (s->euclid_d0 > 0.0f) {
        // Euclidean thick rays: a warp per history over the rows of its capsule
        const uint32_t m = s->params.methods;
        HD_CUDA(hd::launch_euclid(in, n, &s->geom, s->gq, s->cordic, s->params.wepl_miss_lt,
                                  s->params.wepl_hit_gt, (m & (HD_SC | HD_MSC)) ? 1 : 0,
                                  (m & HD_SM) ? 1 : 0, s->euclid_d0, s->thick_ws, s->N, s->M,
                                  &s->ctrl->n_in, nullptr, s->sm_count, st));
        s->launches += 4;
        return HD_OK;
    }
    if (s->thick_k > 0) {
        const hd::TilePlan &tp = s->tp;
        if (tp.ntiles > 0 && tp.ntx == 1 && tp.nty == 1 && tp.tz == 1) {
            // thick rays on the tiled path: the same records and pairs,
            // dilated in the traversal
            hd_status r = upload_desc(s, st);
            if (r != HD_OK) return r;
            r = stage_prepare(s, in, n, st);
            if (r != HD_OK) return r;
            HD_CUDA(hd::launch_thick_scan(s->desc_dev, &s->geom, records_of(s, n), s->ctrl, n,
                                          s->gq, s->thick_k, s->thick_ws, s->N, s->M,
                                          tp.tile_words, tp.threads, s->sm_count, st));
            s->launches += 4;
            return HD_OK;
        }
        // other plans: a lane per history over the whole grid
        const uint32_t m = s->params.methods;
        HD_CUDA(hd::launch_thick(in, n, &s->geom, s->gq, s->cordic, s->params.wepl_miss_lt,
                                 s->params.wepl_hit_gt, (m & (HD_SC | HD_MSC)) ? 1 : 0,
                                 (m & HD_SM) ? 1 : 0, s->thick_k, s->thick_ws, s->N, s->M,
                                 &s->ctrl->n_in, nullptr, s->sm_count, st));
        s->launches += 1;
        return HD_OK;
    }
    hd_status r = upload_desc(s, st);
    if (r != HD_OK) return r;
    cudaEvent_t e0 = prof_begin(s, st);
    r = stage_prepare(s, in, n, st);
    if (r != HD_OK) return r;
    prof_end(s, 0, e0, st);
    cudaEvent_t e1 = prof_begin(s, st);
    if (s->tp.ntiles > 0 && s->trace_grid > 0) {
        HD_CUDA(hd::launch_trace_tiles(s->desc_dev, 1, &s->ctrl->job_next, s->tp.tile_words,
                                       s->tp.threads, s->trace_grid, st));
        s->launches += 1;
        if (s->profiling) s->trace_launches += 1;
    }
    prof_end(s, 1, e1, st);
    cudaEvent_t e2 = prof_begin(s, st);
    r = stage_global(s, n, st);
    if (r != HD_OK) return r;
    prof_end(s, 3, e2, st);
    return HD_OK;
}

}  // namespace

extern "C" {

const char *hd_status_string(hd_status s)
{
    switch (s) {
    case HD_OK: return "HD_OK";
    case HD_ERR_ARG: return "HD_ERR_ARG";
    case HD_ERR_RANGE: return "HD_ERR_RANGE";
    case HD_ERR_NOMEM: return "HD_ERR_NOMEM";
    case HD_ERR_CUDA: return "HD_ERR_CUDA";
    case HD_ERR_STATE: return "HD_ERR_STATE";
    case HD_ERR_TIMEOUT: return "HD_ERR_TIMEOUT";
    case HD_ERR_ADMISSION: return "HD_ERR_ADMISSION";
    case HD_ERR_OVERFLOW: return "HD_ERR_OVERFLOW";
    }
    return "HD_ERR_UNKNOWN";
}

const char *hd_last_cuda_error(void) { return g_last_cuda; }

hd_status hd_params_default(hd_params *out)
{
    if (!out) return HD_ERR_ARG;
    out->wepl_miss_lt = 1.0f;
    out->wepl_hit_gt = 5.0f;
    out->msc_nt = 50;
    out->msc_nbhd = 6;
    out->sm_ge = 1;
    out->sm_per_slice = 1;
    out->methods = HD_SC | HD_MSC | HD_SM;
    return HD_OK;
}

hd_status hd_scan_create(const hd_geometry *geom, const hd_params *params, hd_scan **out)
{
    if (!out) return HD_ERR_ARG;
    *out = nullptr;
    const hd_status v = validate(geom, params);
    if (v != HD_OK) return v;
    hd_scan *s = new (std::nothrow) hd_scan();
    if (!s) return HD_ERR_NOMEM;
    s->geom = *geom;
    s->params = *params;
    if (!make_cordic(s->cordic)) {
        delete s;
        return HD_ERR_RANGE;
    }
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        note_cuda(e, "hd_scan_create: device query");
        delete s;
        return HD_ERR_CUDA;
    }
    s->gq = hd::make_geomq(geom->nx, geom->ny, geom->nz, geom->sx, geom->sy, geom->sz,
                           geom->tracker_half_sep_mm);
    s->V = int64_t(geom->nx) * geom->ny * geom->nz;
    s->words = (s->V + 31) / 32;
    const uint32_t m = params->methods;
    const size_t V = static_cast<size_t>(s->V);
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            ok = false;
        }
    };
    // SC and MSC both read N: H_1 = [N = 0] (Eq. 3.3, the carve of Alg. 1
    // as a set difference) and Eq. 3.6
    if (m & (HD_SC | HD_MSC)) alloc(reinterpret_cast<void **>(&s->N), sizeof(uint32_t) * V);
    if (m & HD_SM) {
        alloc(reinterpret_cast<void **>(&s->M), sizeof(uint32_t) * V);
        alloc(reinterpret_cast<void **>(&s->slice_key), sizeof(unsigned long long) * geom->nz);
        alloc(reinterpret_cast<void **>(&s->mt), sizeof(uint32_t) * geom->nz);
        alloc(reinterpret_cast<void **>(&s->slope), sizeof(uint32_t) * geom->nz);
        alloc(reinterpret_cast<void **>(&s->index), sizeof(long long) * geom->nz);
        alloc(reinterpret_cast<void **>(&s->H3), V);
    }
    if (m & HD_SC) alloc(reinterpret_cast<void **>(&s->H1), V);
    if (m & HD_MSC) alloc(reinterpret_cast<void **>(&s->H2), V);
    alloc(reinterpret_cast<void **>(&s->bits_out), sizeof(uint32_t) * s->words);
    make_tile_plan(s);
    if (s->tp.ntiles > 0) {
        alloc(reinterpret_cast<void **>(&s->tile_count), sizeof(uint32_t) * tile_count_words(s));
        alloc(reinterpret_cast<void **>(&s->tile_cursor), sizeof(uint32_t) * 2 * s->tp.ntiles);
        const int per_sm = hd::trace_tiles_occupancy(s->tp.tile_words, s->tp.threads);
        s->trace_grid = per_sm > 0 ? per_sm * s->sm_count : 0;
    }
    alloc(reinterpret_cast<void **>(&s->ctrl), sizeof(hd::Ctrl));
    alloc(reinterpret_cast<void **>(&s->desc_dev), sizeof(hd::ScanDesc));
    if (!ok) {
        free_scan(s);
        return HD_ERR_NOMEM;
    }
    // zero the counts on a private non-blocking stream: the legacy default
    // stream would serialise with every blocking stream of the process
    cudaStream_t init = nullptr;
    e = cudaStreamCreateWithFlags(&init, cudaStreamNonBlocking);
    const hd_status r = e == cudaSuccess ? hd_scan_reset(s, init) : HD_ERR_CUDA;
    if (r == HD_OK) e = cudaStreamSynchronize(init);
    if (init) cudaStreamDestroy(init);
    if (r != HD_OK || e != cudaSuccess) {
        if (e != cudaSuccess) note_cuda(e, "hd_scan_create: sync");
        free_scan(s);
        return r != HD_OK ? r : HD_ERR_CUDA;
    }
    *out = s;
    return HD_OK;
}

hd_status hd_scan_destroy(hd_scan *scan)
{
    if (!scan) return HD_OK;
    DeviceGuard g(scan->device);
    cudaDeviceSynchronize();
    free_scan(scan);
    return HD_OK;
}

hd_status hd_scan_reset(hd_scan *scan, void *stream)
{
    if (!scan) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    const hd_status r = stage_reset(scan, static_cast<cudaStream_t>(stream));
    if (r != HD_OK) return r;
    scan->n_total = 0;
    scan->finalized = false;
    return HD_OK;
}

hd_status hd_scan_reserve(hd_scan *scan, int64_t n, void *stream)
{
    if (!scan || n < 0) return HD_ERR_ARG;
    if (n == 0) return HD_OK;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    return ensure_records(scan, n < kChunk ? n : kChunk, static_cast<cudaStream_t>(stream));
}

hd_status hd_scan_add_histories(hd_scan *scan, const float *angle_deg, const float *u_in,
                                const float *v_in, const float *u_out, const float *v_out,
                                const float *wepl, int64_t n, int32_t on_device, void *stream)
{
    if (!scan || n < 0) return HD_ERR_ARG;
    if (n == 0) return HD_OK;
    if (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl) return HD_ERR_ARG;
    if (static_cast<uint64_t>(n) > static_cast<uint64_t>(kMaxScanHistories) - scan->n_total)
        return HD_ERR_OVERFLOW;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *src[6] = {angle_deg, u_in, v_in, u_out, v_out, wepl};
    if (on_device) {
        const int64_t chunk = n < kChunk ? n : kChunk;
        hd_status r = ensure_records(scan, chunk, st);
        if (r != HD_OK) return r;
        for (int64_t off = 0; off < n; off += chunk) {
            const int64_t c = (n - off) < chunk ? (n - off) : chunk;
            const hd::Inputs in{src[0] + off, src[1] + off, src[2] + off,
                                src[3] + off, src[4] + off, src[5] + off};
            r = run_chunk(scan, in, c, st);
            if (r != HD_OK) return r;
        }
    } else if (all_mapped_host(src, scan->device)) {
        // page-locked host arrays mapped into the device's address space: the
        // ingest kernel reads them in place over the host link, so the
        // transfer happens inside the kernel that consumes it
        const int64_t chunk = n < kChunk ? n : kChunk;
        hd_status r = ensure_records(scan, chunk, st);
        if (r != HD_OK) return r;
        scan->inputs_on_host = true;
        for (int64_t off = 0; off < n && r == HD_OK; off += chunk) {
            const int64_t c = (n - off) < chunk ? (n - off) : chunk;
            const hd::Inputs in{src[0] + off, src[1] + off, src[2] + off,
                                src[3] + off, src[4] + off, src[5] + off};
            r = run_chunk(scan, in, c, st);
        }
        scan->inputs_on_host = false;
        if (r != HD_OK) return r;
    } else {
        // other host memory: copied to the scan's staging buffer, one chunk
        // at a time, on st
        const int64_t chunk = n < kChunk ? n : kChunk;
        hd_status r = ensure_records(scan, chunk, st);
        if (r != HD_OK) return r;
        r = ensure_staging(scan, chunk, st);
        if (r != HD_OK) return r;
        const int64_t half = scan->staging_half;
        for (int64_t off = 0; off < n; off += chunk) {
            const int64_t c = (n - off) < chunk ? (n - off) : chunk;
            float *base = scan->staging;
            for (int a = 0; a < 6; ++a)
                HD_CUDA(cudaMemcpyAsync(base + a * half, src[a] + off, sizeof(float) * c,
                                        cudaMemcpyHostToDevice, st));
            const hd::Inputs in{base, base + half, base + 2 * half,
                                base + 3 * half, base + 4 * half, base + 5 * half};
            r = run_chunk(scan, in, c, st);
            if (r != HD_OK) return r;
        }
    }
    scan->n_total += static_cast<uint64_t>(n);
    scan->finalized = false;
    return HD_OK;
}

hd_status hd_scan_finalize(hd_scan *scan, void *stream)
{
    if (!scan) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = prof_begin(scan, st);
    const hd_status r = stage_finalize(scan, st);
    if (r != HD_OK) return r;
    scan->launches += finalize_launches(scan);
    prof_end(scan, 2, e0, st);
    scan->finalized = true;
    return HD_OK;
}

static uint8_t *mask_of(hd_scan *s, int32_t method)
{
    switch (method) {
    case HD_SC: return s->H1;
    case HD_MSC: return s->H2;
    case HD_SM: return s->H3;
    default: return nullptr;
    }
}

hd_status hd_scan_system_rows(hd_scan *scan, int32_t method, const float *angle_deg,
                              const float *u_in, const float *v_in, const float *u_out,
                              const float *v_out, int64_t n, int64_t *row_ptr, int32_t *cols,
                              int64_t capacity, int64_t *nnz, void *stream)
{
    if (!scan || !nnz || n < 0 || capacity < 0 || !row_ptr || (capacity > 0 && !cols))
        return HD_ERR_ARG;
    if (n > 0 && (!angle_deg || !u_in || !v_in || !u_out || !v_out)) return HD_ERR_ARG;
    if (method != HD_SC && method != HD_MSC && method != HD_SM) return HD_ERR_ARG;
    if (!(scan->params.methods & static_cast<uint32_t>(method)) || !scan->finalized)
        return HD_ERR_STATE;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *nnz = 0;
    if (n == 0) {
        HD_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
        HD_CUDA(cudaStreamSynchronize(st));
        return HD_OK;
    }
    const int64_t need = hd::rows_scan_scratch(n);
    if (need > scan->rows_scratch_cap) {
        HD_CUDA(cudaStreamSynchronize(st));
        if (scan->rows_scratch) cudaFree(scan->rows_scratch);
        scan->rows_scratch = nullptr;
        scan->rows_scratch_cap = 0;
        if (cudaMalloc(&scan->rows_scratch, sizeof(int64_t) * static_cast<size_t>(need)) !=
            cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_NOMEM;
        }
        scan->rows_scratch_cap = need;
    }
    const uint8_t *hull = mask_of(scan, method);
    if (!scan->rows_bits) {
        if (cudaMalloc(&scan->rows_bits, sizeof(uint32_t) * static_cast<size_t>(scan->words)) !=
            cudaSuccess) {
            cudaGetLastError();
            scan->rows_bits = nullptr;
            return HD_ERR_NOMEM;
        }
    }
    HD_CUDA(hd::launch_pack_bits(hull, scan->V, scan->rows_bits, st));
    const hd::Inputs in{angle_deg, u_in, v_in, u_out, v_out, nullptr};
    HD_CUDA(hd::launch_rows_count(in, n, scan->gq, scan->cordic, hull, scan->rows_bits, row_ptr,
                                  scan->sm_count, st));
    HD_CUDA(hd::launch_rows_scan(row_ptr + 1, n, scan->rows_scratch, st));
    int64_t total = 0;
    HD_CUDA(cudaMemcpyAsync(&total, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    *nnz = total;
    if (total > capacity) return HD_ERR_RANGE;
    HD_CUDA(hd::launch_rows_emit(in, n, scan->gq, scan->cordic, hull, scan->rows_bits, row_ptr,
                                 cols, scan->sm_count, st));
    return HD_OK;
}

hd_status hd_scan_get_mask(hd_scan *scan, int32_t method, int32_t layout, void *dst,
                           size_t dst_bytes, int32_t dst_on_device, void *stream)
{
    if (!scan || !dst) return HD_ERR_ARG;
    if (method != HD_SC && method != HD_MSC && method != HD_SM) return HD_ERR_ARG;
    if (layout != HD_MASK_U8 && layout != HD_MASK_BITS) return HD_ERR_ARG;
    if (!(scan->params.methods & static_cast<uint32_t>(method)) || !scan->finalized)
        return HD_ERR_STATE;
    uint8_t *src = mask_of(scan, method);
    const size_t need = layout == HD_MASK_U8 ? static_cast<size_t>(scan->V)
                                             : sizeof(uint32_t) * static_cast<size_t>(scan->words);
    if (dst_bytes < need) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (layout == HD_MASK_U8) {
        HD_CUDA(cudaMemcpyAsync(dst, src, need, kind, st));
    } else {
        uint32_t *bits = dst_on_device ? static_cast<uint32_t *>(dst) : scan->bits_out;
        HD_CUDA(hd::launch_pack_bits(src, scan->V, bits, st));
        if (!dst_on_device) HD_CUDA(cudaMemcpyAsync(dst, bits, need, kind, st));
    }
    return HD_OK;
}

hd_status hd_scan_get_counts(hd_scan *scan, int32_t method, uint32_t *dst, int64_t n,
                             int32_t dst_on_device, void *stream)
{
    if (!scan || !dst) return HD_ERR_ARG;
    const uint32_t *src = nullptr;
    if (method == HD_MSC || method == HD_SC) src = scan->N;
    else if (method == HD_SM) src = scan->M;
    else return HD_ERR_ARG;
    if (!src) return HD_ERR_STATE;
    if (n < scan->V) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    HD_CUDA(cudaMemcpyAsync(dst, src, sizeof(uint32_t) * static_cast<size_t>(scan->V),
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            static_cast<cudaStream_t>(stream)));
    return HD_OK;
}

hd_status hd_scan_set_counts(hd_scan *scan, int32_t method, const uint32_t *src, int64_t n,
                             int32_t src_on_device, void *stream)
{
    if (!scan || !src) return HD_ERR_ARG;
    uint32_t *dst = nullptr;
    if (method == HD_MSC || method == HD_SC) dst = scan->N;
    else if (method == HD_SM) dst = scan->M;
    else return HD_ERR_ARG;
    if (!dst) return HD_ERR_STATE;
    if (n != scan->V) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    HD_CUDA(cudaMemcpyAsync(dst, src, sizeof(uint32_t) * static_cast<size_t>(scan->V),
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            static_cast<cudaStream_t>(stream)));
    scan->finalized = false;
    return HD_OK;
}

hd_status hd_scan_get_thresholds(hd_scan *scan, uint32_t *mt, uint32_t *slope, int64_t *index,
                                 int32_t nz, void *stream)
{
    if (!scan) return HD_ERR_ARG;
    if (!(scan->params.methods & HD_SM) || !scan->finalized) return HD_ERR_STATE;
    if (nz < scan->geom.nz) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t z = static_cast<size_t>(scan->geom.nz);
    if (mt) HD_CUDA(cudaMemcpyAsync(mt, scan->mt, 4 * z, cudaMemcpyDeviceToHost, st));
    if (slope) HD_CUDA(cudaMemcpyAsync(slope, scan->slope, 4 * z, cudaMemcpyDeviceToHost, st));
    if (index) HD_CUDA(cudaMemcpyAsync(index, scan->index, 8 * z, cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    return HD_OK;
}

hd_status hd_scan_get_stats(hd_scan *scan, hd_stats *out, void *stream)
{
    if (!scan || !out) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    hd::Ctrl c;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // voxel memberships: sum_v N(v) = sum over missed histories of |A_i|
    // (Eq. 3.4), likewise M for the hit ones, so no traversal kernel counts
    // them
    HD_CUDA(hd::launch_volume_sums(scan->N, scan->M, scan->V, &scan->ctrl->steps_miss,
                                   scan->sm_count, st));
    HD_CUDA(cudaMemcpyAsync(&c, scan->ctrl, sizeof(c), cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    out->n_in = static_cast<int64_t>(c.n_in);
    out->n_miss = static_cast<int64_t>(c.n_miss);
    out->n_hit = static_cast<int64_t>(c.n_hit);
    out->n_none = static_cast<int64_t>(c.n_none);
    out->n_reject = static_cast<int64_t>(c.n_reject);
    out->steps_miss = static_cast<int64_t>(c.steps_miss);
    out->steps_hit = static_cast<int64_t>(c.steps_hit);
    out->pairs_general = static_cast<int64_t>(c.pairs_general);
    out->runs = static_cast<int64_t>(c.runs);
    return HD_OK;
}

hd_status hd_scan_get_hull_indices(hd_scan *scan, int32_t method, int32_t *dst,
                                   int64_t capacity, int64_t *count, int32_t dst_on_device,
                                   void *stream)
{
    if (!scan || !count || capacity < 0 || (capacity > 0 && !dst)) return HD_ERR_ARG;
    if (method != HD_SC && method != HD_MSC && method != HD_SM) return HD_ERR_ARG;
    if (!(scan->params.methods & static_cast<uint32_t>(method)) || !scan->finalized)
        return HD_ERR_STATE;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nb = (scan->V + 1023) / 1024;
    if (!scan->compact_blocks) {
        if (cudaMalloc(&scan->compact_blocks, sizeof(uint32_t) * (nb + 1)) != cudaSuccess ||
            cudaMalloc(&scan->d_count, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_NOMEM;
        }
    }
    int32_t *out = dst;
    int64_t cap = capacity;
    if (!dst_on_device) {
        if (!scan->compact_out &&
            cudaMalloc(&scan->compact_out, sizeof(int32_t) * static_cast<size_t>(scan->V)) !=
                cudaSuccess) {
            cudaGetLastError();
            scan->compact_out = nullptr;
            return HD_ERR_NOMEM;
        }
        out = scan->compact_out;
        cap = scan->V;
    }
    HD_CUDA(hd::launch_compact(mask_of(scan, method), scan->V, out, cap, scan->compact_blocks,
                               scan->d_count, st));
    unsigned long long total = 0;
    HD_CUDA(cudaMemcpyAsync(&total, scan->d_count, sizeof(total), cudaMemcpyDeviceToHost, st));
    HD_CUDA(cudaStreamSynchronize(st));
    *count = static_cast<int64_t>(total);
    if (!dst_on_device && capacity > 0) {
        const int64_t k = static_cast<int64_t>(total) < capacity ? static_cast<int64_t>(total)
                                                                 : capacity;
        if (k > 0) {
            HD_CUDA(cudaMemcpyAsync(dst, out, sizeof(int32_t) * static_cast<size_t>(k),
                                    cudaMemcpyDeviceToHost, st));
            HD_CUDA(cudaStreamSynchronize(st));
        }
    }
    return HD_OK;
}

hd_status hd_scan_set_thick(hd_scan *scan, int32_t k)
{
    if (!scan) return HD_ERR_ARG;
    if (k < 0 || k > 16) return HD_ERR_RANGE;
    if (scan->n_total != 0) return HD_ERR_STATE;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    if (k > 0) {
        HD_CUDA(cudaDeviceSynchronize());
        if (!scan->thick_ws) {
            if (cudaMalloc(&scan->thick_ws, hd::thick_workspace_bytes(&scan->geom)) !=
                cudaSuccess) {
                cudaGetLastError();
                scan->thick_ws = nullptr;
                return HD_ERR_NOMEM;
            }
        }
    }
    scan->thick_k = k;
    if (k > 0) scan->euclid_d0 = 0.0f;
    return HD_OK;
}

hd_status hd_scan_set_thick_distance(hd_scan *scan, float d0_mm)
{
    if (!scan) return HD_ERR_ARG;
    if (!(d0_mm >= 0.0f && d0_mm <= 64.0f)) return HD_ERR_RANGE;
    if (scan->n_total != 0) return HD_ERR_STATE;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    if (d0_mm > 0.0f && !scan->thick_ws) {
        HD_CUDA(cudaDeviceSynchronize());
        if (cudaMalloc(&scan->thick_ws, hd::thick_workspace_bytes(&scan->geom)) != cudaSuccess) {
            cudaGetLastError();
            scan->thick_ws = nullptr;
            return HD_ERR_NOMEM;
        }
    }
    scan->euclid_d0 = d0_mm;
    if (d0_mm > 0.0f) scan->thick_k = 0;
    return HD_OK;
}

hd_status hd_scan_set_tuning(hd_scan *scan, const hd_tuning *t)
{
    if (!scan || !t) return HD_ERR_ARG;
    if (t->threads != 256 && t->threads != 512 && t->threads != 768 && t->threads != 1024)
        return HD_ERR_ARG;
    if (t->refill < 1 || t->refill > 32 || t->job_size < 256 || t->job_size > 32767 ||
        t->slab_depth < 0)
        return HD_ERR_ARG;
    if (scan->n_total != 0) return HD_ERR_STATE;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    HD_CUDA(cudaDeviceSynchronize());
    // drop everything sized by the old plan; it regrows on the next add
    void *old[] = {scan->tile_count, scan->tile_cursor, scan->rec_buf, scan->pair_buf, scan->jobs};
    for (void *p : old)
        if (p) cudaFree(p);
    scan->tile_count = scan->tile_cursor = nullptr;
    scan->rec_buf = nullptr;
    scan->pair_buf = nullptr;
    scan->jobs = nullptr;
    scan->rec_cap = 0;
    scan->tuning = *t;
    make_tile_plan(scan);
    scan->trace_grid = 0;
    if (scan->tp.ntiles > 0) {
        if (cudaMalloc(&scan->tile_count, sizeof(uint32_t) * tile_count_words(scan)) != cudaSuccess ||
            cudaMalloc(&scan->tile_cursor, sizeof(uint32_t) * 2 * scan->tp.ntiles) != cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_NOMEM;
        }
        const int per_sm = hd::trace_tiles_occupancy(scan->tp.tile_words, scan->tp.threads);
        scan->trace_grid = per_sm > 0 ? per_sm * scan->sm_count : 0;
    }
    scan->desc_dirty = true;
    return HD_OK;
}

hd_status hd_scan_get_tuning(hd_scan *scan, hd_tuning *out)
{
    if (!scan || !out) return HD_ERR_ARG;
    *out = scan->tuning;
    return HD_OK;
}

hd_status hd_scan_set_profiling(hd_scan *scan, int32_t enable)
{
    if (!scan) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    drain_profile(scan);
    if (enable) {
        scan->ms[0] = scan->ms[1] = scan->ms[2] = scan->ms[3] = 0.0;
        scan->trace_launches = 0;
    }
    scan->profiling = enable != 0;
    return HD_OK;
}

hd_status hd_scan_get_profile(hd_scan *scan, hd_profile *out)
{
    if (!scan || !out) return HD_ERR_ARG;
    DeviceGuard g(scan->device);
    if (!g.ok) return HD_ERR_CUDA;
    drain_profile(scan);
    out->kernel_launches = scan->launches;
    out->trace_launches = scan->trace_launches;
    out->ms_ingest = scan->ms[0];
    out->ms_trace = scan->ms[1];
    out->ms_finalize = scan->ms[2];
    out->ms_trace_global = scan->ms[3];
    return HD_OK;
}

hd_status hd_classify(const float *wepl, int64_t n, const hd_params *params, uint8_t *cls_out,
                      int32_t on_device, void *stream)
{
    if (!params || n < 0) return HD_ERR_ARG;
    if (n == 0) return HD_OK;
    if (!wepl || !cls_out) return HD_ERR_ARG;
    if (std::isnan(params->wepl_miss_lt) || std::isnan(params->wepl_hit_gt) ||
        params->wepl_miss_lt > params->wepl_hit_gt)
        return HD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (on_device) {
        HD_CUDA(hd::launch_classify(wepl, n, params->wepl_miss_lt, params->wepl_hit_gt, cls_out,
                                    st));
        return HD_OK;
    }
    float *dw = nullptr;
    uint8_t *dc = nullptr;
    if (cudaMalloc(&dw, sizeof(float) * static_cast<size_t>(n)) != cudaSuccess ||
        cudaMalloc(&dc, static_cast<size_t>(n)) != cudaSuccess) {
        cudaGetLastError();
        if (dw) cudaFree(dw);
        return HD_ERR_NOMEM;
    }
    hd_status r = HD_OK;
    cudaError_t e = cudaMemcpyAsync(dw, wepl, sizeof(float) * static_cast<size_t>(n),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = hd::launch_classify(dw, n, params->wepl_miss_lt, params->wepl_hit_gt, dc, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cls_out, dc, static_cast<size_t>(n), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        note_cuda(e, "hd_classify");
        r = HD_ERR_CUDA;
    }
    cudaFree(dw);
    cudaFree(dc);
    return r;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct hd_batch {
    int device = 0;
    int sm_count = 0;
    int max_items = 0;
    struct Item {
        hd_scan *scan;
        hd::Inputs in;
        int64_t n;
        bool first = false;  // the scan's first item in this run (reset here)
        bool last = false;   // the scan's last item in this run (finalize here)
        int flags = 0;       // per-item HD_BATCH_RESET / HD_BATCH_FINALIZE
    };
    std::vector<Item> items;
    hd::ScanDesc *descs_dev = nullptr;  // kMaxBatch descriptors
    hd::ScanDesc *descs_pinned = nullptr;  // host staging of the table (pinned)
    cudaEvent_t descs_copied = nullptr;     // the last upload from descs_pinned is done
    int *job_counter = nullptr;
    static constexpr int kSide = 8;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kSide] = {};
    bool use_graph = true;
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;  // items and flags the cached graph was made for
    int64_t graph_kernels = 0;
    int threads = 512;
    hd_batch_stats stats{};
};

namespace {

void free_batch(hd_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto &st : b->side)
        if (st) cudaStreamDestroy(st);
    for (auto &e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->descs_dev) cudaFree(b->descs_dev);
    if (b->descs_pinned) cudaFreeHost(b->descs_pinned);
    if (b->descs_copied) cudaEventDestroy(b->descs_copied);
    if (b->job_counter) cudaFree(b->job_counter);
    delete b;
}

// One round: every item of `round` (distinct scans), issued on `st` with
// the per-scan stages forked to the side streams.  Returns the number of
// kernels issued through *kernels.
hd_status issue_round(hd_batch *b, const std::vector<hd_batch::Item> &round, int flags,
                      int grid, cudaStream_t st, int64_t *kernels)
{
    const int n_items = static_cast<int>(round.size());
    int max_words = 0;
    bool any_tiled = false;
    for (const auto &it : round) {
        if (it.scan->tp.ntiles > 0 && it.scan->trace_grid > 0) {
            any_tiled = true;
            if (it.scan->tp.tile_words > max_words) max_words = it.scan->tp.tile_words;
        }
    }
    auto fork = [&]() -> hd_status {
        HD_CUDA(cudaEventRecord(b->fork, st));
        for (int k = 0; k < hd_batch::kSide; ++k) HD_CUDA(cudaStreamWaitEvent(b->side[k], b->fork, 0));
        return HD_OK;
    };
    auto join = [&]() -> hd_status {
        for (int k = 0; k < hd_batch::kSide; ++k) {
            HD_CUDA(cudaEventRecord(b->join[k], b->side[k]));
            HD_CUDA(cudaStreamWaitEvent(st, b->join[k], 0));
        }
        return HD_OK;
    };
    hd_status r = fork();
    if (r != HD_OK) return r;
    for (int i = 0; i < n_items; ++i) {
        hd_scan *s = round[i].scan;
        cudaStream_t ss = b->side[i % hd_batch::kSide];
        if ((round[i].first && (flags & HD_BATCH_RESET)) || (round[i].flags & HD_BATCH_RESET)) {
            r = stage_reset(s, ss);
            if (r != HD_OK) return r;
        }
        r = stage_prepare(s, round[i].in, round[i].n, ss);
        if (r != HD_OK) return r;
        *kernels += 1 + ((s->tp.ntiles > 0 && s->trace_grid > 0) ? 2 : 0);
    }
    r = join();
    if (r != HD_OK) return r;
    if (any_tiled) {
        HD_CUDA(cudaMemsetAsync(b->job_counter, 0, sizeof(int), st));
        HD_CUDA(hd::launch_trace_tiles(b->descs_dev, n_items, b->job_counter, max_words,
                                       b->threads, grid, st));
        *kernels += 1;
    }
    r = fork();
    if (r != HD_OK) return r;
    for (int i = 0; i < n_items; ++i) {
        hd_scan *s = round[i].scan;
        cudaStream_t ss = b->side[i % hd_batch::kSide];
        r = stage_global(s, round[i].n, ss);
        if (r != HD_OK) return r;
        *kernels += 1;
        if ((round[i].last && (flags & HD_BATCH_FINALIZE)) ||
            (round[i].flags & HD_BATCH_FINALIZE)) {
            r = stage_finalize(s, ss);
            if (r != HD_OK) return r;
            *kernels += finalize_launches(s);
        }
    }
    return join();
}

}  // namespace

extern "C" {

hd_status hd_batch_create(int32_t max_items, hd_batch **out)
{
    if (!out || max_items < 1 || max_items > hd::kMaxBatch) return HD_ERR_ARG;
    *out = nullptr;
    hd_batch *b = new (std::nothrow) hd_batch();
    if (!b) return HD_ERR_NOMEM;
    b->max_items = max_items;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    for (int k = 0; e == cudaSuccess && k < hd_batch::kSide; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->descs_dev, sizeof(hd::ScanDesc) * hd::kMaxBatch);
    if (e == cudaSuccess)
        e = cudaMallocHost(&b->descs_pinned, sizeof(hd::ScanDesc) * hd::kMaxBatch);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->descs_copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->job_counter, sizeof(int));
    if (e != cudaSuccess) {
        note_cuda(e, "hd_batch_create");
        free_batch(b);
        return HD_ERR_CUDA;
    }
    *out = b;
    return HD_OK;
}

hd_status hd_batch_destroy(hd_batch *batch)
{
    if (!batch) return HD_OK;
    DeviceGuard g(batch->device);
    cudaDeviceSynchronize();
    free_batch(batch);
    return HD_OK;
}

hd_status hd_batch_add(hd_batch *batch, hd_scan *scan, const float *angle_deg,
                       const float *u_in, const float *v_in, const float *u_out,
                       const float *v_out, const float *wepl, int64_t n)
{
    return hd_batch_add_item(batch, scan, angle_deg, u_in, v_in, u_out, v_out, wepl, n, 0);
}

hd_status hd_batch_add_item(hd_batch *batch, hd_scan *scan, const float *angle_deg,
                            const float *u_in, const float *v_in, const float *u_out,
                            const float *v_out, const float *wepl, int64_t n, int32_t flags)
{
    if (!batch || !scan || n < 0) return HD_ERR_ARG;
    if (flags & ~(HD_BATCH_RESET | HD_BATCH_FINALIZE)) return HD_ERR_ARG;
    if (n > 0 && (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl)) return HD_ERR_ARG;
    if (scan->device != batch->device) return HD_ERR_ARG;
    if (scan->thick_k > 0 || scan->euclid_d0 > 0.0f)
        return HD_ERR_STATE;  // batches run the tiled thin paths
    if (static_cast<int>(batch->items.size()) >= batch->max_items) return HD_ERR_STATE;
    hd_batch::Item it;
    it.scan = scan;
    it.in = hd::Inputs{angle_deg, u_in, v_in, u_out, v_out, wepl};
    it.n = n;
    it.flags = flags;
    batch->items.push_back(it);
    return HD_OK;
}

hd_status hd_batch_set_graph(hd_batch *batch, int32_t enable)
{
    if (!batch) return HD_ERR_ARG;
    batch->use_graph = enable != 0;
    return HD_OK;
}

hd_status hd_batch_get_stats(hd_batch *batch, hd_batch_stats *out)
{
    if (!batch || !out) return HD_ERR_ARG;
    *out = batch->stats;
    return HD_OK;
}

hd_status hd_batch_run(hd_batch *batch, int32_t flags, void *stream)
{
    if (!batch) return HD_ERR_ARG;
    if (flags & ~(HD_BATCH_RESET | HD_BATCH_FINALIZE)) return HD_ERR_ARG;
    DeviceGuard g(batch->device);
    if (!g.ok) return HD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto items = batch->items;
    batch->items.clear();
    if (items.empty()) return HD_OK;
    for (size_t i = 0; i < items.size(); ++i) {
        items[i].first = items[i].last = true;
        for (size_t j = 0; j < i; ++j)
            if (items[j].scan == items[i].scan) items[i].first = false;
        for (size_t j = i + 1; j < items.size(); ++j)
            if (items[j].scan == items[i].scan) items[i].last = false;
    }
    // rounds: the k-th item of each scan goes to round k
    std::vector<std::vector<hd_batch::Item>> rounds;
    std::vector<std::pair<hd_scan *, int>> seen;
    for (const auto &it : items) {
        int k = 0;
        for (auto &p : seen)
            if (p.first == it.scan) k = ++p.second;
        if (k == 0) seen.push_back({it.scan, 0});
        if (static_cast<int>(rounds.size()) <= k) rounds.emplace_back();
        rounds[k].push_back(it);
    }
    // host-side preparation, outside any capture: buffers, limits, descriptors
    for (const auto &it : items) {
        hd_scan *s = it.scan;
        if (it.n > kChunk) return HD_ERR_RANGE;
        hd_status r = ensure_records(s, it.n > 0 ? it.n : 1, st);
        if (r != HD_OK) return r;
        r = upload_desc(s, st);
        if (r != HD_OK) return r;
    }
    for (const auto &p : seen) {
        uint64_t total = (flags & HD_BATCH_RESET) ? 0 : p.first->n_total;
        for (const auto &it : items)
            if (it.scan == p.first) total += static_cast<uint64_t>(it.n);
        if (total > static_cast<uint64_t>(kMaxScanHistories)) return HD_ERR_OVERFLOW;
    }
    std::vector<uintptr_t> key;
    key.push_back(static_cast<uintptr_t>(flags));
    for (const auto &it : items) {
        key.push_back(static_cast<uintptr_t>(it.flags));
        key.push_back(reinterpret_cast<uintptr_t>(it.scan));
        key.push_back(reinterpret_cast<uintptr_t>(it.in.angle));
        key.push_back(reinterpret_cast<uintptr_t>(it.in.u_in));
        key.push_back(reinterpret_cast<uintptr_t>(it.in.v_in));
        key.push_back(reinterpret_cast<uintptr_t>(it.in.u_out));
        key.push_back(reinterpret_cast<uintptr_t>(it.in.v_out));
        key.push_back(reinterpret_cast<uintptr_t>(it.in.wepl));
        key.push_back(static_cast<uintptr_t>(it.n));
        key.push_back(reinterpret_cast<uintptr_t>(it.scan->desc_dev));
        key.push_back(reinterpret_cast<uintptr_t>(it.scan->pair_buf));
        key.push_back(static_cast<uintptr_t>(it.scan->tp.threads));
    }
    // the legacy default stream cannot be captured: run directly there
    const bool graphable = batch->use_graph && rounds.size() == 1 && st != nullptr;
    int max_words = 1;
    for (const auto &it : items)
        if (it.scan->tp.ntiles > 0 && it.scan->tp.tile_words > max_words)
            max_words = it.scan->tp.tile_words;
    // one launch serves every scan: the first scan's block size
    batch->threads = items.front().scan->tp.threads;
    const int per_sm = hd::trace_tiles_occupancy(max_words, batch->threads);
    const int grid = (per_sm > 0 ? per_sm : 1) * batch->sm_count;
    batch->stats.runs += 1;
    if (graphable && batch->exec && key == batch->key) {
        HD_CUDA(cudaGraphLaunch(batch->exec, st));
        batch->stats.graph_replays += 1;
        batch->stats.kernel_launches += batch->graph_kernels;
    } else {
        // descriptor table of the (single-round) traversal; multi-round runs
        // upload one table per round below
        int64_t kernels = 0;
        if (graphable) {
            std::vector<hd::ScanDesc> descs;
            for (const auto &it : rounds[0]) descs.push_back(it.scan->desc_host);
            HD_CUDA(cudaMemcpyAsync(batch->descs_dev, descs.data(),
                                    sizeof(hd::ScanDesc) * descs.size(), cudaMemcpyHostToDevice, st));
            HD_CUDA(cudaStreamSynchronize(st));
            if (batch->exec) {
                cudaGraphExecDestroy(batch->exec);
                batch->exec = nullptr;
            }
            HD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            hd_status r = issue_round(batch, rounds[0], flags, grid, st, &kernels);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (r != HD_OK) {
                if (graph) cudaGraphDestroy(graph);
                return r;
            }
            if (ec != cudaSuccess) {
                note_cuda(ec, "hd_batch_run: capture");
                return HD_ERR_CUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&batch->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                note_cuda(ei, "hd_batch_run: instantiate");
                batch->exec = nullptr;
                return HD_ERR_CUDA;
            }
            batch->key = key;
            batch->graph_kernels = kernels;
            HD_CUDA(cudaGraphLaunch(batch->exec, st));
            batch->stats.graph_captures += 1;
        } else {
            for (size_t k = 0; k < rounds.size(); ++k) {
                // stream-ordered upload of the table: the pinned staging may be
                // refilled once the previous upload from it has run
                HD_CUDA(cudaEventSynchronize(batch->descs_copied));
                for (size_t i = 0; i < rounds[k].size(); ++i)
                    batch->descs_pinned[i] = rounds[k][i].scan->desc_host;
                HD_CUDA(cudaMemcpyAsync(batch->descs_dev, batch->descs_pinned,
                                        sizeof(hd::ScanDesc) * rounds[k].size(),
                                        cudaMemcpyHostToDevice, st));
                HD_CUDA(cudaEventRecord(batch->descs_copied, st));
                hd_status r = issue_round(batch, rounds[k], flags, grid, st, &kernels);
                if (r != HD_OK) return r;
            }
        }
        batch->stats.kernel_launches += kernels;
    }
    for (const auto &p : seen) {
        hd_scan *s = p.first;
        if (flags & HD_BATCH_RESET) s->n_total = 0;
        for (const auto &it : items)
            if (it.scan == s) s->n_total += static_cast<uint64_t>(it.n);
        bool fin = (flags & HD_BATCH_FINALIZE) != 0;
        for (const auto &it : items)
            if (it.scan == s && (it.flags & HD_BATCH_FINALIZE)) fin = true;
        s->finalized = fin;
    }
    return HD_OK;
}

}  // extern "C"
