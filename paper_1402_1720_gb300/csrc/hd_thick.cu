// Thick rays (Eq. 3.2 with d_0 > 0; the paper leaves the distance measure
// open): A_i(k) = the voxels within k voxels of a voxel of A_i in the same
// slice, by the in-plane Chebyshev distance.  Counted into N and M exactly
// as the thin paths are, once per history for every voxel of its A_i(k).
//
// Within one slice the walk of A_i is a run of consecutive rows (one run of
// voxels along the major in-plane axis per row, rows stepping by one in one
// direction, the runs abutting).  Dilating it by k, target row t receives
// the runs of rows t - k .. t + k, whose union grown by k is the single
// interval [min lo - k, max hi + k]; because lo and hi move monotonically
// along the walk, the minimum and maximum sit at the window's first and last
// run.  So each history emits one interval per target row and slice, into a
// difference array along the major axis (x-major walks along x, y-major ones
// along y), and row prefix sums turn the differences into counts.
//
//   thick_kernel      persistent warps, a lane per history (lanes refilled
//                     from a work counter when enough are idle): the exact
//                     run walk over the whole grid, a ring of the last 2k + 1
//                     runs of the current slice, one interval per target row
//                     (two atomics)
//   thick_rows_kernel thread per x-row / y-column: prefix sums added to N, M
#include <cuda_runtime.h>

#include "hd_geom.cuh"
#include "hd_thick.cuh"

namespace hd {
namespace {

constexpr int kThickThreads = 256;
constexpr int kMaxK = kThickMaxK;

// Difference arrays: along x, (nx + 1) entries per (y, z) row; along y,
// (ny + 1) entries per (x, z) column.  One pair for N and one for M.
struct ThickWs {
    int32_t *dx[2], *dy[2];
    unsigned long long *stats;  // 8 counters (see thick_kernel)
    unsigned long long *next;   // next history to hand out
};

// One lane's walk: the run walk and the state of its current slice.
// Targets of a slice of J runs are centred on runs -k .. J - 1 + k (target
// minor index m0 + s jc); the one centred on run jc = j - k has its whole
// window (runs max(0, j - 2k) .. j) once run j has arrived, the last k when
// the slice ends.  Run j sits in ring slot p = j mod (2k + 1), so run j - 2k
// is in the next slot.
struct ThickLane {
    RunWalk wk;
    int32_t *diff;
    int cls;  // 0 missed, 1 hit
    int nmaj, nminor, s;
    int zc, m0, j, p;
    int prev_row;
    int64_t row0;
};

__device__ __forceinline__ unsigned close_slice(const ThickLane &L, const ThickRing &rg, int k,
                                                unsigned &voxels)
{
    const int R = 2 * k + 1;
    const int pb = L.p == 0 ? R - 1 : L.p - 1;  // the slice's last run
    unsigned e = 0;
    for (int jc = L.j - k; jc <= L.j - 1 + k; ++jc) {
        const int ja = jc - k;
        const int pa = ja <= 0 ? 0 : (ja % R);
        e += thick_emit_global(rg, pa, pb, L.m0 + L.s * jc, k, L.nminor, L.nmaj, L.diff, L.row0,
                               voxels);
    }
    return e;
}

// Per-lane statistics: histories, missed, hit, neither, rejected.
struct ThickCounts {
    unsigned n_in = 0, n_miss = 0, n_hit = 0, n_none = 0, n_reject = 0;
};

// Starts history i on a lane: classification, geometry, walk set-up; false
// when it has nothing to add.
__device__ __forceinline__ bool start_history(const Inputs &in, int64_t i, const GeomQ &g,
                                              const Cordic &cd, float tau_l, float tau_h,
                                              int use_miss, int use_hit, const ThickWs &ws,
                                              ThickLane &L, float &tc_ang, bool &tc_valid,
                                              long long &tc_c, long long &tc_s, ThickCounts &nc)
{
    const float w = in.wepl[i];
    const int cls = w < tau_l ? 0 : (w > tau_h ? 1 : -1);
    nc.n_in += 1;
    nc.n_miss += cls == 0 ? 1 : 0;
    nc.n_hit += cls == 1 ? 1 : 0;
    nc.n_none += cls < 0 ? 1 : 0;
    if (cls < 0 || (cls == 0 && !use_miss) || (cls == 1 && !use_hit)) return false;
    const float ang = in.angle[i];
    bool ok = fabsf(ang) < 1048576.0f;
    int32_t r[6];
    if (ok) {
        if (!tc_valid || ang != tc_ang) {
            cordic_cs(q16_of(ang), cd, tc_c, tc_s);
            tc_ang = ang;
            tc_valid = true;
        }
        ok = endpoints_cs(g, tc_c, tc_s, in.u_in[i], in.v_in[i], in.u_out[i], in.v_out[i], r);
    }
    if (!ok) {
        nc.n_reject += 1;
        return false;
    }
    if (!run_begin(L.wk, r, r + 3, g.nx, g.ny, g.nz)) return false;
    L.cls = cls;
    const bool ymaj = (L.wk.flags >> 5) & 1;
    L.s = (L.wk.flags & 2) ? 1 : -1;  // the in-plane minor axis' direction
    L.nmaj = ymaj ? g.ny : g.nx;
    L.nminor = ymaj ? g.nx : g.ny;
    L.diff = ymaj ? ws.dy[cls] : ws.dx[cls];
    L.zc = -1;
    L.m0 = L.j = L.p = 0;
    L.prev_row = 0;
    L.row0 = 0;
    return true;
}

constexpr int kThickRefill = 8;     // idle lanes that trigger a refill
constexpr int kThickRunsPerStep = 4;

// Persistent warps: each lane walks one history at a time; once enough
// lanes are idle, they take the next histories together (one atomic per
// warp on the work counter), so lanes do not idle behind a long walk.
__global__ void __launch_bounds__(kThickThreads) thick_kernel(Inputs in, int64_t n, GeomQ g,
                                                              Cordic cd, float tau_l, float tau_h,
                                                              int use_miss, int use_hit, int k,
                                                              ThickWs ws,
                                                              unsigned long long *stats)
{
    const unsigned lane = threadIdx.x & 31u;
    ThickCounts nc;
    unsigned vox[2] = {0, 0};  // voxel memberships added, missed and hit
    long long tc_c = 0, tc_s = 0;
    float tc_ang = 0.0f;
    bool tc_valid = false;
    ThickRing rg;
    ThickLane L;
    bool active = false, drained = false;
    unsigned emitted = 0;
    const int R = 2 * k + 1;
    for (;;) {
        const unsigned idle = __ballot_sync(0xffffffffu, !active);
        if (drained && idle == 0xffffffffu) break;
        if (!drained && (__popc(idle) >= kThickRefill || idle == 0xffffffffu)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(ws.next, static_cast<unsigned long long>(__popc(idle)));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= static_cast<unsigned long long>(n)) drained = true;
            if (!active) {
                const unsigned long long i = base + __popc(idle & ((1u << lane) - 1u));
                if (i < static_cast<unsigned long long>(n))
                    active = start_history(in, static_cast<int64_t>(i), g, cd, tau_l, tau_h,
                                           use_miss, use_hit, ws, L, tc_ang, tc_valid, tc_c,
                                           tc_s, nc);
            }
            continue;
        }
        if (!active) continue;
#pragma unroll 1
        for (int u = 0; u < kThickRunsPerStep; ++u) {
            int row, lo, hi;
            if (!run_next(L.wk, row, lo, hi)) {
                if (L.zc >= 0) emitted += close_slice(L, rg, k, vox[L.cls]);
                active = false;
                break;
            }
            // rows are minor + nminor z: inside a slice consecutive runs
            // differ by one row, so only a larger step can start a new slice
            const int step = row - L.prev_row;
            L.prev_row = row;
            if (L.zc < 0 || step > 1 || step < -1 || L.nminor <= 2) {
                const int mz = row / L.nminor;
                if (mz != L.zc) {
                    if (L.zc >= 0) emitted += close_slice(L, rg, k, vox[L.cls]);
                    L.zc = mz;
                    L.m0 = row - mz * L.nminor;
                    L.row0 = static_cast<int64_t>(mz) * L.nminor;
                    L.j = 0;
                    L.p = 0;
                }
            }
            rg.lo[L.p] = lo;
            rg.hi[L.p] = hi;
            const int pa = L.j >= 2 * k ? (L.p + 1 == R ? 0 : L.p + 1) : 0;
            emitted += thick_emit_global(rg, pa, L.p, L.m0 + L.s * (L.j - k), k, L.nminor,
                                         L.nmaj, L.diff, L.row0, vox[L.cls]);
            ++L.j;
            L.p = L.p + 1 == R ? 0 : L.p + 1;
        }
    }
    // stats[0..6]: histories, missed, hit, neither, rejected, voxels of
    // missed and of hit histories; stats[7]: row intervals
    const unsigned long long part[8] = {nc.n_in, nc.n_miss, nc.n_hit, nc.n_none, nc.n_reject,
                                        vox[0], vox[1], emitted};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        unsigned long long e = part[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0 && e != 0) atomicAdd(stats + q, e);
    }
}

// The records of a chunk that take the global path (status 2: too many
// tiles, or beyond the pair budget): each walked whole over the grid into the
// global difference arrays; voxel memberships added to the scan's counters.
__global__ void __launch_bounds__(kThickThreads) thick_records_kernel(Records rec, Ctrl *ctrl,
                                                                      GeomQ g, int k,
                                                                      ThickDiff td)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t total = rec.glist ? static_cast<int64_t>(ctrl->n_global) : rec.cap;
    ThickRing rg;
    unsigned vox[2] = {0, 0};
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < total;
         k += stride) {
        const int64_t i = rec.glist ? static_cast<int64_t>(rec.glist[k]) : k;
        const int32_t stw = rec.status[i];
        if (status_path(stw) != 2) continue;
        const int32_t gi[3] = {rec.g[0][i], rec.g[1][i], rec.g[2][i]};
        const int32_t go[3] = {rec.g[3][i], rec.g[4][i], rec.g[5][i]};
        RunWalk wk;
        if (!run_begin(wk, gi, go, g.nx, g.ny, g.nz)) continue;
        const bool ymaj = (wk.flags >> 5) & 1;
        const int cls = status_cls(stw);
        thick_walk_all(wk, ymaj ? g.nx : g.ny, ymaj ? g.ny : g.nx, 0, k, (wk.flags & 2) ? 1 : -1,
                       ymaj ? td.dy[cls] : td.dx[cls], rg, vox[cls]);
    }
}

__global__ void __launch_bounds__(kThickThreads) thick_rows_kernel(
    const int32_t *__restrict__ diff, int64_t rows, int nmaj, int stride_maj, int nminor,
    int64_t plane, int major_is_y, uint32_t *__restrict__ out)
{
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows || out == nullptr) return;
    const int64_t z = r / nminor;
    const int m = static_cast<int>(r - z * nminor);
    const int32_t *d = diff + r * static_cast<int64_t>(nmaj + 1);
    // x-major rows: voxel x + nx (m + ny z); y-major columns: m + nx (y + ny z)
    uint32_t *o = out + z * plane + (major_is_y ? m : static_cast<int64_t>(m) * nmaj);
    int acc = 0;
    for (int a = 0; a < nmaj; ++a) {
        acc += d[a];
        if (acc != 0) o[static_cast<int64_t>(a) * stride_maj] += static_cast<uint32_t>(acc);
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t thick_layout(const hd_geometry *g, void *base, ThickWs *ws)
{
    const size_t nz = static_cast<size_t>(g->nz);
    const size_t bx = align256(sizeof(int32_t) * (g->nx + 1) * static_cast<size_t>(g->ny) * nz);
    const size_t by = align256(sizeof(int32_t) * (g->ny + 1) * static_cast<size_t>(g->nx) * nz);
    if (ws && base) {
        char *p = static_cast<char *>(base);
        ws->dx[0] = reinterpret_cast<int32_t *>(p);
        ws->dx[1] = reinterpret_cast<int32_t *>(p + bx);
        ws->dy[0] = reinterpret_cast<int32_t *>(p + 2 * bx);
        ws->dy[1] = reinterpret_cast<int32_t *>(p + 2 * bx + by);
        ws->stats = reinterpret_cast<unsigned long long *>(p + 2 * bx + 2 * by);
        ws->next = ws->stats + 8;
    }
    return 2 * bx + 2 * by + 256;
}

__global__ void thick_stats_kernel(const unsigned long long *from, unsigned long long *to,
                                   int64_t *intervals)
{
    if (threadIdx.x < 7 && to != nullptr && from[threadIdx.x] != 0)
        atomicAdd(to + threadIdx.x, from[threadIdx.x]);
    if (threadIdx.x == 7 && intervals != nullptr)
        *intervals = static_cast<int64_t>(from[7]);
}

}  // namespace

size_t thick_workspace_bytes(const hd_geometry *geom) { return thick_layout(geom, nullptr, nullptr); }

cudaError_t launch_thick(const Inputs &in, int64_t n, const hd_geometry *geom, const GeomQ &g,
                         const Cordic &cd, float tau_l, float tau_h, int use_miss, int use_hit,
                         int k, void *workspace, uint32_t *N, uint32_t *M,
                         unsigned long long *stats, int64_t *intervals, int sm_count,
                         cudaStream_t st)
{
    ThickWs ws{};
    const size_t need = thick_layout(geom, workspace, &ws);
    cudaError_t e = cudaMemsetAsync(workspace, 0, need, st);
    if (e == cudaSuccess && n > 0) {
        int64_t blocks = (n + kThickThreads - 1) / kThickThreads;
        const int64_t cap = int64_t(sm_count > 0 ? sm_count : 1) * 4;
        if (blocks > cap) blocks = cap;  // resident, persistent
        thick_kernel<<<static_cast<unsigned>(blocks), kThickThreads, 0, st>>>(
            in, n, g, cd, tau_l, tau_h, use_miss, use_hit, k, ws, ws.stats);
        e = cudaGetLastError();
    }
    const int64_t plane = int64_t(geom->nx) * geom->ny;
    for (int c = 0; c < 2 && e == cudaSuccess && n > 0; ++c) {
        uint32_t *out = c == 0 ? (use_miss ? N : nullptr) : (use_hit ? M : nullptr);
        if (!out) continue;
        const int64_t rx = int64_t(geom->ny) * geom->nz, ry = int64_t(geom->nx) * geom->nz;
        thick_rows_kernel<<<static_cast<unsigned>((rx + 255) / 256), 256, 0, st>>>(
            ws.dx[c], rx, geom->nx, 1, geom->ny, plane, 0, out);
        thick_rows_kernel<<<static_cast<unsigned>((ry + 255) / 256), 256, 0, st>>>(
            ws.dy[c], ry, geom->ny, geom->nx, geom->nx, plane, 1, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && (stats || intervals)) {
        thick_stats_kernel<<<1, 32, 0, st>>>(ws.stats, stats, intervals);
        e = cudaGetLastError();
    }
    return e;
}

unsigned long long *thick_counters_of(const hd_geometry *geom, void *workspace)
{
    ThickWs ws{};
    thick_layout(geom, workspace, &ws);
    return ws.stats;
}

ThickDiff thick_diff_of(const hd_geometry *geom, void *workspace)
{
    ThickWs ws{};
    thick_layout(geom, workspace, &ws);
    ThickDiff td{};
    for (int c = 0; c < 2; ++c) {
        td.dx[c] = ws.dx[c];
        td.dy[c] = ws.dy[c];
    }
    return td;
}

// Adds the global difference arrays to N and M (row prefix sums).
static cudaError_t launch_thick_rows(const hd_geometry *geom, const ThickWs &ws, uint32_t *N,
                                     uint32_t *M, cudaStream_t st)
{
    const int64_t plane = int64_t(geom->nx) * geom->ny;
    for (int c = 0; c < 2; ++c) {
        uint32_t *out = c == 0 ? N : M;
        if (!out) continue;
        const int64_t rx = int64_t(geom->ny) * geom->nz, ry = int64_t(geom->nx) * geom->nz;
        thick_rows_kernel<<<static_cast<unsigned>((rx + 255) / 256), 256, 0, st>>>(
            ws.dx[c], rx, geom->nx, 1, geom->ny, plane, 0, out);
        thick_rows_kernel<<<static_cast<unsigned>((ry + 255) / 256), 256, 0, st>>>(
            ws.dy[c], ry, geom->ny, geom->nx, geom->nx, plane, 1, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_thick_finish(const hd_geometry *geom, void *workspace, uint32_t *N,
                                uint32_t *M, unsigned long long *stats, int64_t *intervals,
                                cudaStream_t st)
{
    ThickWs ws{};
    thick_layout(geom, workspace, &ws);
    cudaError_t e = launch_thick_rows(geom, ws, N, M, st);
    if (e == cudaSuccess && (stats || intervals)) {
        thick_stats_kernel<<<1, 32, 0, st>>>(ws.stats, stats, intervals);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_thick_scan(const ScanDesc *desc_dev, const hd_geometry *geom,
                              const Records &rec, Ctrl *ctrl, int64_t upper, const GeomQ &g,
                              int k, void *workspace, uint32_t *N, uint32_t *M, int smem_words,
                              int threads, int sm_count, cudaStream_t st)
{
    ThickWs ws{};
    const size_t need = thick_layout(geom, workspace, &ws);
    const ThickDiff td = thick_diff_of(geom, workspace);
    cudaError_t e = cudaMemsetAsync(workspace, 0, need, st);
    if (e == cudaSuccess)
        e = launch_trace_thick(desc_dev, &ctrl->job_next, k, td, smem_words, threads,
                               sm_count > 0 ? sm_count : 1, st);
    if (e == cudaSuccess && upper > 0) {
        int64_t blocks = (upper + kThickThreads - 1) / kThickThreads;
        const int64_t cap = int64_t(sm_count > 0 ? sm_count : 1) * 8;
        if (blocks > cap) blocks = cap;
        thick_records_kernel<<<static_cast<unsigned>(blocks), kThickThreads, 0, st>>>(rec, ctrl, g,
                                                                                      k, td);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_thick_rows(geom, ws, N, M, st);
    return e;
}

}  // namespace hd

extern "C" {

hd_status hd_accumulate_thick_workspace(const hd_geometry *geom, size_t *bytes)
{
    if (!geom || !bytes) return HD_ERR_ARG;
    const hd_status s = hd::check_geometry(geom);
    if (s != HD_OK) return s;
    *bytes = hd::thick_workspace_bytes(geom);
    return HD_OK;
}

hd_status hd_accumulate_thick(const hd_geometry *geom, const hd_params *params, int32_t k,
                              const float *angle_deg, const float *u_in, const float *v_in,
                              const float *u_out, const float *v_out, const float *wepl,
                              int64_t n, uint32_t *N, uint32_t *M, void *workspace,
                              size_t workspace_bytes, int64_t *intervals, void *stream)
{
    if (!geom || !params || n < 0 || !workspace) return HD_ERR_ARG;
    if (k < 0 || k > hd::kMaxK) return HD_ERR_RANGE;
    const hd_status gs = hd::check_geometry(geom);
    if (gs != HD_OK) return gs;
    if (std::isnan(params->wepl_miss_lt) || std::isnan(params->wepl_hit_gt) ||
        params->wepl_miss_lt > params->wepl_hit_gt)
        return HD_ERR_ARG;
    const uint32_t m = params->methods;
    if (m == 0 || (m & ~uint32_t(HD_SC | HD_MSC | HD_SM))) return HD_ERR_ARG;
    const int use_miss = (m & (HD_SC | HD_MSC)) ? 1 : 0;
    const int use_hit = (m & HD_SM) ? 1 : 0;
    if ((use_miss && !N) || (use_hit && !M)) return HD_ERR_ARG;
    if (n > 0 && (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl)) return HD_ERR_ARG;
    if (workspace_bytes < hd::thick_workspace_bytes(geom) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return HD_ERR_ARG;
    hd::Cordic cd{};
    if (!hd::make_cordic_table(cd)) return HD_ERR_RANGE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    const hd::GeomQ gq = hd::make_geomq(geom->nx, geom->ny, geom->nz, geom->sx, geom->sy,
                                        geom->sz, geom->tracker_half_sep_mm);
    const hd::Inputs in{angle_deg, u_in, v_in, u_out, v_out, wepl};
    const cudaError_t e = hd::launch_thick(in, n, geom, gq, cd, params->wepl_miss_lt,
                                           params->wepl_hit_gt, use_miss, use_hit, k, workspace, N,
                                           M, nullptr, intervals, sms,
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        hd::note_cuda_error(e, "hd_accumulate_thick");
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // extern "C"
