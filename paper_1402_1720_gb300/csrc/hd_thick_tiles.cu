// Thick rays on the tiled traversal: for a scan whose tiles are whole
// one-slice planes, each (record, slice) pair's lean walk is dilated by k
// voxels in-plane and counted in the block's shared-memory difference
// arrays, the way the thin traversal counts its runs.
//
// A lane walks one pair's runs (rows step by one, runs abut) with the last
// 2k + 1 runs in a ring; target row t receives the union of the runs of rows
// t - k .. t + k grown by k, one interval: +1 at its first voxel and -1 past
// its last in the int16 difference array of the walk's major axis.  Each
// pair adds at most one to a voxel, so a job of at most 32767 pairs keeps
// every difference and prefix sum inside int16, as in the thin traversal.
// Lanes are refilled from the job's pair range when enough are idle.  The
// pairs without a lean form are walked afterwards with the general run walk
// into global difference arrays.
#include "hd_fallback.cuh"
#include "hd_thick.cuh"

namespace hd {
namespace {

constexpr unsigned kAllLanes = 0xffffffffu;
constexpr int kThickRunsPerStep = 4;

__device__ __forceinline__ void load_pair(const Pairs &pairs, int idx, uint4 &a, uint4 &b)
{
    a = __ldg(&pairs.v[2 * static_cast<size_t>(idx)]);
    b = __ldg(&pairs.v[2 * static_cast<size_t>(idx) + 1]);
}

// In-place inclusive prefix sums of int16 rows: `rows` rows of `len`
// elements, one warp per row.
__device__ __forceinline__ void prefix_rows16(int16_t *a, int rows, int len)
{
    const unsigned lane = threadIdx.x & 31u;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int chunk = (len + 31) >> 5;
    for (int r = warp; r < rows; r += nw) {
        int16_t *row = a + static_cast<long long>(r) * len;
        const int b = lane * chunk;
        const int e = min(b + chunk, len);
        int acc = 0;
        for (int i = b; i < e; ++i) acc += row[i];
        int incl = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kAllLanes, incl, o);
            if (lane >= static_cast<unsigned>(o)) incl += t;
        }
        int run = incl - acc;
        for (int i = b; i < e; ++i) {
            run += row[i];
            row[i] = static_cast<int16_t>(run);
        }
    }
}

// Interval of target row t (minor index) into the tile's difference array
// of the walk's major axis (word offset aoff; the -1 of an interval ending
// at its row's end goes to the scratch word).  Returns its voxels.
__device__ __forceinline__ unsigned emit_tile(const ThickRing &rg, int pa, int pb, int t, int k,
                                              int nminor, int nmaj, uint32_t *tile, int aoff,
                                              int scratch)
{
    if (t < 0 || t >= nminor) return 0;
    const int lo = max(min(rg.lo[pa], rg.lo[pb]) - k, 0);
    const int hi = min(max(rg.hi[pa], rg.hi[pb]) + k, nmaj - 1);
    const int e0 = t * nmaj + lo, e1 = t * nmaj + hi + 1;
    atomicAdd(&tile[aoff + (e0 >> 1)], (e0 & 1) ? 65536u : 1u);
    atomicAdd(&tile[hi + 1 < nmaj ? aoff + (e1 >> 1) : scratch],
              (e1 & 1) ? 0xffff0000u : 0xffffffffu);
    return static_cast<unsigned>(hi - lo + 1);
}

// The pairs [start, start + total) of a job, dilated, into the tile.
// Returns the voxel memberships added by this lane.
__device__ __forceinline__ unsigned thick_walk_job(uint32_t *tile, int arr_words, int dx, int dy,
                                                   const Pairs &pairs, int start, int total,
                                                   int refill, unsigned *s_next, int k)
{
    const unsigned lane = threadIdx.x & 31u;
    const int scratch = 2 * arr_words;
    const int R = 2 * k + 1;
    LeanCursor c;
    ThickRing rg;
    bool active = false;
    int nmaj = 0, nminor = 0, aoff = 0;
    int r0 = 0, s = 1, j = 0, p = 0;  // first row and direction of the walk, step, ring slot
    int jlast = -1, pb_last = 0;      // runs of the walk once they are all walked, last slot
    unsigned vox = 0, ends = 0;
    uint4 na = make_uint4(0, 0, 0, 0), nb = na;
    int nidx = -1;
    {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(s_next, 32u);
        base = __shfl_sync(kAllLanes, base, 0);
        const unsigned r = base + lane;
        if (r < static_cast<unsigned>(total)) {
            nidx = start + static_cast<int>(r);
            load_pair(pairs, nidx, na, nb);
        }
    }
    for (;;) {
        const unsigned want = __ballot_sync(kAllLanes, !active && nidx >= 0);
        const unsigned busy = __ballot_sync(kAllLanes, active);
        if ((want | busy) == 0) break;
        if (want != 0 && (__popc(want) >= static_cast<unsigned>(refill) || busy == 0)) {
            if (!active && nidx >= 0) {
                const uint32_t o[kLeanWords] = {na.x, na.y, na.z, na.w, nb.x, nb.y, nb.z, nb.w};
                const bool ymaj = (o[5] >> 18) & 1u;  // LeanWalk::fl bit 2
                nmaj = ymaj ? dy : dx;
                nminor = ymaj ? dx : dy;
                aoff = ymaj ? arr_words : 0;
                active = lean_start(o, 1, c);  // rows counted one by one
                r0 = c.rb;
                s = c.rstep;
                j = 0;
                p = 0;
                jlast = -1;
                nidx = -1;
            }
            unsigned base = 0;
            const unsigned nw = __popc(want);
            if (lane == 0) base = atomicAdd(s_next, nw);
            base = __shfl_sync(kAllLanes, base, 0);
            if (want & (1u << lane)) {
                const unsigned r = base + __popc(want & ((1u << lane) - 1u));
                if (r < static_cast<unsigned>(total)) {
                    nidx = start + static_cast<int>(r);
                    load_pair(pairs, nidx, na, nb);
                }
            }
            continue;
        }
        if (active) {
            // Step j emits the target centred on run j - k (row r0 + s (j - k)),
            // whose window is runs max(0, j - 2k) .. min(j, J - 1): steps
            // 0 .. J - 1 walk the J runs, steps J .. J - 1 + 2k only emit, so
            // every step of every lane costs the same and lanes stay together.
#pragma unroll 1
            for (int u = 0; u < kThickRunsPerStep; ++u) {
                int pb = pb_last;
                if (jlast < 0) {
                    int rb, lo, hi;
                    const bool more = lean_run(c, rb, lo, hi, ends);
                    rg.lo[p] = lo;
                    rg.hi[p] = hi;
                    pb = p;
                    if (!more) {
                        jlast = j + 1;
                        pb_last = p;
                    }
                }
                vox += emit_tile(rg, j >= 2 * k ? (p + 1 == R ? 0 : p + 1) : 0, pb,
                                 r0 + s * (j - k), k, nminor, nmaj, tile, aoff, scratch);
                ++j;
                p = p + 1 == R ? 0 : p + 1;
                if (jlast >= 0 && j >= jlast + 2 * k) {
                    active = false;
                    break;
                }
            }
        }
    }
    return vox;
}

// The fallback pairs (no lean form), 32 per warp claim, each walked with the
// general run walk in its one-slice tile into the global difference arrays.
__device__ __noinline__ void thick_fallback(const ScanDesc *__restrict__ dp, int k,
                                            ThickDiff td)
{
    const unsigned lane = threadIdx.x & 31u;
    const ScanDesc &d = *dp;
    const unsigned nf = d.ctrl->n_pair_fallback;
    if (nf == 0) return;
    const TilePlan tp = d.tp;
    ThickRing rg;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&d.ctrl->fb_next, 32u);
        base = __shfl_sync(kAllLanes, base, 0);
        if (base >= nf) break;
        const unsigned i = base + lane;
        unsigned vox[2] = {0, 0};
        if (i < nf) {
            const uint32_t pos = d.pairs.fb[i].x;
            uint4 a, b;
            load_pair(d.pairs, static_cast<int>(pos), a, b);
            const int32_t gi[3] = {static_cast<int32_t>(a.x), static_cast<int32_t>(a.y),
                                   static_cast<int32_t>(a.z)};
            const int32_t go[3] = {static_cast<int32_t>(a.w), static_cast<int32_t>(b.x),
                                   static_cast<int32_t>(b.z)};
            const int cls = static_cast<int>(b.w & 1u);
            const int z0 = static_cast<int>(b.w >> 1);  // tiles are whole slices
            RunWalk wk;
            if (run_begin(wk, gi, go, tp.nx, tp.ny, 1)) {
                const bool ymaj = (wk.flags >> 5) & 1;
                thick_walk_all(wk, ymaj ? tp.nx : tp.ny, ymaj ? tp.ny : tp.nx, z0, k,
                               (wk.flags & 2) ? 1 : -1, ymaj ? td.dy[cls] : td.dx[cls], rg,
                               vox[cls]);
            }
        }
    }
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1) trace_thick_kernel(const ScanDesc *__restrict__ dp,
                                                                  int *job_counter, int k,
                                                                  ThickDiff td)
{
    extern __shared__ uint32_t tile[];
    __shared__ int s_job;
    __shared__ unsigned s_next;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const ScanDesc &d = *dp;
    const int njobs = d.ctrl->njobs;
    const TilePlan tp = d.tp;
    const int dx = tp.nx, dy = tp.ny;  // whole-plane tiles, one slice deep
    const int nvox = dx * dy;
    const int arr_words = (nvox + 1) >> 1;
    uint32_t *arrX = tile;
    uint32_t *arrY = tile + arr_words;
    for (;;) {
        if (threadIdx.x == 0) {
            s_job = atomicAdd(job_counter, 1);
            s_next = 0;
        }
        __syncthreads();
        if (s_job >= njobs) break;
        const TileJob job = d.jobs[s_job];
        const int z = job.tile;
        for (int w = threadIdx.x; w < 2 * arr_words + 1; w += blockDim.x) tile[w] = 0;
        __syncthreads();
        const unsigned vox = thick_walk_job(tile, arr_words, dx, dy, d.pairs, job.start,
                                            job.end - job.start, tp.refill, &s_next, k);
        __syncthreads();
        // a word holds lo + 65536 hi (mod 2^32) after carries between the
        // halves: split it into two plain int16 values
        for (int wd = threadIdx.x; wd < 2 * arr_words; wd += blockDim.x) {
            const uint32_t v = tile[wd];
            const int lo = static_cast<int16_t>(v & 0xffffu);
            const int hi = static_cast<int>(v - static_cast<uint32_t>(lo)) >> 16;
            tile[wd] = (static_cast<uint32_t>(lo) & 0xffffu) | (static_cast<uint32_t>(hi) << 16);
        }
        __syncthreads();
        prefix_rows16(reinterpret_cast<int16_t *>(arrX), dy, dx);
        prefix_rows16(reinterpret_cast<int16_t *>(arrY), dx, dy);
        __syncthreads();
        const int16_t *X = reinterpret_cast<const int16_t *>(arrX);
        const int16_t *Y = reinterpret_cast<const int16_t *>(arrY);
        uint32_t *vol = job.cls == 0 ? d.N : d.M;
        for (int row = warp; vol != nullptr && row < dy; row += nwarps) {
            const long long gbase = static_cast<long long>(tp.nx) *
                                    (row + static_cast<long long>(tp.ny) * z);
            for (int lx = lane; lx < dx; lx += 32) {
                const int v = X[row * dx + lx] + Y[lx * dy + row];
                if (v) atomicAdd(&vol[gbase + lx], static_cast<uint32_t>(v));
            }
        }
        __syncthreads();
    }
    thick_fallback(dp, k, td);
}

}  // namespace

cudaError_t launch_trace_thick(const ScanDesc *desc_dev, int *job_counter, int k,
                               const ThickDiff &td, int smem_words, int threads, int grid,
                               cudaStream_t st)
{
    if (smem_words * 4 > kTileSmemBytes || k < 0 || k > kThickMaxK) return cudaErrorInvalidValue;
    const size_t smem = static_cast<size_t>(smem_words) * 4;
    switch (threads) {
#define HD_THICK_CASE(T)                                                                          \
    case T: {                                                                                     \
        cudaError_t e = cudaFuncSetAttribute(trace_thick_kernel<T>,                               \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                             kTileSmemBytes);                                      \
        if (e != cudaSuccess) return e;                                                           \
        trace_thick_kernel<T><<<grid, T, smem, st>>>(desc_dev, job_counter, k, td);               \
        break;                                                                                    \
    }
        HD_THICK_CASE(256)
        HD_THICK_CASE(512)
        HD_THICK_CASE(768)
        HD_THICK_CASE(1024)
#undef HD_THICK_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hd
