// Shared-memory privatised traversal: the grid is cut into tiles whose
// counters fit in one block's shared memory, every (record, tile) pair is
// walked with the exact traversal clipped to the tile, and each block adds
// its private tile into N or M once per job.  Persistent blocks take jobs
// (ranges of one tile's pairs, made in hd_scatter.cu); warps refill idle
// lanes from the job's pair range, so lanes do not wait for the longest
// path.
#include "hd_fallback.cuh"

namespace hd {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRunsPerStep = 8;  // runs a traversal lane walks between refill checks

// ---------------------------------------------------------------- traversal
//
// A block's private tile holds one 32-bit word per voxel of the tile box,
// laid out x fastest with one padding column and one padding row:
// word(x, y, z) = x + Wx (y + Hy z), Wx = dx + 1, Hy = dy + 1.  Its low
// 16 bits are the difference counts of runs along x, its high 16 bits those
// of runs along y (z is never a run axis: it is always a minor one).  A run
// lo..hi adds +1 (x runs) or +65536 (y runs) at its first voxel and the
// negative just past its last one, which for a run ending at the box's edge
// is the padding column or row, so no run needs a bounds test.  Each job
// covers at most 32767 pairs, so every difference and every prefix sum of
// either half stays inside int16, and a word read as lo + 65536 hi (mod
// 2^32) decodes exactly even after carries between the halves.  Rows of
// words are an odd number of words apart (for the 200-voxel planes here),
// so lanes walking parallel paths at the same major index hit distinct
// banks.

__device__ __forceinline__ void load_lean(const Pairs &pairs, int idx, uint4 &a, uint4 &b)
{
    a = __ldg(&pairs.v[2 * static_cast<size_t>(idx)]);
    b = __ldg(&pairs.v[2 * static_cast<size_t>(idx) + 1]);
}

// Shared-memory reduction (no value returned) at a shared-space byte address.
__device__ __forceinline__ void smem_red_add(int addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Walks the pairs [start, start + total) of a job into the block's tile:
// each lane walks one pair and holds the packed lean walk of its next one
// (loaded a refill ahead, so starting a walk never waits on memory).  A
// refill happens once enough lanes are idle; then every idle lane with a
// prefetched pair starts it and fetches another, the pair index coming from
// the block's counter *s_next.  Adds the runs walked to `runs`.
__device__ __forceinline__ void walk_job(uint32_t *tile, int dx, int dy, int dz,
                                         const Pairs &pairs, int start, int total, int refill,
                                         unsigned *s_next, unsigned &runs)
{
    const unsigned lane = threadIdx.x & 31u;
    const int sbase = static_cast<int>(__cvta_generic_to_shared(tile));
    TileCursor c;
    bool active = false;
    uint4 na = make_uint4(0, 0, 0, 0), nb = na;
    int nidx = -1;
    {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(s_next, 32u);
        base = __shfl_sync(kFull, base, 0);
        const unsigned r = base + lane;
        if (r < static_cast<unsigned>(total)) {
            nidx = start + static_cast<int>(r);
            load_lean(pairs, nidx, na, nb);
        }
    }
    for (;;) {
        const unsigned want = __ballot_sync(kFull, !active && nidx >= 0);
        const unsigned busy = __ballot_sync(kFull, active);
        if ((want | busy) == 0) break;
        if (want != 0 && (__popc(want) >= static_cast<unsigned>(refill) || busy == 0)) {
            if (!active && nidx >= 0) {
                const uint32_t o[kLeanWords] = {na.x, na.y, na.z, na.w, nb.x, nb.y, nb.z, nb.w};
                active = tile_cursor_start(o, dx, dy, dz, sbase, c);
                // runs of a walk = its minor-0 crossings left at the start
                // minus those left after its last run (see tile_cursor_run)
                if (active) runs += static_cast<unsigned>(c.kleft);
                nidx = -1;
            }
            unsigned base = 0;
            const unsigned nw = __popc(want);
            if (lane == 0) base = atomicAdd(s_next, nw);
            base = __shfl_sync(kFull, base, 0);
            if (want & (1u << lane)) {
                const unsigned r = base + __popc(want & ((1u << lane) - 1u));
                if (r < static_cast<unsigned>(total)) {
                    nidx = start + static_cast<int>(r);
                    load_lean(pairs, nidx, na, nb);
                }
            }
            continue;
        }
        // up to kRunsPerStep runs before the warp checks for refills again.
        // A lane whose walk ends leaves the loop (predicating it instead was
        // 25 % slower), and an unroll by 2 measured best (full unrolling,
        // none, 6, 12 or 16 runs: 5-27 % slower on the head-200 scan).
        if (active) {
#pragma unroll 2
            for (int u = 0; u < kRunsPerStep; ++u) {
                int at_prev, at_cur;
                active = tile_cursor_run(c, at_prev, at_cur);
                smem_red_add(at_prev, c.vprev);
                smem_red_add(at_cur, c.vcur);
                if (!active) {
                    runs -= static_cast<unsigned>(c.kleft);
                    break;
                }
            }
        }
    }
}

// Flush of a job's tile into vol (the scan's N or M) and zeroing of the
// tile for the next job: (1) warps take rows, decode each word into two
// plain int16 halves and prefix-sum the low halves along x; (2) warps take
// columns and prefix-sum the high halves along y; (3) every voxel adds the
// sum of its two halves to vol (one global atomic per nonzero voxel) and
// every word, padding included, is cleared.
__device__ __forceinline__ void flush_tile(uint32_t *tile, int dx, int dy, int dz, uint32_t *vol,
                                           int nx, int ny, int x0, int y0, int z0)
{
    const unsigned lane = threadIdx.x & 31u;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int Wx = dx + 1, Hy = dy + 1;
    // (1) rows along x: decode, then inclusive prefix of the low halves
    {
        const int chunk = (dx + 31) >> 5;
        for (int r = warp; r < dy * dz; r += nwarps) {
            const int y = r % dy, z = r / dy;
            uint32_t *row = tile + Wx * (y + Hy * z);
            const int b = lane * chunk;
            const int e = min(b + chunk, dx);
            int acc = 0;
            for (int i = b; i < e; ++i) acc += static_cast<int16_t>(row[i] & 0xffffu);
            int incl = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= static_cast<unsigned>(o)) incl += t;
            }
            int run = incl - acc;
            for (int i = b; i < e; ++i) {
                const uint32_t w = row[i];
                const int lo = static_cast<int16_t>(w & 0xffffu);
                const int hi = static_cast<int>(w - static_cast<uint32_t>(lo)) >> 16;
                run += lo;
                row[i] = (static_cast<uint32_t>(run) & 0xffffu) | (static_cast<uint32_t>(hi) << 16);
            }
        }
        // (the padding column and row are never read: step 3 clears them)
    }
    __syncthreads();
    // (2) columns along y: inclusive prefix of the (decoded) high halves
    {
        const int chunk = (dy + 31) >> 5;
        for (int col = warp; col < dx * dz; col += nwarps) {
            const int x = col % dx, z = col / dx;
            uint32_t *base = tile + x + Wx * Hy * z;
            const int b = lane * chunk;
            const int e = min(b + chunk, dy);
            int acc = 0;
            for (int i = b; i < e; ++i) acc += static_cast<int>(base[Wx * i]) >> 16;
            int incl = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= static_cast<unsigned>(o)) incl += t;
            }
            int run = incl - acc;
            for (int i = b; i < e; ++i) {
                const uint32_t w = base[Wx * i];
                run += static_cast<int>(w) >> 16;
                base[Wx * i] = (w & 0xffffu) | (static_cast<uint32_t>(run) << 16);
            }
        }
    }
    __syncthreads();
    // (3) add to the volume and clear every word of the box, a warp per row
    // of words (padding row included), its lanes along x
    for (int r = warp; r < Hy * dz; r += nwarps) {
        const int y = r % Hy, z = r / Hy;
        uint32_t *row = tile + Wx * r;
        const bool real = y < dy;
        const long long g0 =
            x0 + static_cast<long long>(nx) * ((y0 + y) + static_cast<long long>(ny) * (z0 + z));
        for (int x = static_cast<int>(lane); x < Wx; x += 32) {
            const uint32_t w = row[x];
            row[x] = 0u;
            if (real && x < dx) {
                const int v = static_cast<int>(w & 0xffffu) + static_cast<int>(w >> 16);
                if (v) atomicAdd(&vol[g0 + x], static_cast<uint32_t>(v));
            }
        }
    }
}

// No job left: the pairs without a lean form (the fallback lists), walked
// with the general run walk in global memory, 32 entries per warp claim, so
// blocks that finish their last job early take them.  Out of line, so its
// registers do not weigh on the lean walk loop.
__device__ __noinline__ void walk_fallback_lists(const ScanDesc *__restrict__ descs, int nscans)
{
    const unsigned lane = threadIdx.x & 31u;
    for (int k = 0; k < nscans; ++k) {
        const ScanDesc &d = descs[k];
        const unsigned nf = d.ctrl->n_pair_fallback;
        if (nf == 0) continue;
        uint32_t *const N = d.N;
        uint32_t *const M = d.M;
        for (;;) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&d.ctrl->fb_next, 32u);
            base = __shfl_sync(kFull, base, 0);
            if (base >= nf) break;
            const unsigned i = base + lane;
            if (i < nf) {
                const uint32_t pos = d.pairs.fb[i].x;
                uint4 a, b;
                load_lean(d.pairs, static_cast<int>(pos), a, b);
                const int32_t gi[3] = {static_cast<int32_t>(a.x), static_cast<int32_t>(a.y),
                                       static_cast<int32_t>(a.z)};
                const int32_t go[3] = {static_cast<int32_t>(a.w), static_cast<int32_t>(b.x),
                                       static_cast<int32_t>(b.z)};
                GlobalVisit v;
                v.vol = (b.w & 1u) == 0 ? N : M;
                walk_tile_global(d.tp, gi, go, static_cast<int>(b.w >> 1), v);
            }
        }
    }
}

}  // namespace

// Persistent traversal: blocks take jobs (one tile's range of pairs) from
// the job counter until none is left, walk them into their shared-memory
// tile and flush it; then they walk the fallback lists.  max_words is the
// largest tile of the scans (the dynamic shared memory of the launch).
template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1) trace_tiles_kernel(
    const ScanDesc *__restrict__ descs, int nscans, int *job_counter, int max_words)
{
    extern __shared__ uint32_t tile[];
    __shared__ int s_job, s_scan;
    __shared__ unsigned s_next;
    __shared__ int s_prefix[kMaxBatch + 1];
    const unsigned lane = threadIdx.x & 31u;
    // jobs of scan k are the global job numbers [s_prefix[k], s_prefix[k+1])
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < nscans; ++k) {
            s_prefix[k] = acc;
            acc += descs[k].ctrl->njobs;
        }
        s_prefix[nscans] = acc;
    }
    // each flush clears its box: the tile starts cleared once
    for (int w = threadIdx.x; w < max_words; w += blockDim.x) tile[w] = 0u;
    __syncthreads();
    const int total_jobs = s_prefix[nscans];
    for (;;) {
        if (threadIdx.x == 0) {
            const int J = atomicAdd(job_counter, 1);
            int k = 0;
            while (k + 1 < nscans && s_prefix[k + 1] <= J) ++k;
            s_job = J;
            s_scan = k;
            s_next = 0;
        }
        __syncthreads();
        if (s_job >= total_jobs) break;
        const ScanDesc &d = descs[s_scan];
        const TilePlan tp = d.tp;
        const TileJob job = d.jobs[s_job - s_prefix[s_scan]];
        const int tix = job.tile % tp.ntx;
        const int tiy = (job.tile / tp.ntx) % tp.nty;
        const int tiz = job.tile / (tp.ntx * tp.nty);
        const int x0 = tix * tp.tx, y0 = tiy * tp.ty, z0 = tiz * tp.tz;
        const int dx = min(tp.tx, tp.nx - x0), dy = min(tp.ty, tp.ny - y0),
                  dz = min(tp.tz, tp.nz - z0);
        unsigned runs = 0;
        walk_job(tile, dx, dy, dz, d.pairs, job.start,
                 job.end - job.start, tp.refill, &s_next, runs);
        __syncthreads();
        flush_tile(tile, dx, dy, dz, job.cls == 0 ? d.N : d.M, tp.nx, tp.ny, x0, y0, z0);
        // runs walked by this job, added to its scan's counter
        unsigned long long ru = runs;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ru += __shfl_xor_sync(kFull, ru, o);
        if (lane == 0 && ru) atomicAdd(&d.ctrl->runs, ru);
        __syncthreads();
    }
    walk_fallback_lists(descs, nscans);
}

template <int kThreads>
int occupancy_of(int smem_words)
{
    // allow the largest tile once, so launches (also inside graph capture)
    // need no attribute change
    if (cudaFuncSetAttribute(trace_tiles_kernel<kThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemBytes) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_tiles_kernel<kThreads>, kThreads,
                                                      static_cast<size_t>(smem_words) * 4) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

int trace_tiles_occupancy(int smem_words, int threads)
{
    switch (threads) {
    case 256: return occupancy_of<256>(smem_words);
    case 512: return occupancy_of<512>(smem_words);
    case 768: return occupancy_of<768>(smem_words);
    case 1024: return occupancy_of<1024>(smem_words);
    default: return 0;
    }
}

cudaError_t launch_trace_tiles(const ScanDesc *descs, int nscans, int *job_counter,
                               int smem_words, int threads, int grid, cudaStream_t s)
{
    if (nscans < 1 || nscans > kMaxBatch || smem_words * 4 > kTileSmemBytes)
        return cudaErrorInvalidValue;
    const size_t smem = static_cast<size_t>(smem_words) * 4;
    switch (threads) {
    case 256:
        trace_tiles_kernel<256><<<grid, 256, smem, s>>>(descs, nscans, job_counter, smem_words);
        break;
    case 512:
        trace_tiles_kernel<512><<<grid, 512, smem, s>>>(descs, nscans, job_counter, smem_words);
        break;
    case 768:
        trace_tiles_kernel<768><<<grid, 768, smem, s>>>(descs, nscans, job_counter, smem_words);
        break;
    case 1024:
        trace_tiles_kernel<1024><<<grid, 1024, smem, s>>>(descs, nscans, job_counter, smem_words);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hd
