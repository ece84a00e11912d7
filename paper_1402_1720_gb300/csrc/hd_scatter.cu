// Bucketing of the (record, tile) pairs of a chunk for the tiled traversal,
// after ingest has counted, per ingest block, its pairs in each tile:
//   bases    per tile, exclusive scan over the blocks -> each block's offset
//   plan     exclusive scan of the tile totals -> tile offsets, job table
//   scatter  counting sort of the pairs by tile: block b of the ingest split
//            writes its pairs from its offsets, with each pair's walk set-up
#include <cooperative_groups.h>
#include "hd_fallback.cuh"

namespace cg = cooperative_groups;

namespace hd {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScatterThreads = 512;

__device__ __forceinline__ unsigned warp_incl_scan_u(unsigned v)
{
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, v, o);
        if (lane >= static_cast<unsigned>(o)) v += t;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x <= 1024).
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *s_warp, unsigned &total)
{
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned nw = blockDim.x >> 5;
    const unsigned incl = warp_incl_scan_u(v);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const unsigned x = lane < nw ? s_warp[lane] : 0u;
        const unsigned xi = warp_incl_scan_u(x);
        if (lane < nw) s_warp[lane] = xi - x;
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    const unsigned r = s_warp[wid] + incl - v;
    total = s_warp[32];
    __syncthreads();
    return r;
}


// One warp per tile-class column: the exclusive prefix over the ingest
// blocks of their pair counts (in place) and the column's total.
__global__ void __launch_bounds__(256) bases_kernel(int ncols, int nblocks, uint32_t *counts,
                                                    uint32_t *totals)
{
    const int c = static_cast<int>(blockIdx.x) * 8 + static_cast<int>(threadIdx.x >> 5);
    const int lane = static_cast<int>(threadIdx.x & 31u);
    if (c >= ncols) return;  // the whole warp
    uint32_t *col = counts + static_cast<size_t>(c) * nblocks;
    unsigned run = 0;
    for (int b0 = 0; b0 < nblocks; b0 += 32) {
        const int b = b0 + lane;
        const unsigned v = b < nblocks ? col[b] : 0u;
        const unsigned incl = warp_incl_scan_u(v);
        if (b < nblocks) col[b] = run + incl - v;
        run += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) totals[c] = run;
}

// One block: tile offsets (exclusive scan of the counts), cursors for the
// scatter, and the job table (chunks of one tile's pairs).  The job size
// adapts to the amount of work: at most tp.job_size pairs, and small enough
// that there are about three jobs per SM (not below kMinJob, so a job's
// flush stays small against its walks; two or four per SM, or a smaller
// floor, measured slower).
__global__ void __launch_bounds__(1024) plan_kernel(TilePlan tp, const uint32_t *tile_count,
                                                    uint32_t *tile_cursor, TileJob *jobs,
                                                    Ctrl *ctrl, int sm_count)
{
    __shared__ unsigned s_warp[33];
    __shared__ unsigned s_js;
    const int nt = 2 * tp.ntiles;
    const int per = (nt + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per;
    unsigned my_pairs = 0;
    for (int t = t0; t < t0 + per && t < nt; ++t) my_pairs += tile_count[t];
    unsigned tot_pairs;
    unsigned off = block_excl_scan(my_pairs, s_warp, tot_pairs);
    if (threadIdx.x == 0) {
        const unsigned want = (tot_pairs + 3u * sm_count - 1u) / (3u * sm_count);
        unsigned js = want < static_cast<unsigned>(tp.job_size) ? want : tp.job_size;
        if (js < static_cast<unsigned>(kMinJob)) js = kMinJob;
        if (js > static_cast<unsigned>(tp.job_size)) js = tp.job_size;
        s_js = js;
    }
    __syncthreads();
    const unsigned js = s_js;
    unsigned my_jobs = 0;
    for (int t = t0; t < t0 + per && t < nt; ++t) my_jobs += (tile_count[t] + js - 1) / js;
    unsigned tot_jobs;
    unsigned joff = block_excl_scan(my_jobs, s_warp, tot_jobs);
    for (int t = t0; t < t0 + per && t < nt; ++t) {
        const unsigned c = tile_count[t];
        tile_cursor[t] = off;
        for (unsigned s = 0; s < c; s += js) {
            TileJob j;
            j.tile = t % tp.ntiles;
            j.cls = t / tp.ntiles;
            j.start = static_cast<int>(off + s);
            j.end = static_cast<int>(off + (s + js < c ? s + js : c));
            jobs[joff++] = j;
        }
        off += c;
    }
    if (threadIdx.x == 0) {
        ctrl->njobs = static_cast<int>(tot_jobs);
        ctrl->job_next = 0;
    }
}

// The general set-up of one (record, tile) pair: its packed lean walk, an
// empty walk, or (returns true) the general form for the fallback list.
__device__ __noinline__ bool general_setup(const int32_t gi[3], const int32_t go[3], int dx,
                                           int dy, int dz, int tile, int cls, uint4 &p0,
                                           uint4 &p1)
{
    RunWalk w;
    LeanWalk L;
    uint32_t pk[kLeanWords];
    bool fallback = false;
    if (!run_begin(w, gi, go, dx, dy, dz)) {
        lean_pack_empty(pk);
    } else if (lean_of(w, L)) {
        lean_pack(L, pk);
    } else {
        // walked from the fallback list by the general run walk
        general_pack(gi, go, tile, cls, pk);
        fallback = true;
    }
    p0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    p1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    return fallback;
}

// Counting sort of (record, tile) pairs by tile.  Block b takes the pairs
// ingest block b listed, one per thread, and writes those of tile c from
// tile_start[c] + block_base[c * blocks + b] on (a shared-memory cursor per
// tile orders them within the block).
__global__ void __launch_bounds__(kScatterThreads, 2) scatter_kernel(
    TilePlan tp, Records rec, int64_t per_block, const uint32_t *tile_start,
    const uint32_t *block_base, const uint32_t *block_pairs, Ctrl *ctrl, Pairs pairs)
{
    extern __shared__ uint32_t s_mem[];
    const int nt = 2 * tp.ntiles;
    uint32_t *s_base = s_mem;       // this block's first position in each tile
    uint32_t *s_next = s_mem + nt;  // pairs written per tile so far
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        s_base[t] = tile_start[t] + block_base[static_cast<size_t>(t) * gridDim.x + blockIdx.x];
        s_next[t] = 0;
    }
    __syncthreads();
    const int64_t h0 = static_cast<int64_t>(blockIdx.x) * per_block;
    const unsigned npairs = block_pairs[blockIdx.x];
    const uint32_t *list = pairs.stage + static_cast<int64_t>(blockIdx.x) * per_block * tp.pairs_per_record;
    for (unsigned e = threadIdx.x; e < npairs; e += kScatterThreads) {
        const uint32_t code = list[e];
        const int64_t slot = h0 + (code >> kRecordTileBits);
        const int j = static_cast<int>(code & (kMaxRecordTiles - 1u));
        const int32_t stw = rec.status[slot];
        const int cls = status_cls(stw);
        int32_t q[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) q[a] = rec.g[a][slot];
        // the j-th tile of the record's box, x fastest; with whole-plane
        // tiles the box is the record's slices alone (in its status word)
        int x = 0, y = 0, z;
        if (tp.ntx == 1 && tp.nty == 1) {
            const unsigned zl = static_cast<unsigned>(status_zlo(stw));
            z = (tp.mtz ? static_cast<int>(umulhi32(zl, tp.mtz)) : static_cast<int>(zl)) + j;
        } else {
            int lo[3], hi[3];
            tile_range_z(tp, q, status_zlo(stw), status_zhi(stw), lo, hi);
            const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1;
            x = lo[0] + j % ex;
            y = lo[1] + (j / ex) % ey;
            z = lo[2] + j / (ex * ey);
        }
        const int t = cls * tp.ntiles + x + tp.ntx * (y + tp.nty * z);
        const uint32_t pos = s_base[t] + atomicAdd(&s_next[t], 1u);
        // set up the walk of this record clipped to this tile
        const int x0 = x * tp.tx, y0 = y * tp.ty, z0 = z * tp.tz;
        const int dx = min(tp.tx, tp.nx - x0), dy = min(tp.ty, tp.ny - y0),
                  dz = min(tp.tz, tp.nz - z0);
        const int32_t gi[3] = {q[0] - (x0 << 16), q[1] - (y0 << 16), q[2] - (z0 << 16)};
        const int32_t go[3] = {q[3] - (x0 << 16), q[4] - (y0 << 16), q[5] - (z0 << 16)};
        // one-slice tiles (the default plan): the direct set-up; the
        // walks it declines (ties at the start, no in-plane motion) go to
        // the fallback list, whose general run walk is exact for any walk.
        // Deeper slabs: the general set-up (out of line).
        uint4 p0, p1;
        bool fallback = false;
        if (dz == 1) {
            LeanWalk L;
            const int rl = slab_lean(gi, go, dx, dy, L);
            uint32_t pk[kLeanWords];
            if (rl == 1) {
                lean_pack(L, pk);
            } else if (rl == 0) {
                lean_pack_empty(pk);
            } else {
                general_pack(gi, go, t - cls * tp.ntiles, cls, pk);
                fallback = true;
            }
            p0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            p1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        } else {
            fallback = general_setup(gi, go, dx, dy, dz, t - cls * tp.ntiles, cls, p0, p1);
        }
        pairs.v[2 * static_cast<size_t>(pos)] = p0;
        pairs.v[2 * static_cast<size_t>(pos) + 1] = p1;
        if (fallback) {
            // append to the fallback list, one counter update per group of
            // lanes arriving together
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned at = 0;
            if (grp.thread_rank() == 0) {
                at = atomicAdd(&ctrl->n_pair_fallback, grp.size());
                atomicAdd(&ctrl->pairs_general, static_cast<unsigned long long>(grp.size()));
            }
            at = grp.shfl(at, 0) + grp.thread_rank();
            pairs.fb[at] = make_uint2(pos, 0u);
        }
    }
}

}  // namespace

cudaError_t launch_plan(const TilePlan &tp, int64_t n, uint32_t *block_count,
                        uint32_t *tile_count, uint32_t *tile_cursor, TileJob *jobs, Ctrl *ctrl,
                        int sm_count, cudaStream_t s)
{
    const int ncols = 2 * tp.ntiles;
    const ChunkSplit sp = chunk_split(n, sm_count);
    bases_kernel<<<static_cast<unsigned>((ncols + 7) / 8), 256, 0, s>>>(ncols, sp.blocks,
                                                                        block_count, tile_count);
    plan_kernel<<<1, 1024, 0, s>>>(tp, tile_count, tile_cursor, jobs, ctrl,
                                   sm_count > 0 ? sm_count : 1);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const TilePlan &tp, const Records &rec, int64_t n, Ctrl *ctrl,
                           const uint32_t *tile_cursor, const uint32_t *block_count,
                           const uint32_t *block_pairs, const Pairs &pairs, int sm_count,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const ChunkSplit sp = chunk_split(n, sm_count);
    const size_t smem = sizeof(uint32_t) * 4 * static_cast<size_t>(tp.ntiles);
    scatter_kernel<<<static_cast<unsigned>(sp.blocks), kScatterThreads, smem, s>>>(
        tp, rec, sp.per_block, tile_cursor, block_count, block_pairs, ctrl, pairs);
    return cudaGetLastError();
}

}  // namespace hd
