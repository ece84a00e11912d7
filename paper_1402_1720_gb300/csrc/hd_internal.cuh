// Internal definitions shared by the CUDA translation units of libhulld.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hulld.h"

namespace hd {

constexpr int64_t kQ16 = 65536;
constexpr int kMaxN = 4096;
constexpr int kMaxTiles = 2048;       // tiles per class for the shared-memory path
constexpr int kTraceThreads = 512;    // threads per block of the tiled traversal
constexpr int kTileSmemBytes = 224 * 1024;  // shared memory per block for a private tile

// Gantry-rotation constants: theta[i] = round(atan(2^-i) * 180/pi * 2^30)
// (degrees, 30 fractional bits) and K = round(2^30 prod (1 + 2^-2i)^-1/2).
struct Cordic {
    long long theta[32];
    long long K;
};

// Geometry in the fixed-point units the kernels use.
struct GeomQ {
    int32_t nx, ny, nz;
    int32_t pad;
    long long sx, sy, sz;  // voxel sizes, mm * 2^16
    long long T;           // tracker half-separation, mm * 2^16
    unsigned long long mx, my, mz;  // floor(2^64 / (2 s)): division by multiply-high
};

// Device-side counters of one scan.  The block from njobs to the end is
// cleared before every chunk of histories.
struct Ctrl {
    unsigned long long n_in, n_miss, n_hit, n_none, n_reject;
    unsigned long long steps_miss, steps_hit;
    unsigned long long pairs_general;  // pairs sent to the fallback list (cumulative)
    unsigned long long runs;           // runs walked by the tiled pass (cumulative)
    int njobs;                // jobs of the tiled traversal
    unsigned int n_global;    // records listed for the global path (Records::glist)
    int job_next;             // next job to hand out
    unsigned int n_fallback;  // records traversed by the global-memory path
    unsigned int n_pair_fallback;  // entries of the pair fallback list
    unsigned int fb_next;          // next fallback entry to hand out
};

// Traversal records of one chunk, one slot per history (slot = the
// history's index in the chunk): grid Q16 entry and exit points, int32 each
// (|G| < 2^30), and a status word (record_status in hd_geom.cuh: path 0 for
// a history without a record, 1 tiled, 2 global; its class; its slices).
// Structure of arrays; each array starts on a 16-byte boundary when the
// chunk's slot count is padded to a multiple of four (records_stride).
struct Records {
    int32_t *g[6];  // x0, y0, z0, x1, y1, z1
    int32_t *status;
    int32_t *glist;  // slots of the global-path records, Ctrl::n_global of them
                     // (null: that path finds them by their status words)
    int64_t cap;     // slots (the chunk's histories)
};

inline int64_t records_stride(int64_t n) { return (n + 3) & ~int64_t(3); }

// How a chunk of n histories is split among the ingest blocks; the scatter
// uses the same split, so that each of its blocks finds the pairs of the
// records one ingest block wrote.  Block b takes histories
// [b per_block, min((b + 1) per_block, n)); per_block is a multiple of 4.
constexpr int kIngestThreads = 256;
constexpr int kIngestBlocksPerSm = 8;
struct ChunkSplit {
    int blocks;
    int64_t per_block;
};
inline ChunkSplit chunk_split(int64_t n, int sm_count)
{
    const int64_t units = (n + 3) / 4;  // groups of four histories
    int64_t blocks = (units + kIngestThreads - 1) / kIngestThreads;
    const int64_t cap = static_cast<int64_t>(sm_count > 0 ? sm_count : 1) * kIngestBlocksPerSm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    ChunkSplit c;
    c.per_block = 4 * ((units + blocks - 1) / blocks);
    c.blocks = static_cast<int>((n + c.per_block - 1) / c.per_block);
    if (c.blocks < 1) c.blocks = 1;
    return c;
}

// Tiling of the grid into boxes whose counters fit in shared memory.
struct TilePlan {
    int nx, ny, nz;
    int tx, ty, tz;     // tile size in voxels
    int ntx, nty, ntz;  // tiles per axis
    int ntiles;         // tiles per class (0: tiled path off)
    int max_tiles;      // records touching more tiles take the global path
    int pairs_per_record;  // pair budget per history (pair_cap = this * slots)
    int job_size;       // pairs per job
    long long pair_cap;
    int tile_words;     // 32-bit words of shared memory per block
    int refill;         // idle lanes that trigger a warp refill
    int threads;        // threads per block of the traversal (256, 512, 768, 1024)
    unsigned mtx, mty, mtz;  // floor(2^32 / t) + 1 (0 when t = 1): division by a tile size
};

// (record, tile) pairs sorted by tile: the packed lean walk of the record
// clipped to the tile, 32 bytes per pair (two uint4: one 32-byte sector;
// class and tile come from the job).  A pair whose walk has no lean form
// (a tie, a pending start, or a z crossing inside the tile) holds instead
// its tile-local endpoints, tile and class, marked empty for the lean pass,
// and its position goes to the fallback list; traversal blocks that run out
// of jobs walk those with the general run walk in global memory.
struct Pairs {
    uint4 *v;   // 2 per pair
    uint2 *fb;  // fallback list: (pair position, 0), pair_cap entries
    // Each ingest block's pairs in the order its budget assigned them, from
    // the block's share (block * per_block * pairs_per_record) on: the
    // record's slot less the block's first slot, times kMaxRecordTiles,
    // plus the pair's tile index within the record.
    uint32_t *stage;
};

// Tiles a record may touch on the tiled path (its box of tiles; more take
// the global path), and the bits of a tile index within a record.
constexpr int kMaxRecordTiles = 32;
constexpr int kRecordTileBits = 5;
static_assert(kMaxRecordTiles == 1 << kRecordTileBits, "tile index bits");

struct TileJob {
    int tile;   // tile id within its class
    int cls;    // 0 missed (N), 1 hit (M)
    int start;  // pair range [start, end)
    int end;
};

// Everything the traversal kernel needs about one scan; a batch passes a
// table of these and one job counter for all of them.
struct ScanDesc {
    TilePlan tp;
    Pairs pairs;
    const TileJob *jobs;
    Ctrl *ctrl;  // njobs of the scan (read) and its step counters (added to)
    uint32_t *N, *M;
};

constexpr int kMaxBatch = 64;  // scans per batched traversal launch
constexpr int kMinJob = 8192;  // smallest job the plan makes (pairs), unless the tuning is lower

struct Inputs {
    const float *angle, *u_in, *v_in, *u_out, *v_out, *wepl;
};

// ---- launchers (stream-ordered; return the launch's cudaError_t) ----

// Classification, records and pair counts of a chunk.  block_count (null
// when tp.ntiles is 0) receives, per tile-class column c (2 tp.ntiles of
// them) and ingest block b, the pairs of that block's records in that tile
// at [c * blocks + b]; block_pairs[b] the block's pairs in all, listed in
// stage (Pairs::stage).  Each block keeps to a pair budget of
// tp.pairs_per_record per history; its records beyond it take the global
// path.  on_host: the inputs are page-locked host memory read in place.
cudaError_t launch_ingest(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cordic,
                          float tau_l, float tau_h, int use_miss, int use_hit, const TilePlan &tp,
                          const Records &rec, Ctrl *ctrl, uint32_t *block_count,
                          uint32_t *block_pairs, uint32_t *stage, int on_host, int sm_count,
                          cudaStream_t s);

// Per column: the exclusive prefix over blocks of block_count (in place) and
// the column total into tile_count; then the plan (tile offsets into
// tile_cursor, the job table).
cudaError_t launch_plan(const TilePlan &tp, int64_t n, uint32_t *block_count,
                        uint32_t *tile_count, uint32_t *tile_cursor, TileJob *jobs, Ctrl *ctrl,
                        int sm_count, cudaStream_t s);

// Counting sort of the (record, tile) pairs by tile, with the walk set-up of
// each pair; block b of the chunk split takes the block_pairs[b] pairs that
// ingest block b listed and writes those of tile c from
// tile_cursor[c] + block_count[c * blocks + b] on.
cudaError_t launch_scatter(const TilePlan &tp, const Records &rec, int64_t n, Ctrl *ctrl,
                           const uint32_t *tile_cursor, const uint32_t *block_count,
                           const uint32_t *block_pairs, const Pairs &pairs, int sm_count,
                           cudaStream_t s);

// Persistent traversal over the jobs of nscans scans (descs on the device),
// handed out through *job_counter (zero before the launch).  smem_words is
// the largest tile of the scans; threads is 256, 512, 768 or 1024.
cudaError_t launch_trace_tiles(const ScanDesc *descs, int nscans, int *job_counter,
                               int smem_words, int threads, int grid, cudaStream_t s);

// Global-memory traversal of the records whose path is 2 (or of every
// record when all_records is set); upper is the chunk's slot count.
cudaError_t launch_trace_global(const Records &rec, Ctrl *ctrl, int64_t upper, const GeomQ &g,
                                uint32_t *N, uint32_t *M, int all_records,
                                int sm_count, cudaStream_t s);

cudaError_t launch_classify(const float *wepl, int64_t n, float tau_l, float tau_h,
                            uint8_t *cls, cudaStream_t s);

// Blocks per SM the tiled traversal can keep resident with this much shared
// memory per block and this many threads (0 when the launch is impossible).
int trace_tiles_occupancy(int smem_words, int threads);

struct DecideArgs {
    int32_t nx, ny, nz;
    int32_t methods;
    int32_t nt, nbhd, sm_ge, sm_per_slice;
    const uint32_t *N;       // null when neither SC nor MSC is on
    const uint32_t *M;       // null when SM is off
    unsigned long long *slice_key;  // nz entries (SM)
    uint32_t *mt, *slope;    // nz entries (SM)
    long long *index;        // nz entries (SM)
    uint8_t *H1, *H2, *H3;
};

cudaError_t launch_finalize(const DecideArgs &a, int sm_count, cudaStream_t s);

// sum_v N(v) and sum_v M(v) (each 0 when its volume is null) into out[0],
// out[1]: by Eq. 3.4 and 3.9 these are the sums of |A_i| over the missed and
// the hit histories, the voxel memberships the statistics report.
cudaError_t launch_volume_sums(const uint32_t *N, const uint32_t *M, int64_t V,
                               unsigned long long *out, int sm_count, cudaStream_t s);

cudaError_t launch_pack_bits(const uint8_t *mask, int64_t V, uint32_t *bits, cudaStream_t s);

// Compaction: writes ascending indices of mask != 0 to out (if count fits
// capacity) and the total to *d_count.  `block_counts` holds
// ceil(V / 1024) + 1 uint32 of scratch.
cudaError_t launch_compact(const uint8_t *mask, int64_t V, int32_t *out, int64_t capacity,
                           uint32_t *block_counts, unsigned long long *d_count, cudaStream_t s);

// Shared host helpers of the C ABI (defined with the scan objects).
bool make_cordic_table(Cordic &c);
void note_cuda_error(cudaError_t e, const char *where);
hd_status check_geometry(const hd_geometry *g);

}  // namespace hd
