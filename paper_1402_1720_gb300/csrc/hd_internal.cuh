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
constexpr int kTileSmemBytes = 200 * 1024;  // shared memory per block for a private tile

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

// Device-side counters of one scan.  The block from rec_miss to job_next is
// cleared before every chunk of histories.
struct Ctrl {
    unsigned long long n_in, n_miss, n_hit, n_none, n_reject;
    unsigned long long steps_miss, steps_hit;
    unsigned long long pairs_general;  // pairs sent to the fallback list (cumulative)
    unsigned long long runs;           // runs walked by the tiled pass (cumulative)
    unsigned int rec_miss;    // records appended from the front of the list
    unsigned int rec_hit;     // records appended from the back of the list
    unsigned int pairs_used;  // (record, tile) pairs admitted to the tiled path
    int njobs;                // jobs of the tiled traversal
    int job_next;             // next job to hand out
    unsigned int n_fallback;  // records traversed by the global-memory path
    unsigned int n_pair_fallback;  // entries of the pair fallback list
    unsigned int fb_next;          // next fallback entry to hand out
};

// Compacted traversal records: grid Q16 entry and exit points, int32 each
// (|G| < 2^30), and a status (1 tiled, 2 global path).  Missed histories
// fill [0, rec_miss), hit ones [cap - rec_hit, cap).  Structure of arrays.
struct Records {
    int32_t *g[6];  // x0, y0, z0, x1, y1, z1
    int32_t *status;
    int64_t cap;
};

// Tiling of the grid into boxes whose counters fit in shared memory.
struct TilePlan {
    int nx, ny, nz;
    int tx, ty, tz;     // tile size in voxels
    int ntx, nty, ntz;  // tiles per axis
    int ntiles;         // tiles per class (0: tiled path off)
    int max_tiles;      // records touching more tiles take the global path
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
};

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
constexpr int kMinJob = 2048;  // smallest job the plan makes (pairs), unless the tuning is lower

struct Inputs {
    const float *angle, *u_in, *v_in, *u_out, *v_out, *wepl;
};

// ---- launchers (stream-ordered; return the launch's cudaError_t) ----
cudaError_t launch_ingest(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cordic,
                          float tau_l, float tau_h, int use_miss, int use_hit, const TilePlan &tp,
                          const Records &rec, Ctrl *ctrl, uint32_t *tile_count, int sm_count,
                          cudaStream_t s);

cudaError_t launch_plan(const TilePlan &tp, const uint32_t *tile_count, uint32_t *tile_cursor,
                        TileJob *jobs, Ctrl *ctrl, int sm_count, cudaStream_t s);

cudaError_t launch_scatter(const TilePlan &tp, const Records &rec, Ctrl *ctrl,
                           uint32_t *tile_cursor, const Pairs &pairs, int64_t n, int sm_count,
                           cudaStream_t s);

// Persistent traversal over the jobs of nscans scans (descs on the device),
// handed out through *job_counter (zero before the launch).  smem_words is
// the largest tile of the scans; threads is 256, 512, 768 or 1024.
cudaError_t launch_trace_tiles(const ScanDesc *descs, int nscans, int *job_counter,
                               int smem_words, int threads, int grid, cudaStream_t s);

// Global-memory traversal of the records whose status is 2 (or of every
// record when all_records is set).
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
