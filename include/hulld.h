/*
 * hulld.h -- C ABI of the GB300 hull-detection library for proton CT.
 *
 * The library computes the three hull-detection methods of Schultze et al.,
 * "Performance of Hull-Detection Algorithms for Proton Computed Tomography
 * Reconstruction" (arXiv 1402.1720):
 *   SC  (silhouette/space carving, Sec. 3.2, Eq. 3.1-3.3, Alg. 1),
 *   MSC (modified space carving,   Sec. 3.3, Eq. 3.4-3.6, Alg. 2),
 *   SM  (space modeling,           Sec. 3.4, Eq. 3.7-3.10, Alg. 3),
 * from proton histories given as gantry angle, entry/exit tracker
 * coordinates and WEPL (Sec. 2.1-2.2).  All compute runs in CUDA kernels for
 * sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every call
 * --------------------------------
 * Geometry.  World frame in mm, origin at the centre of the reconstruction
 * volume, z the vertical rotation axis (Sec. 2.2).  At gantry angle phi
 * (degrees) the beam runs along b = (cos phi, sin phi, 0), the lateral
 * tracker axis is e_u = (-sin phi, cos phi, 0), the vertical one e_v = z.
 * Entry point = -T b + u_in e_u + v_in e_v, exit point = +T b + u_out e_u +
 * v_out e_v, with T the tracker half-separation.  The path L_i is the closed
 * straight segment between them (Sec. 2.1; the definition of L_i before
 * Eq. 3.2).
 *
 * Voxels.  nx*ny*nz voxels of sx*sy*sz mm centred on the origin; linear index
 * x + nx*(y + ny*z) (x fastest).  A_i (Eq. 3.2, read with d_0 = 0) is the set
 * of voxels whose half-open cube [k, k+1)^3 in voxel units contains a point
 * of L_i.  Coordinates are made exact by rounding each float32 input to 16
 * fractional bits (ties to even), an integer CORDIC rotation (Q30 cos/sin)
 * and integer floor divisions; everything after that is exact integer
 * arithmetic, so counts and masks are bit-reproducible.
 *
 * Classification (Eq. 3.1, Eq. 3.7; cutoffs of Sec. 3.2-3.4): a history is
 * missed when wepl < wepl_miss_lt, hit when wepl > wepl_hit_gt, otherwise
 * unused (NaN included).  No angular cutoff is applied (the paper used none).
 *
 * Rejection.  A missed or hit history whose angle is not finite or has
 * |angle| >= 2^20 degrees, whose u/v coordinates are not finite or have
 * magnitude >= 4096 mm, or whose grid coordinates reach magnitude >= 2^30 /
 * 2^16 = 16384 voxels, is not traversed and is counted in n_reject.
 * Histories are never silently clipped.
 *
 * Streams and memory.  `stream` arguments are cudaStream_t values passed as
 * void* (NULL = the legacy default stream).  Work is stream-ordered; the
 * caller keeps input buffers valid until the stream has passed the call.
 * All calls on one scan must be ordered by the caller (one stream, or
 * events between streams).  Pointers flagged `on_device` are device
 * pointers on the scan's device; otherwise they are host pointers (pinned
 * memory gives asynchronous copies).  The caller owns every buffer it
 * passes; the library owns the scan state and frees it in hd_scan_destroy.
 *
 * Errors.  Every call returns hd_status and never throws.  A CUDA error is
 * returned as HD_ERR_CUDA from the call that observed it.
 */
#ifndef HULLD_H
#define HULLD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HD_API __attribute__((visibility("default")))
#else
#define HD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HD_OK = 0,
    HD_ERR_ARG = 1,       /* null pointer, bad enum, bad size or layout */
    HD_ERR_RANGE = 2,     /* geometry or parameter outside supported range */
    HD_ERR_NOMEM = 3,     /* device or host allocation failed */
    HD_ERR_CUDA = 4,      /* a CUDA runtime call failed */
    HD_ERR_STATE = 5,     /* call not valid in the object's current state */
    HD_ERR_TIMEOUT = 6,   /* a bounded wait gave up */
    HD_ERR_ADMISSION = 7, /* serving: request exceeds the memory budget */
    HD_ERR_OVERFLOW = 8   /* a scan reached 2^32 - 1 histories (uint32 counts) */
} hd_status;

/* Methods (bit mask). */
enum { HD_SC = 1, HD_MSC = 2, HD_SM = 4 };

/* Mask layouts for hd_scan_get_mask. */
enum {
    HD_MASK_U8 = 0,  /* one byte per voxel, 0 or 1, linear voxel order */
    HD_MASK_BITS = 1 /* ceil(V/32) uint32 words, voxel v at bit (v & 31) of word v >> 5 */
};

/* Reconstruction grid.  Supported: 1 <= n <= 4096 per axis, V < 2^31,
 * voxel sizes in [1/64, 64] mm, n * s <= 8192 mm per axis,
 * 0 < tracker_half_sep_mm < 4096. */
typedef struct {
    int32_t nx, ny, nz;
    float sx, sy, sz;          /* voxel size, mm */
    float tracker_half_sep_mm; /* T: trackers at -T and +T along the beam */
} hd_geometry;

/* Method parameters.  hd_params_default gives the paper's values. */
typedef struct {
    float wepl_miss_lt;    /* missed if WEPL < this (1.0 mm, Sec. 3.2/3.3) */
    float wepl_hit_gt;     /* hit if WEPL > this (5.0 mm, Sec. 3.4) */
    int32_t msc_nt;        /* MSC threshold N_t (50, Sec. 3.3) */
    int32_t msc_nbhd;      /* B(v) of Eq. 3.5: 6 = face neighbours, 4 = in-plane only */
    int32_t sm_ge;         /* H_3 = [M >= M_t] (1, text of Sec. 3.4) or [M > M_t] (0, Eq. 3.10) */
    int32_t sm_per_slice;  /* M_t per slice (1, Sec. 3.4) or over the whole volume (0, Alg. 3) */
    uint32_t methods;      /* bit mask of HD_SC | HD_MSC | HD_SM */
} hd_params;

/* Per-scan counters (cumulative since create/reset). */
typedef struct {
    int64_t n_in;       /* histories received */
    int64_t n_miss;     /* classified missed (Eq. 3.1) */
    int64_t n_hit;      /* classified hit (Eq. 3.7) */
    int64_t n_none;     /* neither */
    int64_t n_reject;   /* missed/hit histories with unusable geometry (not traversed) */
    int64_t steps_miss; /* sum of |A_i| over traversed missed histories */
    int64_t steps_hit;  /* sum of |A_i| over traversed hit histories */
    int64_t pairs_general; /* (history, tile) pairs of the tiled pass whose walk has a tie
                              or crosses z inside the tile, walked by the general run walk
                              in global memory instead of the closed-form lean walk */
    int64_t runs;          /* major-axis runs walked by the lean walks of the tiled pass
                              (each adds +1 and -1 to a difference array: two
                              shared-memory atomics in count mode) */
} hd_stats;

/* Kernel-level timing of a scan (enabled by hd_scan_set_profiling):
 * CUDA-event time on the scan's stream of each phase, summed over calls,
 * and the number of kernels the library launched (always counted). */
typedef struct {
    int64_t kernel_launches;  /* kernels launched by this scan since create */
    int64_t trace_launches;   /* traversal kernel launches (profiled window) */
    double ms_ingest;         /* classification, geometry, bucketing by tile */
    double ms_trace;          /* voxel traversal and accumulation (shared-memory tiles) */
    double ms_finalize;       /* decisions (H_1, H_2, M_t, H_3) */
    double ms_trace_global;   /* traversal of records outside the tiled path */
} hd_profile;

typedef struct hd_scan hd_scan;

/* Human-readable name of a status code (static storage). */
HD_API const char *hd_status_string(hd_status s);

/* Text of the last CUDA error this thread saw inside the library (the call
 * and cudaGetErrorString), or "" if none.  Thread-local static storage. */
HD_API const char *hd_last_cuda_error(void);

/* Fill *out with the paper's parameters: 1.0 mm, 5.0 mm, N_t = 50 (Sec. 3.3),
 * B6, H_3 with >=, per-slice M_t, all three methods. */
HD_API hd_status hd_params_default(hd_params *out);

/* Create a scan on the current CUDA device: validates geometry and
 * parameters, allocates the count volumes N (Eq. 3.4; also for SC alone,
 * whose hull H_1 = [N = 0] of Eq. 3.3 is the carve of Alg. 1 written as a
 * set difference) and M (Eq. 3.9) and the output masks, and zeroes them on the legacy default stream (synchronised before
 * return).  HD_ERR_RANGE for unsupported geometry, HD_ERR_ARG for bad
 * parameters (including wepl_miss_lt > wepl_hit_gt or a NaN cutoff). */
HD_API hd_status hd_scan_create(const hd_geometry *geom, const hd_params *params, hd_scan **out);

/* Release everything the scan owns.  Synchronises the scan's device first.
 * NULL is accepted. */
HD_API hd_status hd_scan_destroy(hd_scan *scan);

/* Zero the counts and statistics, stream-ordered, so the scan can take a
 * new acquisition. */
HD_API hd_status hd_scan_reset(hd_scan *scan, void *stream);

/* Size the scan's per-chunk scratch (records, tile pairs, job table) for
 * calls of up to n histories now, so that later calls of that size allocate
 * nothing and never synchronise the stream to grow it.  Optional: the
 * scratch otherwise grows on demand.  May synchronise `stream`. */
HD_API hd_status hd_scan_reserve(hd_scan *scan, int64_t n, void *stream);

/* Add n proton histories (structure of arrays, float32, n entries each):
 * classify each (Eq. 3.1, Eq. 3.7), traverse the voxel set A_i of every
 * missed and hit history (Eq. 3.2) and accumulate N (Eq. 3.4, which SC and
 * MSC read) and M (Eq. 3.9).  Counts stay
 * resident on the device, so histories may arrive in any number of calls
 * (streamed per-angle chunks, Sec. 4 online mode) in any order; the result
 * depends only on the multiset of histories.  on_device = 0 takes host
 * arrays: page-locked arrays mapped into the device's address space (as
 * cudaHostAlloc gives) are read in place by the first kernel over the host
 * link; other host memory is copied to a device staging buffer inside the
 * call.  Either way the arrays must stay unchanged until the work this call
 * queued on `stream` has completed.  n = 0 is a no-op.
 * HD_ERR_OVERFLOW if the scan would exceed 2^32 - 1 histories. */
HD_API hd_status hd_scan_add_histories(hd_scan *scan, const float *angle_deg, const float *u_in,
                                const float *v_in, const float *u_out, const float *v_out,
                                const float *wepl, int64_t n, int32_t on_device,
                                void *stream);

/* Compute the hulls from the resident counts, stream-ordered:
 *   H_1 = V minus the union of missed paths = {v : N(v) = 0} (Eq. 3.3),
 *   H_2 = {v : max_{w in B(v)} N(v) - N(w) < N_t} (Eq. 3.6),
 *   H_3 = {v : M(v) >= M_t(z)} (or >), M_t(z) = M(v*) where v* is the last
 *         voxel (x-fastest order) reaching the steepest drop
 *         max_{w in B(v)} M(v) - M(w) of its slice (Alg. 3 per slice); a
 *         slice whose steepest drop is 0 has no edge and H_3 = 0 there.
 * Only the requested methods are computed.  May be called again after more
 * histories arrive. */
HD_API hd_status hd_scan_finalize(hd_scan *scan, void *stream);

/* Copy a finalized mask (method = one of HD_SC, HD_MSC, HD_SM) into dst in
 * the given layout.  dst_bytes must be at least V (HD_MASK_U8) or
 * 4*ceil(V/32) (HD_MASK_BITS).  For HD_MASK_BITS, bits past V are 0.
 * HD_ERR_STATE if the method was not requested or finalize has not run. */
HD_API hd_status hd_scan_get_mask(hd_scan *scan, int32_t method, int32_t layout, void *dst,
                           size_t dst_bytes, int32_t dst_on_device, void *stream);

/* Copy the count volume of a method into dst (n >= V uint32):
 * HD_MSC or HD_SC -> N (missed paths per voxel, Eq. 3.4; the scan must have
 * SC or MSC), HD_SM -> M (hit paths per voxel, Eq. 3.9).  HD_ERR_STATE when
 * the scan does not hold that volume. */
HD_API hd_status hd_scan_get_counts(hd_scan *scan, int32_t method, uint32_t *dst, int64_t n,
                             int32_t dst_on_device, void *stream);

/* Replace a count volume with src (exactly V uint32, host or device):
 * HD_MSC or HD_SC -> N, HD_SM -> M, as hd_scan_get_counts names them.  For a
 * scan whose histories were split over several processes or GPUs (each
 * accumulating its share, Eq. 3.4 and 3.9 being sums over histories): load
 * the element-wise sum of the shares' counts, then hd_scan_finalize decides
 * the hulls of the whole acquisition.  The statistics' voxel memberships
 * follow the loaded counts; the history counts stay this scan's own.
 * Stream-ordered; src must stay valid until the copy has run.  HD_ERR_STATE
 * when the scan does not hold that volume, HD_ERR_ARG when n != V.  A
 * deployment aid: the paper processes one data set in one place. */
HD_API hd_status hd_scan_set_counts(hd_scan *scan, int32_t method, const uint32_t *src,
                                    int64_t n, int32_t src_on_device, void *stream);

/* Copy the SM thresholds of the last finalize to host arrays of nz entries:
 * M_t per slice, the steepest drop per slice and the linear index of v*.
 * With sm_per_slice = 0 every slice holds the volume's values.  Any of the
 * pointers may be NULL.  Synchronises the stream. */
HD_API hd_status hd_scan_get_thresholds(hd_scan *scan, uint32_t *mt, uint32_t *slope, int64_t *index,
                                 int32_t nz, void *stream);

/* Read the scan's counters (synchronises the stream). */
HD_API hd_status hd_scan_get_stats(hd_scan *scan, hd_stats *out, void *stream);

/* Linear indices, ascending, of the voxels in a finalized hull (the
 * compaction that shrinks the unknown vector x of Sec. 1).  Writes up to
 * `capacity` int32 indices to dst and the hull size to *count (host).
 * Synchronises the stream. */
HD_API hd_status hd_scan_get_hull_indices(hd_scan *scan, int32_t method, int32_t *dst,
                                   int64_t capacity, int64_t *count, int32_t dst_on_device,
                                   void *stream);

/* Launch parameters of the traversal, chosen per volume class by the
 * autotuner (paper_1402_1720_gb300/autotune.py) or left at their defaults:
 *   threads     threads per block of the traversal: 256, 512, 768 or 1024 (1024)
 *   refill      idle lanes of a warp that trigger taking new walks, 1..32 (12)
 *   job_size    (record, tile) pairs per job, 256..32767 (32767)
 *   slab_depth  z-slices per shared-memory tile when whole x-y planes fit,
 *               at most as many as fit; 0 = one slice (0).  Walks that cross
 *               z inside a deeper slab take the general walk in global memory
 * A deployment aid: the paper has no counterpart. */
typedef struct {
    int32_t threads, refill, job_size, slab_depth;
} hd_tuning;

/* Set the scan's traversal parameters.  Only while the scan holds no
 * histories (after create or reset): HD_ERR_STATE otherwise; HD_ERR_ARG for
 * values outside the ranges above. */
HD_API hd_status hd_scan_set_tuning(hd_scan *scan, const hd_tuning *tuning);
HD_API hd_status hd_scan_get_tuning(hd_scan *scan, hd_tuning *out);

/* Thick rays for this scan (Eq. 3.2 with d_0 > 0): every history's A_i is
 * replaced by A_i(k), the voxels within k voxels of A_i in-plane in the same
 * slice (see hd_accumulate_thick), for all three methods; N, M, the hulls,
 * thresholds and statistics follow from the thick sets (the statistics'
 * voxel counts are the thick sets' sizes; runs and pairs_general stay 0).
 * k = 0 restores the thin paths.  Only before any histories (after create or
 * reset): HD_ERR_STATE otherwise; HD_ERR_RANGE for k outside [0, 16].
 * Allocates the thick rays' difference arrays (about 16 bytes
 * per voxel).  When the scan's tiles are whole one-slice planes (the
 * default plan whenever a slice fits the shared-memory budget) the thick
 * sets are counted in the tiled traversal; otherwise each history is walked
 * over the whole grid as in hd_accumulate_thick.  Thick scans cannot join a
 * batch (hd_batch_add_item returns HD_ERR_STATE). */
HD_API hd_status hd_scan_set_thick(hd_scan *scan, int32_t k);

/* Start (enable = 1) or stop (0) recording CUDA events around the scan's
 * kernels; starting also clears the accumulated times.  A library aid for
 * measurement: no counterpart in the paper. */
HD_API hd_status hd_scan_set_profiling(hd_scan *scan, int32_t enable);

/* Accumulated phase times and launch counts.  Waits for the recorded events
 * (host synchronisation on them). */
HD_API hd_status hd_scan_get_profile(hd_scan *scan, hd_profile *out);

/* ------------------------------------------------------------------------
 * Batched execution: many scans of different sizes in one traversal launch.
 *
 * A batch collects work items (a scan and a chunk of its histories, device
 * SoA arrays) without launching anything; hd_batch_run then runs every item:
 * classification, geometry and bucketing of each item on its own stream (they
 * overlap on the GPU), ONE persistent traversal launch whose blocks take the
 * jobs of all scans from a device job counter, the global-memory pass, and
 * (with HD_BATCH_FINALIZE) each scan's decisions.  With graph replay on (the
 * default), the first run of a batch shape is captured into a CUDA graph and
 * later runs with the same items (same scans, pointers and sizes) replay it.
 * Results are identical to running the items one by one with
 * hd_scan_add_histories (and hd_scan_finalize).  Batching is the paper's
 * online mode (Sec. 4) applied to many scans at once; the paper itself
 * processes one data set at a time.
 * ------------------------------------------------------------------------ */
typedef struct hd_batch hd_batch;

enum { HD_BATCH_RESET = 1, HD_BATCH_FINALIZE = 2 };

typedef struct {
    int64_t runs;            /* hd_batch_run calls */
    int64_t graph_captures;  /* runs that captured a new CUDA graph */
    int64_t graph_replays;   /* runs that replayed the cached graph */
    int64_t kernel_launches; /* kernels launched (a replay counts its graph's kernels) */
} hd_batch_stats;

/* Create an empty batch on the current device for up to max_items items
 * (1 <= max_items <= 64; at most 64 different scans per run). */
HD_API hd_status hd_batch_create(int32_t max_items, hd_batch **out);
HD_API hd_status hd_batch_destroy(hd_batch *batch);

/* Queue n histories (device arrays, valid until the run has finished on the
 * GPU) for `scan`.  A scan may appear several times; its items then run in
 * successive rounds.  Nothing is launched.  HD_ERR_STATE when full. */
HD_API hd_status hd_batch_add(hd_batch *batch, hd_scan *scan, const float *angle_deg,
                              const float *u_in, const float *v_in, const float *u_out,
                              const float *v_out, const float *wepl, int64_t n);

/* As hd_batch_add, with per-item flags: HD_BATCH_RESET resets the scan just
 * before this item, HD_BATCH_FINALIZE finalizes it right after this item
 * (for example when the item carries the scan's last angle). */
HD_API hd_status hd_batch_add_item(hd_batch *batch, hd_scan *scan, const float *angle_deg,
                                   const float *u_in, const float *v_in, const float *u_out,
                                   const float *v_out, const float *wepl, int64_t n,
                                   int32_t flags);

/* Run and then drop the queued items, stream-ordered on `stream`.
 * flags: HD_BATCH_RESET resets every scan of the batch first (as
 * hd_scan_reset); HD_BATCH_FINALIZE finalizes every scan afterwards (as
 * hd_scan_finalize).  May synchronise the stream when scan buffers grow. */
HD_API hd_status hd_batch_run(hd_batch *batch, int32_t flags, void *stream);

/* Enable (1, default) or disable (0) CUDA-graph capture and replay. */
HD_API hd_status hd_batch_set_graph(hd_batch *batch, int32_t enable);

HD_API hd_status hd_batch_get_stats(hd_batch *batch, hd_batch_stats *out);

/* ------------------------------------------------------------------------
 * Serving: a request loop for streamed scans (continuous batching).
 *
 * Clients open scans and submit per-angle chunks as they are acquired (the
 * online mode of Sec. 4).  A submit copies its chunk into the scan's open
 * staging segment (device memory for segment_histories histories), so the
 * chunks of a scan that arrive while the GPU is busy lie side by side.  A
 * housekeeping thread admits scans first come, first served while their
 * device footprint fits hbm_budget_bytes (and creates and destroys their
 * device state); a worker thread keeps up to max_in_flight batched
 * launches queued on the GPU, each taking the oldest filled segment of each
 * of up to max_batch admitted scans (one persistent traversal over all of
 * them, as hd_batch_run): every chunk a scan received since its last launch
 * goes in as one item.  A scan's hulls are computed in the launch that
 * carries its last chunk; they stay on the device until the client closes
 * the scan.  A closed scan is kept (its memory still counted in the budget)
 * and reset for a later scan of the same geometry and parameters, or
 * destroyed when an admission needs its memory.  Results equal those of
 * the same chunks added to a lone scan.  Staging memory is bounded by
 * staging_bytes: a submit that finds none free waits for a launch to finish
 * (at most submit_timeout_ms).  Times are seconds since the server was
 * created (-1 when the event has not happened).
 * ------------------------------------------------------------------------ */
typedef struct hd_server hd_server;

typedef struct {
    size_t hbm_budget_bytes; /* device memory the server may give to admitted scans */
    int64_t max_chunk;       /* largest chunk a client submits (histories) */
    int32_t max_batch;       /* scans per launch, 1..64 */
    int32_t max_in_flight;   /* launches queued on the GPU at once, 1..8 */
    int32_t min_batch;       /* while a launch runs, wait for this many scans with
                                pending chunks before queueing the next one (>= 1) */
    int64_t segment_histories; /* histories per staging segment, max_chunk..2^25 */
    size_t staging_bytes;      /* device memory for staging segments (>= one segment,
                                  24 bytes per history) */
    int64_t submit_timeout_ms; /* longest a submit waits for staging space (>= 0) */
} hd_server_config;

typedef struct {
    double t_open, t_admit, t_first_chunk, t_last_chunk, t_ready;
    int64_t histories;
    int32_t chunks_submitted, chunks_done;
    int32_t state; /* 0 waiting for admission, 1 admitted, 2 hulls ready, 3 failed */
} hd_server_scan_info;

typedef struct {
    int64_t scans_opened, scans_admitted, scans_done;
    int64_t chunks_submitted, chunks_launched, launches;
    int64_t bytes_in_use; /* footprint of the admitted scans */
    double issue_seconds; /* host time the worker spent issuing launches */
    double submit_seconds; /* host time spent inside hd_server_submit_chunk (all threads) */
    int64_t items_launched; /* (scan, segment) items over all launches */
    double copy_seconds;    /* of submit_seconds: copying chunks (issue and wait) */
    double alloc_seconds;   /* of submit_seconds: allocating staging segments */
    int64_t scans_reused;   /* admissions that reset a pooled scan instead of creating one */
    int64_t bytes_pooled;   /* footprint of closed scans kept for reuse (counts in the
                               budget; evicted, oldest first, when an admission needs it) */
} hd_server_stats;

/* 64 GiB budget, chunks up to 100000 histories, 64 scans per launch, 2 in
 * flight, min_batch 8, segments of 2^19 histories, 4 GiB of staging, 60 s
 * submit timeout. */
HD_API hd_status hd_server_config_default(hd_server_config *out);

/* Start a server (and its worker thread) on the current device. */
HD_API hd_status hd_server_create(const hd_server_config *cfg, hd_server **out);

/* Stop the worker, wait for the GPU and release every scan. */
HD_API hd_status hd_server_destroy(hd_server *server);

/* Queue a scan that will receive n_chunks chunks.  HD_ERR_ADMISSION when its
 * footprint (counts, masks and chunk scratch) can never fit the budget. */
HD_API hd_status hd_server_open_scan(hd_server *server, const hd_geometry *geom,
                                     const hd_params *params, int32_t n_chunks,
                                     int64_t *scan_id);

/* Submit the next chunk of a scan (1 <= n <= max_chunk; host arrays, or
 * device arrays with on_device = 1).  The data is copied before the call
 * returns, one copy per array.  HD_ERR_STATE when the scan already has all its chunks (or is
 * finished); HD_ERR_TIMEOUT when no staging space freed up within
 * submit_timeout_ms (the chunk was not taken: submit it again);
 * HD_ERR_CUDA when the copy failed (the scan is then failed).  Several
 * threads may submit at once, to the same scan or to different ones. */
HD_API hd_status hd_server_submit_chunk(hd_server *server, int64_t scan_id,
                                        const float *angle_deg, const float *u_in,
                                        const float *v_in, const float *u_out,
                                        const float *v_out, const float *wepl, int64_t n,
                                        int32_t on_device);

/* The same for a chunk whose six columns are rows of one array (one
 * allocation): angle, u_in, v_in, u_out, v_out and WEPL at rows,
 * rows + pitch, ..., rows + 5 pitch (floats; pitch >= n), as a detector
 * readout or a 6 x N tensor holds them.  One strided copy instead of six,
 * which matters when many client threads submit small chunks.  HD_ERR_ARG
 * when pitch < n; otherwise as hd_server_submit_chunk. */
HD_API hd_status hd_server_submit_rows(hd_server *server, int64_t scan_id, const float *rows,
                                       int64_t pitch, int64_t n, int32_t on_device);

/* *done = 1 once the scan's hulls are ready (or it failed: see scan_status). */
HD_API hd_status hd_server_poll(hd_server *server, int64_t scan_id, int32_t *done,
                                hd_status *scan_status);

/* Wait at most timeout_ms for the scan's hulls: HD_OK, HD_ERR_TIMEOUT, or the
 * scan's error. */
HD_API hd_status hd_server_wait(hd_server *server, int64_t scan_id, int64_t timeout_ms);

/* The finished scan, to read with hd_scan_get_mask and the other getters
 * (owned by the server until hd_server_close_scan). */
HD_API hd_status hd_server_scan(hd_server *server, int64_t scan_id, hd_scan **out);

HD_API hd_status hd_server_get_info(hd_server *server, int64_t scan_id,
                                    hd_server_scan_info *out);
HD_API hd_status hd_server_get_stats(hd_server *server, hd_server_stats *out);

/* Release a scan that is finished (or has no chunk in flight). */
HD_API hd_status hd_server_close_scan(hd_server *server, int64_t scan_id);

/* Rows of the hull-restricted system matrix (the step the hull exists for:
 * a reconstruction solves only for the voxels inside it, Sec. 1).  For each
 * of the n histories (device arrays of n float32, as hd_scan_add_histories
 * with on_device = 1; WEPL is not needed), row i lists, in the order the
 * path meets them, the voxels of A_i (Eq. 3.2) that are in the finalised
 * scan's hull of `method` (HD_SC, HD_MSC or HD_SM).  Every history has a
 * row; one with unusable geometry has an empty row.  row_ptr (device, n + 1
 * int64) receives the CSR offsets and *nnz (host) the total; cols (device,
 * `capacity` int32 voxel indices, x fastest) receives the rows when the
 * total fits, otherwise HD_ERR_RANGE with row_ptr and *nnz set, so the
 * caller can size cols and call again.  HD_ERR_STATE when the scan is not
 * finalised or did not run the method.  Synchronises `stream` (to read the
 * total).  Not in the paper's evaluation: the next step of its pipeline. */
HD_API hd_status hd_scan_system_rows(hd_scan *scan, int32_t method, const float *angle_deg,
                                     const float *u_in, const float *v_in, const float *u_out,
                                     const float *v_out, int64_t n, int64_t *row_ptr,
                                     int32_t *cols, int64_t capacity, int64_t *nnz,
                                     void *stream);

/* Atomic-throughput probe: the rate a traversal spending one atomic per
 * voxel-step could reach, measured by kernels that do nothing else (a
 * measurement aid for the roofline; the paper has no counterpart).
 *   HD_PROBE_SMEM_RANDOM    shared-memory atomicAdd to uniformly random words
 *                           of a 128 KB array, one 1024-thread block per SM
 *   HD_PROBE_SMEM_COHERENT  the same with a warp's lanes on consecutive words
 *   HD_PROBE_L2_RANDOM      global atomicAdd to random words of a 16 MB
 *                           (L2-resident) array
 *   HD_PROBE_HBM_RANDOM     the same over a 2 GB array
 * *ops_per_s = atomics per second, the best of three timed launches after a
 * warm-up.  Allocates and frees its own buffers and synchronises the calling
 * thread; call it outside any stream capture. */
enum { HD_PROBE_SMEM_RANDOM = 0, HD_PROBE_SMEM_COHERENT = 1, HD_PROBE_L2_RANDOM = 2,
       HD_PROBE_HBM_RANDOM = 3 };
HD_API hd_status hd_probe_atomics(int32_t kind, double *ops_per_s);

/* Allocation-free accumulation of path counts, for callers that cannot
 * allocate device memory when they run it (inside a stream capture that must
 * stay free of allocation nodes, under a memory pool that forbids
 * cudaMalloc/cudaFree after start-up, or on a latency-critical path).  The
 * paper has no counterpart: this is a deployment aid.
 *
 * Classifies the n histories (device SoA arrays, as in
 * hd_scan_add_histories) and ADDS one to N[v] (uint32, V entries, device)
 * for every voxel v of every missed path and one to M[v] for every voxel of
 * every hit path, exactly as a scan's N and M accumulate; N is required when
 * params->methods has HD_SC or HD_MSC, M when it has HD_SM (the other may be
 * NULL).  The caller zeroes N and M before the first call of an acquisition.
 * Histories that are rejected or unused leave no trace (no statistics are
 * kept).
 *
 * Scratch: one fixed array of about 7.3 MB in the library's device image
 * (records of at most 262144 histories per call), held by every GPU that
 * loads the library until the process exits.  n above 262144 returns
 * HD_ERR_RANGE: split larger batches into several calls.  The first call on
 * a device looks up the array's device address (once per device), so make
 * that first call before any stream capture (made during a capture of
 * `stream` it returns HD_ERR_STATE).  The address is kept for the life of
 * the process: do not use this entry point across a reset of the device.  All calls share the array:
 * calls that overlap on the GPU (different streams, or unordered host
 * threads) race on it, so order them on one stream.  Nothing is allocated
 * or freed by any call.  Stream-ordered on `stream`; errors as elsewhere. */
HD_API hd_status hd_accumulate_noalloc(const hd_geometry *geom, const hd_params *params,
                                       const float *angle_deg, const float *u_in,
                                       const float *v_in, const float *u_out,
                                       const float *v_out, const float *wepl, int64_t n,
                                       uint32_t *N, uint32_t *M, void *stream);

/* Classify n WEPL values (Eq. 3.1, Eq. 3.7): cls_out[i] = 1 missed, 2 hit,
 * 0 neither.  Only the two cutoffs of params are used.  wepl and cls_out
 * are both device pointers (on_device = 1) or both host pointers. */
HD_API hd_status hd_classify(const float *wepl, int64_t n, const hd_params *params, uint8_t *cls_out,
                      int32_t on_device, void *stream);

/* ------------------------------------------------------------------------
 * Thick rays (Eq. 3.2 with d_0 > 0; the paper leaves the distance measure
 * d open).  A_i(k) = the voxels within k voxels of a voxel of A_i (reading
 * 1) in the same slice, by the in-plane Chebyshev distance: |dx| <= k,
 * |dy| <= k, same z.  For in-plane voxel size s, k = floor(d_0 / s) (a
 * thickness below the slice thickness).  k = 0 gives A_i itself.
 *
 * A standalone accumulation (no scan, no tiles: each history is walked over
 * the whole grid by one lane; a scan set to thick rays with hd_scan_set_thick
 * counts on its tiled traversal instead).
 * Classifies the n histories (device SoA arrays, as hd_scan_add_histories
 * with on_device = 1) and ADDS one to N[v] for every voxel v of the thick set
 * of every missed history and to M[v] for every hit one (each voxel once per
 * history; uint32, V entries, device; N required when params->methods has
 * HD_SC or HD_MSC, M when it has HD_SM).  The caller zeroes N and M before
 * the first call; the decisions of hd_scan_finalize are then the caller's
 * to apply (for instance H_1 = [N = 0]).  workspace: device memory of at
 * least hd_accumulate_thick_workspace bytes (two int32 difference arrays of
 * about V entries per class), 256-byte aligned; the call clears it.
 * intervals (device, one int64, may be NULL) receives the number of dilated
 * row intervals the call added (each costs two atomics; a measurement aid).
 * HD_ERR_RANGE for k outside [0, 16] or an unsupported geometry.
 * Stream-ordered on `stream`. */
HD_API hd_status hd_accumulate_thick_workspace(const hd_geometry *geom, size_t *bytes);
HD_API hd_status hd_accumulate_thick(const hd_geometry *geom, const hd_params *params, int32_t k,
                                     const float *angle_deg, const float *u_in, const float *v_in,
                                     const float *u_out, const float *v_out, const float *wepl,
                                     int64_t n, uint32_t *N, uint32_t *M, void *workspace,
                                     size_t workspace_bytes, int64_t *intervals, void *stream);

/* ------------------------------------------------------------------------
 * Thick rays as Eq. 3.2 states them with d the Euclidean distance:
 * A_i(d_0) = the voxels whose centre lies within d_0 mm of the closed segment
 * L_i from the entry to the exit point (Sec. 2.1).  Exact: the entry and exit
 * points are the thin paths' fixed-point world points (mm * 2^16, after the
 * integer CORDIC), voxel centres ((2 i + 1 - n) s / 2 with s rounded to
 * 2^-16 mm) and d_0 (rounded to 2^-16 mm, ties to even) enter the distance
 * test in integers, so membership never depends on floating-point rounding
 * (a float filter with certified error bounds settles the tests whose
 * answer it makes certain; the integer test decides the rest).  Thickness
 * reaches across slices whenever d_0 exceeds the distance to the
 * neighbouring slice's centres.
 *
 * Standalone accumulation: classifies the n histories (device SoA arrays)
 * and ADDS one to N[v] for every voxel v of A_i(d_0) of every usable missed
 * history and to M[v] for every hit one (N required when params->methods has
 * HD_SC or HD_MSC, M when it has HD_SM; uint32, V entries, device; the caller
 * zeroes them first).  Histories rejected by the thin paths' rule add
 * nothing.  workspace: at least hd_accumulate_thick_workspace bytes, 256-byte
 * aligned; the call clears it.  rows (device, one int64, may be NULL)
 * receives the number of row intervals added (two atomics each; a
 * measurement aid).  HD_ERR_RANGE for d_0 outside [0, 64] mm or an
 * unsupported geometry.  Stream-ordered on `stream`. */
HD_API hd_status hd_accumulate_euclid(const hd_geometry *geom, const hd_params *params,
                                      float d0_mm, const float *angle_deg, const float *u_in,
                                      const float *v_in, const float *u_out, const float *v_out,
                                      const float *wepl, int64_t n, uint32_t *N, uint32_t *M,
                                      void *workspace, size_t workspace_bytes, int64_t *rows,
                                      void *stream);

/* Set a scan to the Euclidean thick rays above (d_0 in (0, 64] mm) or back to
 * thin paths (0): N, M, the three hulls, the thresholds and the statistics
 * then follow from the sets A_i(d_0) (the statistics' voxel counts are their
 * sizes).  Replaces an in-plane dilation set with hd_scan_set_thick (and is
 * replaced by one).  Only before any histories: HD_ERR_STATE otherwise;
 * HD_ERR_RANGE outside [0, 64] mm.  Allocates the thick rays' workspace.
 * Such scans cannot join a batch (hd_batch_add_item returns HD_ERR_STATE). */
HD_API hd_status hd_scan_set_thick_distance(hd_scan *scan, float d0_mm);

/* ------------------------------------------------------------------------
 * Hull diagnostics (not steps of the method: the measures the paper reports
 * and a fill variant of MSC's hull).  All pointers are device pointers; the
 * volumes are uint8 masks of nx * ny * nz voxels, x fastest.
 *
 * Extra and missing voxels of `hull` against the true object `object` (the
 * counts of Tables 1-2, Sec. 4): counts (device, 2 nz + 2 int64) receives
 * per slice z the extra voxels (hull, not object) at [z] and the missing
 * ones (object, not hull) at [nz + z], and the totals at [2 nz] and
 * [2 nz + 1].  Stream-ordered. */
HD_API hd_status hd_hull_compare(const uint8_t *hull, const uint8_t *object, int32_t nx,
                                 int32_t ny, int32_t nz, int64_t *counts, void *stream);

/* The part of `mask` it encloses within each slice: out = mask minus every
 * mask voxel joined to the slice's border by a 4-connected path of mask
 * voxels.  Applied to the literal MSC hull H_2 (Eq. 3.6), which excludes only
 * the shell of voxels with a steep drop of N, it keeps the region the shell
 * encloses (Eq. 3.6 alone also keeps the far exterior, where N is smooth).
 * HD_ERR_RANGE when ny * ceil(nx / 32) > 24576 (the two slice bitmaps must
 * fit shared memory: up to 784 x 784 voxels per slice).  out may not alias
 * mask.  Stream-ordered. */
HD_API hd_status hd_fill_enclosed(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz,
                                  uint8_t *out, void *stream);

/* SM threshold by edge detection: a documented form of the "modified Canny"
 * picker the paper used for M_t (Sec. 4; the paper does not say what it
 * modified).  Per slice of the SM count volume M (device, uint32, as
 * hd_scan_get_counts gives it):
 *   S = M smoothed by the 3x3 binomial kernel (edge values replicated);
 *   Sobel derivatives of S (replicated), magnitude |Gx| + |Gy|;
 *   non-maximum suppression along the gradient direction (along x when
 *   5 |Gy| < 2 |Gx|, along y when 5 |Gx| < 2 |Gy|, else diagonal): a voxel
 *   is kept when its magnitude is positive, at least its neighbour's against
 *   the gradient and above its neighbour's along it, so a tie keeps the
 *   voxel on the side of larger M;
 *   hysteresis: kept voxels with 2 mag >= the slice's largest kept magnitude
 *   are edges, and so are kept voxels with 5 mag >= it joined to an edge
 *   (8-connected);
 *   M_t = the element of rank floor(q_pct (k - 1) / 100) of the sorted M of
 *   the k edge voxels; H3 = [M >= M_t].  A slice without edges gets M_t = 0,
 *   has_edge = 0 and H3 = 0.
 * Integer arithmetic throughout (exact).  Outputs are device arrays: mt and
 * has_edge nz entries, H3 nx ny nz bytes.  workspace: device memory of at
 * least hd_sm_canny_workspace bytes, 256-byte aligned, not used by anything
 * else while the call's work runs.  HD_ERR_RANGE when ny * ceil(nx / 32) >
 * 24576 (the slice bitmaps must fit shared memory).  Stream-ordered. */
HD_API hd_status hd_sm_canny_workspace(int32_t nx, int32_t ny, int32_t nz, size_t *bytes);
HD_API hd_status hd_sm_canny(const uint32_t *M, int32_t nx, int32_t ny, int32_t nz,
                             int32_t q_pct, void *workspace, size_t workspace_bytes, uint32_t *mt,
                             uint8_t *has_edge, uint8_t *H3, void *stream);

/* ------------------------------------------------------------------------
 * Binned SC: SC as the paper ran it (Sec. 2.2 data cuts; Sec. 3.2, its
 * implementation paragraphs).  Histories are binned by gantry angle and by
 * the lateral and vertical displacement of the path's mid-point,
 * ((u_in + u_out) / 2, (v_in + v_out) / 2), from the volume's centre; angle
 * bins are centred on multiples of the bin size, displacement bin i covers
 * [lo + i size, lo + (i + 1) size).  In each bin a history is cut when its
 * WEPL, lateral slope (u_out - u_in) or vertical slope (v_out - v_in) lies
 * more than k_sigma population standard deviations from the bin's mean (the
 * slopes over the fixed tracker separation stand for the relative angles).
 * A bin whose kept histories have mean WEPL below miss_wepl_mm is missed:
 * in every slice whose centre height lies in its vertical interval, the
 * straight line along the beam at the bin's centre angle and lateral centre,
 * at the slice's centre height, is carved.  The carved image is averaged
 * over a window x window neighbourhood in each slice (outside the grid counts
 * as carved) and a voxel is in the hull when at least min_count voxels of
 * its window are not carved (min_count 11 of 25: the average exceeds 0.4).
 *
 * Exactness: WEPL and slopes are taken in 1/256 mm (rounded to nearest
 * even), angles and displacements in Q16 as for the paths, the per-bin sums
 * in 64-bit integers (exact while a bin holds fewer than 2^27 histories) and
 * the cut as (n x - S)^2 <= k^2 (n Q - S^2) in 128 bits, so the result does
 * not depend on the order of histories or chunks.  A history is binned when
 * its angle and coordinates are in the paths' accepted range, |WEPL| <
 * 1024 mm, both slopes are below 1024 mm in magnitude and its bin exists;
 * others are skipped.
 *
 * Use: create; hd_binned_add_histories for every chunk (the statistics);
 * hd_binned_cut_histories for the same histories again (the cuts; the first
 * call closes the statistics, so add then returns HD_ERR_STATE);
 * hd_binned_finalize; read the hull.  hd_binned_run does all four for one
 * resident array.  History arrays are n float32 each, readable by the
 * device (device, managed or page-locked host memory; HD_ERR_ARG for
 * pageable host memory).  Calls are stream-ordered on `stream` unless they
 * say otherwise. */
typedef struct {
    float angle_bin_deg;  /* 4.0; 360 / angle_bin_deg bins, tiling 360 exactly in Q16 */
    float u_bin_mm;       /* lateral bin size, 1.0 */
    float v_bin_mm;       /* vertical bin size, 5.0 */
    float u_lo_mm;        /* lower edge of the first lateral bin */
    float v_lo_mm;        /* lower edge of the first vertical bin */
    int32_t n_u, n_v;     /* lateral and vertical bins */
    int32_t k_sigma;      /* cut beyond k standard deviations, 3 */
    float miss_wepl_mm;   /* missed when the kept mean WEPL is below this, 1.0 */
    int32_t window;       /* averaging window (odd, 1..15), 5 */
    int32_t min_count;    /* uncarved voxels a window needs, 11 */
} hd_binned_params;

typedef struct {
    int64_t histories_binned; /* histories that fell in a bin */
    int64_t histories_cut;    /* of those, removed by the cuts */
    int64_t bins;             /* bins in the table */
    int64_t bins_used;        /* bins with histories */
    int64_t bins_missed;      /* bins found missed */
    int64_t lines;            /* lines carved: missed bins times the slices each covers */
    int64_t lines_outside;    /* of those, lines whose endpoints are out of range */
} hd_binned_stats;

typedef struct hd_binned hd_binned;

/* The paper's values for `geom`: displacement bins covering the volume's
 * in-plane half-diagonal (rounded up to whole bins) and its height. */
HD_API hd_status hd_binned_params_default(const hd_geometry *geom, hd_binned_params *out);

/* HD_ERR_RANGE when a bin size is outside [1/16, 4096] mm (angle: [1/16,
 * 360] degrees, dividing 360 in Q16), |lo| > 4096 mm, the table exceeds 2^24
 * bins, k_sigma is outside [1, 64], the window is even or outside [1, 15],
 * min_count is outside [0, window^2] or |miss_wepl_mm| >= 1024; otherwise as
 * hd_scan_create.  Allocates 72 bytes per bin and about
 * V * 2.2 bytes on the current device. */
HD_API hd_status hd_binned_create(const hd_geometry *geom, const hd_binned_params *params,
                                  hd_binned **out);
HD_API hd_status hd_binned_destroy(hd_binned *b);

/* Empty the bin table and return to the statistics phase. */
HD_API hd_status hd_binned_reset(hd_binned *b, void *stream);

/* Statistics phase: add n histories' WEPL and slopes to their bins. */
HD_API hd_status hd_binned_add_histories(hd_binned *b, const float *angle_deg, const float *u_in,
                                         const float *v_in, const float *u_out,
                                         const float *v_out, const float *wepl, int64_t n,
                                         void *stream);

/* Cut phase: test n histories against their bins' statistics and add the
 * kept ones' WEPL to the bins.  Give every history added, once. */
HD_API hd_status hd_binned_cut_histories(hd_binned *b, const float *angle_deg, const float *u_in,
                                         const float *v_in, const float *u_out,
                                         const float *v_out, const float *wepl, int64_t n,
                                         void *stream);

/* Decide the missed bins, carve their lines and filter.  HD_ERR_STATE
 * before any cut call. */
HD_API hd_status hd_binned_finalize(hd_binned *b, void *stream);

/* reset, add, cut and finalize over one array of n histories. */
HD_API hd_status hd_binned_run(hd_binned *b, const float *angle_deg, const float *u_in,
                               const float *v_in, const float *u_out, const float *v_out,
                               const float *wepl, int64_t n, void *stream);

/* After finalize: the hull (which = HD_BINNED_HULL) or the carved image
 * before filtering (HD_BINNED_CARVED: 1 = not carved), V bytes in linear
 * voxel order, to device (dst_on_device = 1) or host memory.  HD_ERR_STATE
 * before finalize. */
enum { HD_BINNED_HULL = 0, HD_BINNED_CARVED = 1 };
HD_API hd_status hd_binned_get_image(hd_binned *b, int32_t which, uint8_t *dst, int64_t n,
                                     int32_t dst_on_device, void *stream);

/* The bin table, n_bins x 9 int64 (bin index = angle + n_ang (u + n_u v)):
 * histories, sums of WEPL, lateral and vertical slope (1/256 mm), sums of
 * their squares, kept histories, kept WEPL sum. */
HD_API hd_status hd_binned_get_bins(hd_binned *b, int64_t *dst, int64_t n_bins,
                                    int32_t dst_on_device, void *stream);

/* Counters; synchronises `stream`. */
HD_API hd_status hd_binned_get_stats(hd_binned *b, hd_binned_stats *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HULLD_H */
