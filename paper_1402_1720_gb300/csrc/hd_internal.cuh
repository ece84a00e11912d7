// Internal definitions shared by the CUDA translation units of libhulld.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hulld.h"

namespace hd {

constexpr int64_t kQ16 = 65536;
constexpr int kMaxN = 4096;

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
};

// Device-side counters of one scan.
struct Ctrl {
    unsigned long long n_in, n_miss, n_hit, n_none, n_reject;
    unsigned long long steps_miss, steps_hit;
    unsigned int rec_miss;  // records appended from the front of the list
    unsigned int rec_hit;   // records appended from the back of the list
    unsigned long long slice_key_pad;
};

// Compacted traversal records: grid Q16 entry and exit points, int32 each
// (|G| < 2^30).  Missed histories fill [0, rec_miss), hit ones fill
// [cap - rec_hit, cap).  Structure of arrays.
struct Records {
    int32_t *g[6];  // x0, y0, z0, x1, y1, z1
    int64_t cap;
};

struct Inputs {
    const float *angle, *u_in, *v_in, *u_out, *v_out, *wepl;
};

// Which voxel update a traversal applies.
enum TraceMode : int { kCount = 0, kCarve = 1 };

// ---- launchers (stream-ordered; return the launch's cudaError_t) ----
cudaError_t launch_ingest(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cordic,
                          float tau_l, float tau_h, int use_miss, int use_hit,
                          const Records &rec, Ctrl *ctrl, int sm_count, cudaStream_t s);

cudaError_t launch_trace(const Records &rec, const Ctrl *ctrl_counts, Ctrl *ctrl_stats,
                         int64_t miss_upper, int64_t hit_upper, const GeomQ &g,
                         uint32_t *N, uint32_t *M, uint32_t *carve, int sm_count, cudaStream_t s);

cudaError_t launch_classify(const float *wepl, int64_t n, float tau_l, float tau_h,
                            uint8_t *cls, cudaStream_t s);

struct DecideArgs {
    int32_t nx, ny, nz;
    int32_t methods;
    int32_t nt, nbhd, sm_ge, sm_per_slice;
    const uint32_t *N;       // may be null when MSC is off
    const uint32_t *M;       // may be null when SM is off
    const uint32_t *carve;   // SC carve bits (used when N is null)
    unsigned long long *slice_key;  // nz entries (SM)
    uint32_t *mt, *slope;    // nz entries (SM)
    long long *index;        // nz entries (SM)
    uint8_t *H1, *H2, *H3;
};

cudaError_t launch_finalize(const DecideArgs &a, int sm_count, cudaStream_t s);

cudaError_t launch_pack_bits(const uint8_t *mask, int64_t V, uint32_t *bits, cudaStream_t s);

// Compaction: writes ascending indices of mask != 0 to out (if count fits
// capacity) and the total to *d_count.  `block_counts` holds
// ceil(V / 1024) + 1 uint32 of scratch.
cudaError_t launch_compact(const uint8_t *mask, int64_t V, int32_t *out, int64_t capacity,
                           uint32_t *block_counts, unsigned long long *d_count, cudaStream_t s);

}  // namespace hd
