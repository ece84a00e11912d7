// Thick rays inside the library: the launch sequence of hd_accumulate_thick,
// shared with scans set to thick rays (hd_scan_set_thick).
#pragma once

#include "hd_internal.cuh"

namespace hd {

// Workspace bytes of one thick accumulation over this grid.
size_t thick_workspace_bytes(const hd_geometry *geom);

// Clears the workspace, adds the thick sets of n histories to N (missed) and
// M (hit) (either may be null when its class is not used), and, when
// `stats` is not null, adds to stats[0..6]: histories, missed, hit, neither,
// rejected, voxel memberships of missed and of hit histories.  `intervals`
// (may be null) receives the row intervals emitted.
cudaError_t launch_thick(const Inputs &in, int64_t n, const hd_geometry *geom, const GeomQ &g,
                         const Cordic &cd, float tau_l, float tau_h, int use_miss, int use_hit,
                         int k, void *workspace, uint32_t *N, uint32_t *M,
                         unsigned long long *stats, int64_t *intervals, int sm_count,
                         cudaStream_t st);

}  // namespace hd
