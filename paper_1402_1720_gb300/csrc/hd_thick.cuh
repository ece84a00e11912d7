// Thick rays inside the library: the dilated-interval emission shared by the
// thick kernels, and the launch sequences of hd_accumulate_thick and of scans
// set to thick rays (hd_scan_set_thick).
#pragma once

#include "hd_geom.cuh"

namespace hd {

constexpr int kThickMaxK = 16;

// Global difference arrays of the thick counts: along x, (nx + 1) entries
// per (y, z) row; along y, (ny + 1) entries per (x, z) column; one pair for
// the missed class (0) and one for the hit class (1).
struct ThickDiff {
    int32_t *dx[2], *dy[2];
};

// The last 2k + 1 runs of a walk in the current slice.
struct ThickRing {
    int lo[2 * kThickMaxK + 1], hi[2 * kThickMaxK + 1];
};

// Adds the interval of target row t (minor index) of a slice to a global
// difference array: the union of the window's runs (first and last in ring
// slots pa and pb) grown by k, clipped to the row.  Returns 1 and adds the
// interval's voxels to `voxels` when t is inside the slice.
__device__ __forceinline__ unsigned thick_emit_global(const ThickRing &rg, int pa, int pb, int t,
                                                      int k, int nminor, int nmaj, int32_t *diff,
                                                      int64_t slice_row0, unsigned &voxels)
{
    if (t < 0 || t >= nminor) return 0;
    const int lo = max(min(rg.lo[pa], rg.lo[pb]) - k, 0);
    const int hi = min(max(rg.hi[pa], rg.hi[pb]) + k, nmaj - 1);
    int32_t *row = diff + (slice_row0 + t) * static_cast<int64_t>(nmaj + 1);
    atomicAdd(row + lo, 1);
    atomicAdd(row + hi + 1, -1);
    voxels += static_cast<unsigned>(hi - lo + 1);
    return 1;
}

// A whole walk (begun on a box whose rows are minor + nminor zl, the box's
// slice zl being grid slice z0 + zl) streamed through the ring: in each
// slice of J runs, the targets centred on runs -k .. J - 1 + k, the one
// centred on run j - k once run j has arrived and the last k at the slice's
// end.  Returns the intervals emitted; adds their voxels to `voxels`.
__device__ __forceinline__ unsigned thick_walk_all(RunWalk &wk, int nminor, int nmaj, int z0,
                                                   int k, int s, int32_t *diff, ThickRing &rg,
                                                   unsigned &voxels)
{
    const int R = 2 * k + 1;
    unsigned e = 0;
    int zc = -1, m0 = 0, j = 0, p = 0, prev = 0;
    int64_t row0 = 0;
    int row, lo, hi;
    auto close = [&]() {
        const int pb = p == 0 ? R - 1 : p - 1;
        for (int jc = j - k; jc <= j - 1 + k; ++jc) {
            const int ja = jc - k;
            e += thick_emit_global(rg, ja <= 0 ? 0 : ja % R, pb, m0 + s * jc, k, nminor, nmaj, diff,
                                   row0, voxels);
        }
    };
    while (run_next(wk, row, lo, hi)) {
        // inside a slice consecutive runs differ by one row
        const int step = row - prev;
        prev = row;
        if (zc < 0 || step > 1 || step < -1 || nminor <= 2) {
            const int mz = row / nminor;
            if (mz != zc) {
                if (zc >= 0) close();
                zc = mz;
                m0 = row - mz * nminor;
                row0 = static_cast<int64_t>(z0 + mz) * nminor;
                j = 0;
                p = 0;
            }
        }
        rg.lo[p] = lo;
        rg.hi[p] = hi;
        e += thick_emit_global(rg, j >= 2 * k ? (p + 1 == R ? 0 : p + 1) : 0, p, m0 + s * (j - k), k,
                               nminor, nmaj, diff, row0, voxels);
        ++j;
        p = p + 1 == R ? 0 : p + 1;
    }
    if (zc >= 0) close();
    return e;
}

// Workspace bytes of the thick counts over this grid (difference arrays and
// counters), and the difference arrays inside a workspace.
size_t thick_workspace_bytes(const hd_geometry *geom);
ThickDiff thick_diff_of(const hd_geometry *geom, void *workspace);

// The workspace's 8 counters (see launch_thick) and its work counter.
unsigned long long *thick_counters_of(const hd_geometry *geom, void *workspace);

// Adds the workspace's difference arrays to N and M (either may be null)
// by prefix sums along their rows, and, when `stats` / `intervals` are not
// null, adds the counters 0..6 to stats and stores counter 7 in *intervals.
cudaError_t launch_thick_finish(const hd_geometry *geom, void *workspace, uint32_t *N,
                                uint32_t *M, unsigned long long *stats, int64_t *intervals,
                                cudaStream_t st);

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

// Euclidean thick rays (hd_euclid.cu): clears the workspace, adds the sets
// A_i(d0) = {v : centre of v within d0 mm of L_i} of n histories to N and M
// (either may be null when its class is not used), and, when `stats` is not
// null, adds to stats[0..6] as launch_thick does; *rows (may be null)
// receives the number of row intervals added.
cudaError_t launch_euclid(const Inputs &in, int64_t n, const hd_geometry *geom, const GeomQ &g,
                          const Cordic &cd, float tau_l, float tau_h, int use_miss, int use_hit,
                          float d0, void *workspace, uint32_t *N, uint32_t *M,
                          unsigned long long *stats, int64_t *rows, int sm_count,
                          cudaStream_t st);

// The tiled traversal of thick rays over one scan's jobs (trace_thick_kernel).
cudaError_t launch_trace_thick(const ScanDesc *desc_dev, int *job_counter, int k,
                               const ThickDiff &td, int smem_words, int threads, int grid,
                               cudaStream_t st);

// The tiled form for a scan whose tiles are whole one-slice planes: the
// lean pairs into shared-memory difference arrays flushed per job, the
// fallback pairs and the records of the global path into the workspace's
// global difference arrays (cleared first), which are then added to N and M.
cudaError_t launch_thick_scan(const ScanDesc *desc_dev, const hd_geometry *geom,
                              const Records &rec, Ctrl *ctrl, int64_t upper, const GeomQ &g,
                              int k, void *workspace, uint32_t *N, uint32_t *M, int smem_words,
                              int threads, int sm_count, cudaStream_t st);

}  // namespace hd
