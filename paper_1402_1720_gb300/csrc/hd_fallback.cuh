// General-walk traversal in global memory: histories (or tile pieces of
// them) whose walk has no closed form or does not fit the tiled pass.
#pragma once

#include "hd_geom.cuh"

namespace hd {
namespace {

// Global-memory voxel update of one history: one atomic add into N or M.
struct GlobalVisit {
    uint32_t *vol;  // N or M
    __device__ __forceinline__ void operator()(uint32_t v) const { atomicAdd(vol + v, 1u); }
};

// The voxels of a segment clipped to one tile of tp (gi, go relative to the
// tile's origin, grid Q16), by the general run walk, visited with global
// indices; returns how many.
__device__ unsigned walk_tile_global(const TilePlan &tp, const int32_t gi[3], const int32_t go[3],
                                     int tile, const GlobalVisit &visit)
{
    const int tix = tile % tp.ntx;
    const int tiy = (tile / tp.ntx) % tp.nty;
    const int tiz = tile / (tp.ntx * tp.nty);
    const int x0 = tix * tp.tx, y0 = tiy * tp.ty, z0 = tiz * tp.tz;
    const int dx = min(tp.tx, tp.nx - x0), dy = min(tp.ty, tp.ny - y0), dz = min(tp.tz, tp.nz - z0);
    RunWalk w;
    if (!run_begin(w, gi, go, dx, dy, dz)) return 0;
    const bool ymaj = (w.flags >> 5) & 1;
    unsigned c = 0;
    int row, lo, hi;
    while (run_next(w, row, lo, hi)) {
        // x-major rows are y + dy z, y-major rows x + dx z (box-local)
        const int ra = ymaj ? row % dx : row % dy;
        const int lz = ymaj ? row / dx : row / dy;
        for (int m = lo; m <= hi; ++m) {
            const uint32_t X = static_cast<uint32_t>(x0 + (ymaj ? ra : m));
            const uint32_t Y = static_cast<uint32_t>(y0 + (ymaj ? m : ra));
            const uint32_t Z = static_cast<uint32_t>(z0 + lz);
            visit(X + static_cast<uint32_t>(tp.nx) * (Y + static_cast<uint32_t>(tp.ny) * Z));
        }
        c += static_cast<unsigned>(hi - lo + 1);
    }
    return c;
}

// A pair slot holding a general walk instead of a lean one: the segment's
// tile-local endpoints, marked empty for the lean pass (LeanWalk flag bit 3
// in word 5), with 2 tile + class in word 7.
__device__ __forceinline__ void general_pack(const int32_t gi[3], const int32_t go[3], int tile,
                                             int cls, uint32_t o[kLeanWords])
{
    o[0] = static_cast<uint32_t>(gi[0]);
    o[1] = static_cast<uint32_t>(gi[1]);
    o[2] = static_cast<uint32_t>(gi[2]);
    o[3] = static_cast<uint32_t>(go[0]);
    o[4] = static_cast<uint32_t>(go[1]);
    o[5] = 8u << 16;
    o[6] = static_cast<uint32_t>(go[2]);
    o[7] = 2u * static_cast<uint32_t>(tile) + static_cast<uint32_t>(cls);
}

}  // namespace
}  // namespace hd
