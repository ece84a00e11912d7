// Thick rays by the Euclidean distance of Eq. 3.2 (d_0 > 0, d the distance
// from a voxel's centre to the closed segment L_i, Sec. 2.1): A_i(d_0) = the
// voxels whose centre lies within d_0 mm of L_i.  Counted into N and M like
// the thin paths, once per history for every voxel of its A_i(d_0).  The
// exact membership test, its float filter and the row search are in
// hd_euclid.cuh.
//
// Work.  A warp takes groups of 32 consecutive histories (so each lane's
// gantry cos/sin rarely change); each lane classifies one history and sets
// its capsule up (endpoints, index box, the float part) in shared memory.  Then the
// warp takes the group's histories one at a time: its lanes take the rows of
// voxels along the segment's major in-plane axis that cross the box bounding
// the capsule (segment grown by d_0).  Each nonempty row adds +1 / -1 to a
// difference array along the major axis (the thick rays' workspace), and row
// prefix sums add them to N and M.
#include <cmath>
#include <cstdint>

#include "hd_euclid.cuh"
#include "hd_thick.cuh"

namespace hd {
namespace {

constexpr int kEuThreads = 256;
constexpr int kEuBlocksPerSm = 2;  // resident blocks per SM (the launch bounds)
constexpr int kEuGroup = 32;  // consecutive histories a warp takes at once, one per lane

struct EuCounts {
    unsigned n_in = 0, n_miss = 0, n_hit = 0, n_none = 0, n_reject = 0;
};

// One history of a warp's group, as the lane that set it up left it.
struct EuSlot {
    long long A[3], B[3];  // doubled endpoints in the capsule's frame
    CapF cf;               // the float part of its capsule
    int16_t blo1, bhi1, blo2, bhi2;  // index box of the rows on axes 1 and 2
    int flags;             // bit 0: hit class, bit 1: rows along y, bit 2: has rows
};

__global__ void __launch_bounds__(kEuThreads, kEuBlocksPerSm) euclid_kernel(Inputs in, int64_t n, GeomQ g,
                                                            Cordic cd, float tau_l, float tau_h,
                                                            int use_miss, int use_hit,
                                                            long long R2, ThickDiff td,
                                                            unsigned long long *stats,
                                                            unsigned long long *next)
{
    const unsigned lane = threadIdx.x & 31u;
    const int warp = static_cast<int>(threadIdx.x >> 5);
    // per warp: a queue of rows to process (at most 31 left + 32 new), the
    // group's histories, and the exact part of the current one's capsule
    __shared__ int s_queue[kEuThreads / 32][64];
    __shared__ EuSlot s_slot[kEuThreads / 32][kEuGroup];
    __shared__ CapX s_cx[kEuThreads / 32];
    int *const queue = s_queue[warp];
    EuSlot *const slot = s_slot[warp];
    CapX *const cxs = &s_cx[warp];
    EuCounts nc;
    unsigned long long vox[2] = {0, 0}, rows = 0;
    bool tc_valid = false;
    float tc_ang = 0.0f;
    long long tc_c = 0, tc_s = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(next, static_cast<unsigned long long>(kEuGroup));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= static_cast<unsigned long long>(n)) break;
        // each lane sets one history of the group up: class, endpoints
        // (rejected by the thin rule like the thin paths), capsule frame
        const int64_t i = static_cast<int64_t>(base) + lane;
        EuSlot &e = slot[lane];
        __syncwarp();  // the previous group is done with the slots
        int flags = 0;
        if (i < n) {
            const float w = in.wepl[i];
            const int cls = w < tau_l ? 0 : (w > tau_h ? 1 : -1);
            nc.n_in += 1;
            nc.n_miss += cls == 0;
            nc.n_hit += cls == 1;
            nc.n_none += cls < 0;
            if (!(cls < 0 || (cls == 0 && !use_miss) || (cls == 1 && !use_hit))) {
                const float ang = in.angle[i];
                const float ui = in.u_in[i], vi = in.v_in[i], uo = in.u_out[i], vo = in.v_out[i];
                bool ok = fabsf(ang) < 1048576.0f;
                int32_t G[6];
                if (ok) {
                    if (!tc_valid || ang != tc_ang) {
                        cordic_cs(q16_of(ang), cd, tc_c, tc_s);
                        tc_ang = ang;
                        tc_valid = true;
                    }
                    ok = endpoints_cs(g, tc_c, tc_s, ui, vi, uo, vo, G);  // the thin rule
                }
                if (!ok) {
                    nc.n_reject += 1;
                } else {
                    long long W[6];
                    world_cs(g, tc_c, tc_s, ui, vi, uo, vo, W);
                    bool ymaj;
                    int blo[3], bhi[3];
                    float S;
                    long long A[3], B[3];
                    if (capsule_frame(g, W, R2, A, B, ymaj, blo, bhi, S)) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            e.A[q] = A[q];
                            e.B[q] = B[q];
                        }
                        CapX cx;
                        capx_of(g, A, B, ymaj, R2, cx);
                        e.cf = capf_of(cx, S, R2);
                        e.blo1 = static_cast<int16_t>(blo[1]);
                        e.bhi1 = static_cast<int16_t>(bhi[1]);
                        e.blo2 = static_cast<int16_t>(blo[2]);
                        e.bhi2 = static_cast<int16_t>(bhi[2]);
                        flags = cls | (ymaj ? 2 : 0) | 4;
                    }
                }
            }
        }
        e.flags = flags;
        __syncwarp();
        // the group's histories one at a time, all lanes on the rows of each
        for (int j = 0; j < kEuGroup; ++j) {
            const int fl = slot[j].flags;
            if (!(fl & 4)) continue;
            const int cls = fl & 1;
            const bool ymaj = (fl & 2) != 0;
            __syncwarp();  // the previous history is done with *cxs
            if (lane == 0) capx_of(g, slot[j].A, slot[j].B, ymaj, R2, *cxs);
            __syncwarp();
            const CapF cf = slot[j].cf;
            const int blo1 = slot[j].blo1, bhi1 = slot[j].bhi1;
            const int blo2 = slot[j].blo2, bhi2 = slot[j].bhi2;
            int32_t *diff = ymaj ? td.dy[cls] : td.dx[cls];
            const int n1 = ymaj ? g.nx : g.ny;
            // the rows that can meet the capsule queue up in shared memory;
            // whenever 32 are queued all lanes take one each, so the interval
            // search runs with full warps
            int qn = 0;
            auto drain = [&](int keep) {
                while (qn > keep) {
                    __syncwarp();
                    int lo, hi;
                    if (static_cast<int>(lane) < qn &&
                        row_interval(cf, *cxs, queue[lane] & 0xffff, queue[lane] >> 16, lo, hi)) {
                        const int ra = queue[lane] & 0xffff, rk = queue[lane] >> 16;
                        // x-major rows: (nx + 1) entries per (y, z); y-major:
                        // (ny + 1) per (x, z)
                        int32_t *row = diff + (static_cast<int64_t>(ra) +
                                               static_cast<int64_t>(n1) * rk) *
                                                  (cf.n0 + 1);
                        atomicAdd(row + lo, 1);
                        atomicAdd(row + hi + 1, -1);
                        vox[cls] += static_cast<unsigned>(hi - lo + 1);
                        rows += 1;
                    }
                    __syncwarp();
                    // keep what did not fit (fewer than 32 entries)
                    const int rest = qn > 32 ? qn - 32 : 0;
                    const int moved = static_cast<int>(lane) < rest ? queue[32 + lane] : 0;
                    __syncwarp();
                    if (static_cast<int>(lane) < rest) queue[lane] = moved;
                    __syncwarp();
                    qn = rest;
                }
            };
            // each lane one index a of the box, with the band of k whose rows
            // can meet the capsule
            for (int ab = blo1; ab <= bhi1; ab += 32) {
                const int a = ab + static_cast<int>(lane);
                int klo = 1, khi = 0;
                if (a <= bhi1) k_range(cf, a, blo2, bhi2, klo, khi);
                const int cnt = khi >= klo ? khi - klo + 1 : 0;
                const int most = __reduce_max_sync(0xffffffffu, cnt);
                for (int t = 0; t < most; ++t) {
                    const int k = klo + t;
                    // inside the band nearly every row meets the capsule, and
                    // the row search is exact for any row: the band's rows go
                    // to it directly; a whole box is filtered first
                    const bool meets = t < cnt && (cf.kband || row_meets_at(cf, *cxs, a, k));
                    const unsigned bal = __ballot_sync(0xffffffffu, meets);
                    if (meets) queue[qn + __popc(bal & ((1u << lane) - 1u))] = a | (k << 16);
                    qn += __popc(bal);
                    drain(31);
                }
            }
            drain(0);
        }
    }
    const unsigned long long part[8] = {nc.n_in, nc.n_miss, nc.n_hit, nc.n_none, nc.n_reject,
                                        vox[0], vox[1], rows};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        unsigned long long e = part[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0 && e != 0) atomicAdd(stats + q, e);
    }
}

}  // namespace

cudaError_t launch_euclid(const Inputs &in, int64_t n, const hd_geometry *geom, const GeomQ &g,
                          const Cordic &cd, float tau_l, float tau_h, int use_miss, int use_hit,
                          float d0, void *workspace, uint32_t *N, uint32_t *M,
                          unsigned long long *stats, int64_t *rows, int sm_count,
                          cudaStream_t st)
{
    const size_t need = thick_workspace_bytes(geom);
    cudaError_t e = cudaMemsetAsync(workspace, 0, need, st);
    if (e == cudaSuccess && n > 0) {
        const long long R2 = 2 * q16_of(d0);
        const ThickDiff td = thick_diff_of(geom, workspace);
        unsigned long long *cnt = thick_counters_of(geom, workspace);
        // persistent warps
        int64_t blocks = int64_t(sm_count > 0 ? sm_count : 1) * kEuBlocksPerSm;
        const int64_t want = (n + kEuGroup * (kEuThreads / 32) - 1) /
                             (kEuGroup * (kEuThreads / 32));
        if (blocks > want) blocks = want;
        euclid_kernel<<<static_cast<unsigned>(blocks), kEuThreads, 0, st>>>(
            in, n, g, cd, tau_l, tau_h, use_miss, use_hit, R2, td, cnt, cnt + 8);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_thick_finish(geom, workspace, use_miss ? N : nullptr, use_hit ? M : nullptr,
                                stats, rows, st);
    return e;
}

}  // namespace hd

extern "C" {

hd_status hd_accumulate_euclid(const hd_geometry *geom, const hd_params *params, float d0_mm,
                               const float *angle_deg, const float *u_in, const float *v_in,
                               const float *u_out, const float *v_out, const float *wepl,
                               int64_t n, uint32_t *N, uint32_t *M, void *workspace,
                               size_t workspace_bytes, int64_t *rows, void *stream)
{
    if (!geom || !params || n < 0 || !workspace) return HD_ERR_ARG;
    if (!(d0_mm >= 0.0f && d0_mm <= 64.0f)) return HD_ERR_RANGE;
    const hd_status gs = hd::check_geometry(geom);
    if (gs != HD_OK) return gs;
    if (std::isnan(params->wepl_miss_lt) || std::isnan(params->wepl_hit_gt) ||
        params->wepl_miss_lt > params->wepl_hit_gt)
        return HD_ERR_ARG;
    const uint32_t m = params->methods;
    if (m == 0 || (m & ~uint32_t(HD_SC | HD_MSC | HD_SM))) return HD_ERR_ARG;
    const int use_miss = (m & (HD_SC | HD_MSC)) ? 1 : 0;
    const int use_hit = (m & HD_SM) ? 1 : 0;
    if ((use_miss && !N) || (use_hit && !M)) return HD_ERR_ARG;
    if (n > 0 && (!angle_deg || !u_in || !v_in || !u_out || !v_out || !wepl)) return HD_ERR_ARG;
    if (workspace_bytes < hd::thick_workspace_bytes(geom) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return HD_ERR_ARG;
    hd::Cordic cd{};
    if (!hd::make_cordic_table(cd)) return HD_ERR_RANGE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    const hd::GeomQ gq = hd::make_geomq(geom->nx, geom->ny, geom->nz, geom->sx, geom->sy,
                                        geom->sz, geom->tracker_half_sep_mm);
    const hd::Inputs in{angle_deg, u_in, v_in, u_out, v_out, wepl};
    const cudaError_t e = hd::launch_euclid(in, n, geom, gq, cd, params->wepl_miss_lt,
                                            params->wepl_hit_gt, use_miss, use_hit, d0_mm,
                                            workspace, N, M, nullptr, rows, sms,
                                            static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        hd::note_cuda_error(e, "hd_accumulate_euclid");
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // extern "C"
