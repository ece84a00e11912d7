// Ingest (classification, fixed-point geometry, each record at its
// history's slot with its path decided against the block's pair budget) and
// the global-memory traversal that accumulates N and M for the records that
// do not take the tiled path.
//
// Classification: Eq. 3.1 (missed, WEPL below the cutoff) and Eq. 3.7 (hit,
// WEPL above the cutoff).  Path: the closed segment between entry and exit
// (Sec. 2.1), A_i of Eq. 3.2 read with d_0 = 0 against half-open voxel
// cubes.  Accumulation: N of Eq. 3.4 (Alg. 2; SC's H_1 = [N = 0] of Eq. 3.3
// is the carve of Alg. 1 as a set difference), M of Eq. 3.9 (Alg. 3).
//
// The global traversal is an exact integer DDA.  For the segment
// P(t) = G_in + t D (grid coordinates with 16 fractional bits) the next
// plane crossing of axis a happens at t_a = num_a / |D_a|; the walk keeps the
// three cross-multiplied differences E_ab = num_a |D_b| - num_b |D_a| (their
// signs order the crossings) and updates them with additions only.  Ties
// follow the floor semantics of half-open cubes: at equal t an axis moving
// + enters its next voxel at t itself, an axis moving - leaves its voxel
// just after t, so a mixed tie visits the corner voxel between the two.
// The walk starts at the parameter where the segment enters the grid box
// (exact rational), so voxels outside the grid cost nothing.
#include "hd_fallback.cuh"

namespace hd {

namespace {

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ ingest

struct LaneAcc {
    unsigned n_in = 0, n_miss = 0, n_hit = 0, n_none = 0, n_reject = 0;
};

// Classify one history and, when it is traversed, compute its record.
// Returns 1 (missed record), 2 (hit record) or 0 (nothing to traverse).
// cos/sin of the last gantry angle a lane quantised (histories arrive
// grouped by angle, so consecutive ones usually share it).
// cos/sin of a gantry angle, kept out of line: it runs about once per
// thread and grid-stride step (histories arrive grouped by angle), and
// inlining its 32 unrolled iterations into each of the four history slots
// costs more in instruction fetch than the call.
__device__ __noinline__ void trig_refresh(float ang, const Cordic &cd, long long &c, long long &s)
{
    cordic_cs(q16_of(ang), cd, c, s);
}

struct TrigCache {
    bool valid = false;
    float ang = 0.0f;
    long long c = 0, s = 0;
};

__device__ __forceinline__ int ingest_one(const GeomQ &g, const Cordic &cd, float tau_l,
                                          float tau_h, int use_miss, int use_hit, float ang,
                                          float ui, float vi, float uo, float vo, float w,
                                          int32_t rec[6], LaneAcc &acc, TrigCache &tc)
{
    acc.n_in += 1;
    int cls = 0;
    if (w < tau_l) {
        cls = 1;
        acc.n_miss += 1;
    } else if (w > tau_h) {
        cls = 2;
        acc.n_hit += 1;
    } else {
        acc.n_none += 1;
    }
    if (!((cls == 1 && use_miss) || (cls == 2 && use_hit))) return 0;
    bool ok = fabsf(ang) < 1048576.0f;
    if (ok) {
        if (!tc.valid || ang != tc.ang) {
            trig_refresh(ang, cd, tc.c, tc.s);
            tc.ang = ang;
            tc.valid = true;
        }
        ok = endpoints_cs(g, tc.c, tc.s, ui, vi, uo, vo, rec);
    }
    if (!ok) {
        acc.n_reject += 1;
        return 0;
    }
    return cls;
}


__device__ __forceinline__ unsigned warp_incl_scan(unsigned v)
{
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= static_cast<unsigned>(o)) v += t;
    }
    return v;
}

// Decide the path of each lane's record (tiled within the block's pair
// budget, else global), count its tiles in the block histogram, list its
// pairs in the block's share of stage, and write it at its history's slot
// i (when i < i1; cls 0: no record).  Budget reservations are per warp on a
// shared-memory counter, so the block never waits at a barrier.  The pairs
// the budget admits fill the list from its start without gaps: the
// reservations tile [0, total) in the order of their ends, and only the one
// record that straddles the budget, and the records after it, are turned
// away (they take the global path, exact either way).
__device__ __forceinline__ void admit_and_write(const TilePlan &tp, const Records &rec,
                                                Ctrl *ctrl, uint32_t *s_hist, unsigned *s_demand,
                                                unsigned budget, int64_t h0, int64_t i,
                                                int64_t i1, uint32_t *stage, int cls,
                                                const int32_t r[6])
{
    int tcount = 0;
    int zlo = 0, zhi = 0;
    bool ok = false;
    if (cls != 0) {
        int c = 0;
        if (grid_z_range(tp, r, zlo, zhi)) {
            if (tp.ntx == 1 && tp.nty == 1) {
                // whole-plane tiles: the part inside the grid's x-y extent
                // meets every plane tile of its slices
                const unsigned m = tp.mtz;
                const int t0 = m ? static_cast<int>(umulhi32(static_cast<unsigned>(zlo), m)) : zlo;
                const int t1 = m ? static_cast<int>(umulhi32(static_cast<unsigned>(zhi), m)) : zhi;
                c = t1 - t0 + 1;
            } else {
                int lo[3], hi[3];
                c = tile_range_z(tp, r, zlo, zhi, lo, hi);
            }
        }
        ok = c != 0;  // else no voxel of the grid: nothing to traverse
        tcount = (tp.ntiles > 0 && c <= tp.max_tiles) ? c : -1;
    }
    const unsigned demand = ok && tcount > 0 ? static_cast<unsigned>(tcount) : 0u;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned incl = warp_incl_scan(demand);
    const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned wbase = 0;
    if (lane == 31 && tot) wbase = atomicAdd(s_demand, tot);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    const unsigned long long end = static_cast<unsigned long long>(wbase) + incl;
    const int path = ok ? (demand > 0 && end <= budget ? 1 : 2) : 0;
    if (rec.glist) {
        // the global path's list: one counter update per warp
        const unsigned gm = __ballot_sync(0xffffffffu, path == 2);
        if (gm) {
            const int lead = __ffs(gm) - 1;
            unsigned gb = 0;
            if (static_cast<int>(lane) == lead) gb = atomicAdd(&ctrl->n_global, __popc(gm));
            gb = __shfl_sync(0xffffffffu, gb, lead);
            if (path == 2) rec.glist[gb + __popc(gm & ((1u << lane) - 1u))] = static_cast<int32_t>(i);
        }
    }
    if (i >= i1) return;
    int32_t st = 0;
    if (ok) {
        st = record_status(path, cls - 1, zlo, zhi);
        if (path == 1) {
            int lo[3], hi[3];
            if (tp.ntx == 1 && tp.nty == 1) {
                const unsigned m = tp.mtz;
                lo[0] = hi[0] = lo[1] = hi[1] = 0;
                lo[2] = m ? static_cast<int>(umulhi32(static_cast<unsigned>(zlo), m)) : zlo;
                hi[2] = m ? static_cast<int>(umulhi32(static_cast<unsigned>(zhi), m)) : zhi;
            } else {
                tile_range_z(tp, r, zlo, zhi, lo, hi);
            }
            const int off = (cls - 1) * tp.ntiles;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x)
                        atomicAdd(&s_hist[off + x + tp.ntx * (y + tp.nty * z)], 1u);
            // the record's pairs hold positions end - c .. end - 1 of the
            // block's list (all below its budget)
            const uint32_t code = static_cast<uint32_t>(i - h0) << kRecordTileBits;
            const unsigned first = static_cast<unsigned>(end) - demand;
            for (int j = 0; j < tcount; ++j) stage[first + j] = code | static_cast<uint32_t>(j);
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) rec.g[a][i] = r[a];
    }
    rec.status[i] = st;
}

// One block per range of the chunk split.  Inputs in device memory: one
// history per thread and step (coalesced 32-bit loads of each array), which
// keeps a single inlined copy of the per-history code (four per step ran
// slower from HBM, for the instruction-cache misses and register spills).
// kWide, for inputs read in place from page-locked host memory: four
// consecutive histories per thread and step from 128-bit loads, since the
// host link serves fewer, larger requests faster.
template <bool kWide>
__global__ void __launch_bounds__(kIngestThreads, 4) ingest_kernel(
    Inputs in, int64_t n, int64_t per_block, GeomQ g, Cordic cd, float tau_l, float tau_h,
    int use_miss, int use_hit, TilePlan tp, Records rec, Ctrl *ctrl, uint32_t *block_count,
    uint32_t *block_pairs, uint32_t *stage)
{
    extern __shared__ uint32_t s_hist[];  // 2 * ntiles counters
    __shared__ unsigned s_demand, s_total;
    const int nh = 2 * tp.ntiles;
    for (int t = threadIdx.x; t < nh; t += blockDim.x) s_hist[t] = 0;
    if (threadIdx.x == 0) {
        s_demand = 0;
        s_total = 0;
    }
    __syncthreads();
    LaneAcc acc;
    TrigCache tc;
    // the block's histories arrive grouped by gantry angle, so a thread's
    // angle, and its cos/sin, rarely change; every thread of a block runs
    // the same number of steps (warp-wide budget reservations)
    const int64_t h0 = static_cast<int64_t>(blockIdx.x) * per_block;
    const int64_t h1 = h0 + per_block < n ? h0 + per_block : n;
    const unsigned budget =
        h1 > h0 ? static_cast<unsigned>(h1 - h0) * static_cast<unsigned>(tp.pairs_per_record) : 0u;
    uint32_t *const list =
        stage ? stage + static_cast<int64_t>(blockIdx.x) * per_block * tp.pairs_per_record : nullptr;
    if (kWide) {
        for (int64_t base = h0; base < h1; base += 4 * static_cast<int64_t>(blockDim.x)) {
            const int64_t i0 = base + 4 * static_cast<int64_t>(threadIdx.x);
            float a[4] = {0, 0, 0, 0}, ui[4] = {0, 0, 0, 0}, vi[4] = {0, 0, 0, 0},
                  uo[4] = {0, 0, 0, 0}, vo[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
            if (i0 + 3 < h1) {
                const int64_t u = i0 >> 2;
                const float4 A = __ldg(reinterpret_cast<const float4 *>(in.angle) + u);
                const float4 UI = __ldg(reinterpret_cast<const float4 *>(in.u_in) + u);
                const float4 VI = __ldg(reinterpret_cast<const float4 *>(in.v_in) + u);
                const float4 UO = __ldg(reinterpret_cast<const float4 *>(in.u_out) + u);
                const float4 VO = __ldg(reinterpret_cast<const float4 *>(in.v_out) + u);
                const float4 W = __ldg(reinterpret_cast<const float4 *>(in.wepl) + u);
                a[0] = A.x; a[1] = A.y; a[2] = A.z; a[3] = A.w;
                ui[0] = UI.x; ui[1] = UI.y; ui[2] = UI.z; ui[3] = UI.w;
                vi[0] = VI.x; vi[1] = VI.y; vi[2] = VI.z; vi[3] = VI.w;
                uo[0] = UO.x; uo[1] = UO.y; uo[2] = UO.z; uo[3] = UO.w;
                vo[0] = VO.x; vo[1] = VO.y; vo[2] = VO.z; vo[3] = VO.w;
                w[0] = W.x; w[1] = W.y; w[2] = W.z; w[3] = W.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t i = i0 + k;
                    if (i < h1) {
                        a[k] = in.angle[i]; ui[k] = in.u_in[i]; vi[k] = in.v_in[i];
                        uo[k] = in.u_out[i]; vo[k] = in.v_out[i]; w[k] = in.wepl[i];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t i = i0 + k;
                int cls = 0;
                int32_t r[6] = {0, 0, 0, 0, 0, 0};
                if (i < h1)
                    cls = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, a[k], ui[k], vi[k],
                                     uo[k], vo[k], w[k], r, acc, tc);
                admit_and_write(tp, rec, ctrl, s_hist, &s_demand, budget, h0, i, h1, list, cls, r);
            }
        }
    } else {
        for (int64_t base = h0; base < h1; base += blockDim.x) {
            const int64_t i = base + threadIdx.x;
            int cls = 0;
            int32_t r[6] = {0, 0, 0, 0, 0, 0};
            if (i < h1)
                cls = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, in.angle[i],
                                 in.u_in[i], in.v_in[i], in.u_out[i], in.v_out[i], in.wepl[i], r,
                                 acc, tc);
            admit_and_write(tp, rec, ctrl, s_hist, &s_demand, budget, h0, i, h1, list, cls, r);
        }
    }
    const unsigned a0 = warp_sum_u32(acc.n_in), a1 = warp_sum_u32(acc.n_miss),
                   a2 = warp_sum_u32(acc.n_hit), a3 = warp_sum_u32(acc.n_none),
                   a4 = warp_sum_u32(acc.n_reject);
    if ((threadIdx.x & 31u) == 0) {
        if (a0) atomicAdd(&ctrl->n_in, static_cast<unsigned long long>(a0));
        if (a1) atomicAdd(&ctrl->n_miss, static_cast<unsigned long long>(a1));
        if (a2) atomicAdd(&ctrl->n_hit, static_cast<unsigned long long>(a2));
        if (a3) atomicAdd(&ctrl->n_none, static_cast<unsigned long long>(a3));
        if (a4) atomicAdd(&ctrl->n_reject, static_cast<unsigned long long>(a4));
    }
    if (block_count == nullptr) return;
    __syncthreads();
    unsigned mine = 0;
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
        block_count[static_cast<size_t>(t) * gridDim.x + blockIdx.x] = s_hist[t];
        mine += s_hist[t];
    }
    mine = warp_sum_u32(mine);
    if ((threadIdx.x & 31u) == 0 && mine) atomicAdd(&s_total, mine);
    __syncthreads();
    if (threadIdx.x == 0) block_pairs[blockIdx.x] = s_total;
}

// ---------------------------------------------------------------- traversal

__global__ void __launch_bounds__(256) trace_global_kernel(Records rec, Ctrl *ctrl, GeomQ g,
                                                           uint32_t *N, uint32_t *M,
                                                           int all_records)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t total = rec.glist ? static_cast<int64_t>(ctrl->n_global) : rec.cap;
    unsigned taken = 0;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < total;
         k += stride) {
        const int64_t i = rec.glist ? static_cast<int64_t>(rec.glist[k]) : k;
        const int32_t stw = rec.status[i];
        const int path = status_path(stw);
        if (all_records ? path == 0 : path != 2) continue;
        const int32_t gi[3] = {rec.g[0][i], rec.g[1][i], rec.g[2][i]};
        const int32_t go[3] = {rec.g[3][i], rec.g[4][i], rec.g[5][i]};
        GlobalVisit v;
        v.vol = status_cls(stw) ? M : N;
        walk_all(gi, go, g.nx, g.ny, g.nz, v);
        ++taken;
    }
    const unsigned tk = warp_sum_u32(taken);
    if ((threadIdx.x & 31u) == 0 && tk && !all_records) atomicAdd(&ctrl->n_fallback, tk);
}

__global__ void classify_kernel(const float *__restrict__ w, int64_t n, float tau_l, float tau_h,
                                uint8_t *__restrict__ cls)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        const float x = w[i];
        cls[i] = x < tau_l ? 1 : (x > tau_h ? 2 : 0);
    }
}

}  // namespace

cudaError_t launch_ingest(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cordic,
                          float tau_l, float tau_h, int use_miss, int use_hit, const TilePlan &tp,
                          const Records &rec, Ctrl *ctrl, uint32_t *block_count,
                          uint32_t *block_pairs, uint32_t *stage, int on_host, int sm_count,
                          cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const ChunkSplit sp = chunk_split(n, sm_count);
    // without the tiled path's buffers every record takes the global path
    const bool tiled = tp.ntiles > 0 && block_count && block_pairs && stage;
    TilePlan tpl = tp;
    if (!tiled) tpl.ntiles = 0;
    const size_t smem = sizeof(uint32_t) * 2 * static_cast<size_t>(tpl.ntiles);
    uint32_t *bc = tiled ? block_count : nullptr;
    uint32_t *bp = tiled ? block_pairs : nullptr;
    uint32_t *sg = tiled ? stage : nullptr;
    const uintptr_t bits =
        reinterpret_cast<uintptr_t>(in.angle) | reinterpret_cast<uintptr_t>(in.u_in) |
        reinterpret_cast<uintptr_t>(in.v_in) | reinterpret_cast<uintptr_t>(in.u_out) |
        reinterpret_cast<uintptr_t>(in.v_out) | reinterpret_cast<uintptr_t>(in.wepl);
    if (on_host && (bits & 15u) == 0)
        ingest_kernel<true><<<static_cast<unsigned>(sp.blocks), kIngestThreads, smem, s>>>(
            in, n, sp.per_block, g, cordic, tau_l, tau_h, use_miss, use_hit, tpl, rec, ctrl, bc,
            bp, sg);
    else
        ingest_kernel<false><<<static_cast<unsigned>(sp.blocks), kIngestThreads, smem, s>>>(
            in, n, sp.per_block, g, cordic, tau_l, tau_h, use_miss, use_hit, tpl, rec, ctrl, bc,
            bp, sg);
    return cudaGetLastError();
}

cudaError_t launch_trace_global(const Records &rec, Ctrl *ctrl, int64_t upper, const GeomQ &g,
                                uint32_t *N, uint32_t *M, int all_records,
                                int sm_count, cudaStream_t s)
{
    if (upper <= 0) return cudaSuccess;
    int64_t blocks = (upper + 255) / 256;
    const int64_t cap_blocks = static_cast<int64_t>(sm_count) * 8;
    if (blocks > cap_blocks) blocks = cap_blocks;
    trace_global_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(rec, ctrl, g, N, M,
                                                                       all_records);
    return cudaGetLastError();
}

cudaError_t launch_classify(const float *wepl, int64_t n, float tau_l, float tau_h, uint8_t *cls,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    classify_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(wepl, n, tau_l, tau_h, cls);
    return cudaGetLastError();
}

}  // namespace hd
