// Ingest (classification + fixed-point geometry + compaction) and the voxel
// traversal that accumulates N and M.
//
// Classification: Eq. 3.1 (missed, WEPL below the cutoff) and Eq. 3.7 (hit,
// WEPL above the cutoff).  Path: the closed segment between entry and exit
// (Sec. 2.1), A_i of Eq. 3.2 read with d_0 = 0 against half-open voxel
// cubes.  Accumulation: N of Eq. 3.4 (Alg. 2; SC's H_1 = [N = 0] of Eq. 3.3
// is the carve of Alg. 1 as a set difference), M of Eq. 3.9 (Alg. 3).
//
// The traversal is an exact integer DDA.  For the segment
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

// Per-block staging of the appends: each warp's pair demand and record
// counts, and the block's bases (two sets, alternating by iteration, so that
// a warp starting the next iteration never overwrites what a slower warp of
// this one still reads).
constexpr int kIngestWarps = 8;  // 256-thread blocks
struct AppendStage {
    unsigned pairs[2][kIngestWarps];
    unsigned recs[2][kIngestWarps];  // missed + 65536 hit
    unsigned base_pairs[2], base_miss[2], base_hit[2];
};

// Decide tiled / global path for up to 4 records per lane, count tiles in
// the block histogram, and append the records.  The pair budget and the two
// record counters are reserved once per block and iteration (all threads
// call this together): same-address atomics on the three counters are what
// limit a warp-per-reservation scheme.
__device__ __forceinline__ void admit_and_append(const TilePlan &tp, const Records &rec,
                                                 Ctrl *ctrl, uint32_t *s_hist, int cls[4],
                                                 const int32_t r[4][6], AppendStage &st, int par)
{
    const unsigned lane = threadIdx.x & 31u;
    int tcount[4];
    int zr[4];  // the record's slices, zlo + 4096 zhi (computed once here)
    unsigned demand = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        tcount[k] = 0;
        zr[k] = 0;
        if (cls[k] == 0) continue;
        int lo[3], hi[3], zlo, zhi;
        const int c = grid_z_range(tp, r[k], zlo, zhi) ? tile_range_z(tp, r[k], zlo, zhi, lo, hi) : 0;
        if (c == 0) {
            cls[k] = 0;  // no voxel of the grid: nothing to traverse
            continue;
        }
        zr[k] = zlo + 4096 * zhi;
        tcount[k] = (tp.ntiles > 0 && c <= tp.max_tiles) ? c : -1;
        if (tcount[k] > 0) demand += static_cast<unsigned>(c);
    }
    // records this lane appends: missed + 65536 hit (a record kept here
    // keeps its class whatever path it takes)
    unsigned mine = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) mine += (cls[k] == 1) ? 1u : (cls[k] == 2 ? 65536u : 0u);
    const unsigned warp = threadIdx.x >> 5;
    const unsigned incl = warp_incl_scan(demand);
    const unsigned inc2 = warp_incl_scan(mine);
    if (lane == 31) {
        st.pairs[par][warp] = incl;
        st.recs[par][warp] = inc2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tp_ = 0, tr = 0;
        for (int w = 0; w < kIngestWarps; ++w) {
            tp_ += st.pairs[par][w];
            tr += st.recs[par][w];
        }
        st.base_pairs[par] = tp_ ? atomicAdd(&ctrl->pairs_used, tp_) : 0u;
        st.base_miss[par] = (tr & 0xffffu) ? atomicAdd(&ctrl->rec_miss, tr & 0xffffu) : 0u;
        st.base_hit[par] = (tr >> 16) ? atomicAdd(&ctrl->rec_hit, tr >> 16) : 0u;
    }
    __syncthreads();
    unsigned wp = 0, wr = 0;  // earlier warps' pairs and records
    for (unsigned w = 0; w < warp; ++w) {
        wp += st.pairs[par][w];
        wr += st.recs[par][w];
    }
    const unsigned base = st.base_pairs[par] + wp;
    unsigned long long end = static_cast<unsigned long long>(base) + (incl - demand);
    int status[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        status[k] = 2;
        if (tcount[k] > 0) {
            end += static_cast<unsigned>(tcount[k]);
            if (end <= static_cast<unsigned long long>(tp.pair_cap)) status[k] = 1;
        }
        if (cls[k] != 0 && status[k] == 1) {
            int lo[3], hi[3];
            tile_range_z(tp, r[k], zr[k] & 4095, zr[k] >> 12, lo, hi);
            const int off = (cls[k] - 1) * tp.ntiles;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x)
                        atomicAdd(&s_hist[off + x + tp.ntx * (y + tp.nty * z)], 1u);
        }
    }
    // append at the block's bases plus the earlier warps' and lanes' records
    if (mine == 0) return;
    const unsigned excl = inc2 - mine;
    unsigned pm = st.base_miss[par] + (wr & 0xffffu) + (excl & 0xffffu);
    unsigned ph = st.base_hit[par] + (wr >> 16) + (excl >> 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (cls[k] == 0) continue;
        const int64_t slot =
            cls[k] == 1 ? static_cast<int64_t>(pm++) : rec.cap - 1 - static_cast<int64_t>(ph++);
#pragma unroll
        for (int a = 0; a < 6; ++a) rec.g[a][slot] = r[k][a];
        rec.status[slot] = record_status(status[k], zr[k] & 4095, zr[k] >> 12);
    }
}

template <bool kVec>
__global__ void __launch_bounds__(256, 4) ingest_kernel(Inputs in, int64_t n, GeomQ g, Cordic cd,
                                                     float tau_l, float tau_h, int use_miss,
                                                     int use_hit, TilePlan tp, Records rec,
                                                     Ctrl *ctrl, uint32_t *tile_count)
{
    extern __shared__ uint32_t s_hist[];  // 2 * ntiles counters
    __shared__ AppendStage s_stage;
    const int nh = 2 * tp.ntiles;
    for (int t = threadIdx.x; t < nh; t += blockDim.x) s_hist[t] = 0;
    __syncthreads();
    LaneAcc acc;
    TrigCache tc;
    // each block takes a contiguous range of units (histories arrive grouped
    // by gantry angle, so a thread's angle, and its cos/sin, rarely change),
    // in coalesced steps of one unit per thread; every thread of a block runs
    // the same number of steps (block-wide appends and histogram flush)
    const int64_t units = kVec ? (n + 3) / 4 : n;
    const int64_t per_block = (units + gridDim.x - 1) / gridDim.x;
    const int64_t u0 = static_cast<int64_t>(blockIdx.x) * per_block;
    const int64_t u1 = u0 + per_block < units ? u0 + per_block : units;
    const int64_t iters = (per_block + blockDim.x - 1) / blockDim.x;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t uu = u0 + it * blockDim.x + threadIdx.x;
        const int64_t u = uu < u1 ? uu : units;  // past the block's range: no history
        int cls[4] = {0, 0, 0, 0};
        int32_t r[4][6];
        if (kVec) {
            const int64_t i0 = u * 4;
            if (i0 + 3 < n) {
                const float4 A = __ldg(reinterpret_cast<const float4 *>(in.angle) + u);
                const float4 UI = __ldg(reinterpret_cast<const float4 *>(in.u_in) + u);
                const float4 VI = __ldg(reinterpret_cast<const float4 *>(in.v_in) + u);
                const float4 UO = __ldg(reinterpret_cast<const float4 *>(in.u_out) + u);
                const float4 VO = __ldg(reinterpret_cast<const float4 *>(in.v_out) + u);
                const float4 W = __ldg(reinterpret_cast<const float4 *>(in.wepl) + u);
                cls[0] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.x, UI.x, VI.x,
                                    UO.x, VO.x, W.x, r[0], acc, tc);
                cls[1] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.y, UI.y, VI.y,
                                    UO.y, VO.y, W.y, r[1], acc, tc);
                cls[2] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.z, UI.z, VI.z,
                                    UO.z, VO.z, W.z, r[2], acc, tc);
                cls[3] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.w, UI.w, VI.w,
                                    UO.w, VO.w, W.w, r[3], acc, tc);
            } else {
                for (int k = 0; k < 4; ++k) {
                    const int64_t i = i0 + k;
                    if (i < n)
                        cls[k] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit,
                                            in.angle[i], in.u_in[i], in.v_in[i], in.u_out[i],
                                            in.v_out[i], in.wepl[i], r[k], acc, tc);
                }
            }
        } else if (u < n) {
            cls[0] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, in.angle[u], in.u_in[u],
                                in.v_in[u], in.u_out[u], in.v_out[u], in.wepl[u], r[0], acc, tc);
        }
        admit_and_append(tp, rec, ctrl, s_hist, cls, r, s_stage, static_cast<int>(it & 1));
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
    __syncthreads();
    for (int t = threadIdx.x; t < nh; t += blockDim.x)
        if (s_hist[t]) atomicAdd(&tile_count[t], s_hist[t]);
}

// ---------------------------------------------------------------- traversal

__global__ void __launch_bounds__(256) trace_global_kernel(Records rec, Ctrl *ctrl, GeomQ g,
                                                           uint32_t *N, uint32_t *M,
                                                           int all_records)
{
    const unsigned nm = ctrl->rec_miss, nh = ctrl->rec_hit;
    const int64_t total = static_cast<int64_t>(nm) + nh;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned taken = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += stride) {
        const bool miss = i < nm;
        const int64_t slot = miss ? i : rec.cap - 1 - (i - nm);
        if (!all_records && status_path(rec.status[slot]) != 2) continue;
        const int32_t gi[3] = {rec.g[0][slot], rec.g[1][slot], rec.g[2][slot]};
        const int32_t go[3] = {rec.g[3][slot], rec.g[4][slot], rec.g[5][slot]};
        GlobalVisit v;
        v.vol = miss ? N : M;
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
                          const Records &rec, Ctrl *ctrl, uint32_t *tile_count, int sm_count,
                          cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(in.angle) | reinterpret_cast<uintptr_t>(in.u_in) |
                       reinterpret_cast<uintptr_t>(in.v_in) | reinterpret_cast<uintptr_t>(in.u_out) |
                       reinterpret_cast<uintptr_t>(in.v_out) | reinterpret_cast<uintptr_t>(in.wepl)) &
                      15u) == 0;
    const int64_t units = vec ? (n + 3) / 4 : n;
    int64_t blocks = (units + 255) / 256;
    const int64_t cap_blocks = static_cast<int64_t>(sm_count) * 8;
    if (blocks > cap_blocks) blocks = cap_blocks;
    if (blocks < 1) blocks = 1;
    const size_t smem = sizeof(uint32_t) * 2 * static_cast<size_t>(tp.ntiles);
    if (vec)
        ingest_kernel<true><<<static_cast<unsigned>(blocks), 256, smem, s>>>(
            in, n, g, cordic, tau_l, tau_h, use_miss, use_hit, tp, rec, ctrl, tile_count);
    else
        ingest_kernel<false><<<static_cast<unsigned>(blocks), 256, smem, s>>>(
            in, n, g, cordic, tau_l, tau_h, use_miss, use_hit, tp, rec, ctrl, tile_count);
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
