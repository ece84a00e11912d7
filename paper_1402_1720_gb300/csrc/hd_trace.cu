// Ingest (classification + fixed-point geometry + compaction) and the voxel
// traversal that accumulates N, M and the SC carve.
//
// Classification: Eq. 3.1 (missed, WEPL below the cutoff) and Eq. 3.7 (hit,
// WEPL above the cutoff).  Path: the closed segment between entry and exit
// (Sec. 2.1), A_i of Eq. 3.2 read with d_0 = 0 against half-open voxel
// cubes.  Accumulation: N of Eq. 3.4 (Alg. 2), M of Eq. 3.9 (Alg. 3), the SC
// carve of Alg. 1.
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
#include <cmath>

#include "hd_internal.cuh"

namespace hd {

namespace {

// The geometry and traversal helpers are also compiled for the host so the
// same code can be exercised without a GPU.
#define HD_HD __host__ __device__ __forceinline__

HD_HD long long q16_of(float x)
{
#ifdef __CUDA_ARCH__
    return __double2ll_rn(static_cast<double>(x) * 65536.0);
#else
    return llrint(static_cast<double>(x) * 65536.0);
#endif
}

HD_HD long long floordiv_pos(long long a, long long b)
{
    long long q = a / b;
    if (a - q * b != 0 && a < 0) --q;
    return q;
}

// Rotation-mode CORDIC of an angle in degrees * 2^16: cos and sin * 2^30.
HD_HD void cordic_cs(long long a_q16, const Cordic &cd, long long &c,
                                          long long &s)
{
    const long long full = 360LL * kQ16, quarter = 90LL * kQ16;
    long long a = a_q16 % full;
    if (a < 0) a += full;
    const int k = static_cast<int>(a / quarter);
    const long long r = a - k * quarter;
    long long z = r << 14;
    long long x = cd.K, y = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const long long xs = x >> i, ys = y >> i;
        const long long th = cd.theta[i];
        if (z >= 0) {
            x -= ys;
            y += xs;
            z -= th;
        } else {
            x += ys;
            y -= xs;
            z += th;
        }
    }
    switch (k) {
    case 0: c = x; s = y; break;
    case 1: c = -y; s = x; break;
    case 2: c = -x; s = -y; break;
    default: c = y; s = -x; break;
    }
}

HD_HD long long to_grid(long long w, int n, long long s_q)
{
    return floordiv_pos((2 * w + static_cast<long long>(n) * s_q) * kQ16, 2 * s_q);
}

// Grid Q16 endpoints of one history; false when the history is rejected.
HD_HD bool endpoints(const GeomQ &g, const Cordic &cd, float ang, float ui,
                                          float vi, float uo, float vo, int32_t out[6])
{
    if (!(fabsf(ang) < 1048576.0f)) return false;
    if (!(fabsf(ui) < 4096.0f) || !(fabsf(vi) < 4096.0f) || !(fabsf(uo) < 4096.0f) ||
        !(fabsf(vo) < 4096.0f))
        return false;
    long long c, s;
    cordic_cs(q16_of(ang), cd, c, s);
    const long long T = g.T;
    const long long qui = q16_of(ui), qvi = q16_of(vi), quo = q16_of(uo), qvo = q16_of(vo);
    const long long wxi = (-T * c - qui * s) >> 30;
    const long long wyi = (-T * s + qui * c) >> 30;
    const long long wxo = (T * c - quo * s) >> 30;
    const long long wyo = (T * s + quo * c) >> 30;
    const long long G[6] = {to_grid(wxi, g.nx, g.sx), to_grid(wyi, g.ny, g.sy),
                            to_grid(qvi, g.nz, g.sz), to_grid(wxo, g.nx, g.sx),
                            to_grid(wyo, g.ny, g.sy), to_grid(qvo, g.nz, g.sz)};
    const long long lim = 1LL << 30;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (G[a] >= lim || G[a] <= -lim) return false;
        out[a] = static_cast<int32_t>(G[a]);
    }
    return true;
}

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
__device__ __forceinline__ int ingest_one(const GeomQ &g, const Cordic &cd, float tau_l,
                                          float tau_h, int use_miss, int use_hit, float ang,
                                          float ui, float vi, float uo, float vo, float w,
                                          int32_t rec[6], LaneAcc &acc)
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
    if (!endpoints(g, cd, ang, ui, vi, uo, vo, rec)) {
        acc.n_reject += 1;
        return 0;
    }
    return cls;
}

// Append up to 4 records per lane with one pair of atomics per warp.
__device__ __forceinline__ void append_records(const Records &rec, Ctrl *ctrl, const int cls[4],
                                               const int32_t r[4][6])
{
    const unsigned lane = threadIdx.x & 31u;
    unsigned mine = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) mine += (cls[k] == 1) ? 1u : (cls[k] == 2 ? 65536u : 0u);
    // inclusive scan of packed (miss | hit << 16) counts
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= static_cast<unsigned>(o)) incl += t;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned base_m = 0, base_h = 0;
    if (lane == 31) {
        if (total & 0xffffu) base_m = atomicAdd(&ctrl->rec_miss, total & 0xffffu);
        if (total >> 16) base_h = atomicAdd(&ctrl->rec_hit, total >> 16);
    }
    base_m = __shfl_sync(0xffffffffu, base_m, 31);
    base_h = __shfl_sync(0xffffffffu, base_h, 31);
    const unsigned excl = incl - mine;
    unsigned pm = base_m + (excl & 0xffffu);
    unsigned ph = base_h + (excl >> 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (cls[k] == 0) continue;
        int64_t slot;
        if (cls[k] == 1) {
            slot = pm++;
        } else {
            slot = rec.cap - 1 - static_cast<int64_t>(ph++);
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) rec.g[a][slot] = r[k][a];
    }
}

template <bool kVec>
__global__ void __launch_bounds__(256) ingest_kernel(Inputs in, int64_t n, GeomQ g, Cordic cd,
                                                     float tau_l, float tau_h, int use_miss,
                                                     int use_hit, Records rec, Ctrl *ctrl)
{
    LaneAcc acc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    // every lane of a warp runs the same number of iterations (warp-wide
    // appends), so the loop bound is rounded up to a multiple of the stride
    const int64_t units = kVec ? (n + 3) / 4 : n;
    const int64_t iters = (units + stride - 1) / stride;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t u = tid + it * stride;
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
                                    UO.x, VO.x, W.x, r[0], acc);
                cls[1] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.y, UI.y, VI.y,
                                    UO.y, VO.y, W.y, r[1], acc);
                cls[2] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.z, UI.z, VI.z,
                                    UO.z, VO.z, W.z, r[2], acc);
                cls[3] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, A.w, UI.w, VI.w,
                                    UO.w, VO.w, W.w, r[3], acc);
            } else {
                for (int k = 0; k < 4; ++k) {
                    const int64_t i = i0 + k;
                    if (i < n)
                        cls[k] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit,
                                            in.angle[i], in.u_in[i], in.v_in[i], in.u_out[i],
                                            in.v_out[i], in.wepl[i], r[k], acc);
                }
            }
        } else if (u < n) {
            cls[0] = ingest_one(g, cd, tau_l, tau_h, use_miss, use_hit, in.angle[u], in.u_in[u],
                                in.v_in[u], in.u_out[u], in.v_out[u], in.wepl[u], r[0], acc);
        }
        append_records(rec, ctrl, cls, r);
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
}

// ---------------------------------------------------------------- traversal

// Voxel update of one history: count (atomic add) or SC carve (clear bit).
struct Visit {
    uint32_t *vol;   // N or M (count mode)
    uint32_t *bits;  // carve mask (carve mode, vol == nullptr)
    __device__ __forceinline__ void operator()(uint32_t v) const
    {
        if (vol != nullptr) {
            atomicAdd(vol + v, 1u);
        } else {
            const uint32_t w = v >> 5, b = 1u << (v & 31u);
            if (__ldcg(bits + w) & b) atomicAnd(bits + w, ~b);
        }
    }
};

// Walk A_i of the segment gi -> go, calling visit(v) once per voxel of the
// set in traversal order; returns |A_i|.
template <class VisitT>
HD_HD unsigned walk(const int32_t gi[3], const int32_t go[3], int nx, int ny, int nz,
                    const VisitT &visit)
{
    const long long hx = static_cast<long long>(nx) << 16, hy = static_cast<long long>(ny) << 16,
                    hz = static_cast<long long>(nz) << 16;
    const long long dx = static_cast<long long>(go[0]) - gi[0];
    const long long dy = static_cast<long long>(go[1]) - gi[1];
    const long long dz = static_cast<long long>(go[2]) - gi[2];
    const long long x0 = gi[0], y0 = gi[1], z0 = gi[2];

    // parameter t_enter = tN / tQ at which the segment enters the grid box
    long long tN = 0, tQ = 1;
    auto entry = [&](long long p0, long long d, long long hi) -> bool {
        long long cN = -1, cQ = 1;
        if (d > 0) {
            if (p0 >= hi) return false;
            if (p0 < 0) { cN = -p0; cQ = d; }
        } else if (d < 0) {
            if (p0 < 0) return false;
            if (p0 >= hi) { cN = p0 - hi; cQ = -d; }
        } else if (p0 < 0 || p0 >= hi) {
            return false;
        }
        if (cN >= 0 && cN * tQ > tN * cQ) { tN = cN; tQ = cQ; }
        return true;
    };
    if (!entry(x0, dx, hx) || !entry(y0, dy, hy) || !entry(z0, dz, hz)) return 0;
    if (tN > tQ) return 0;

    int ix, iy, iz;
    if (tN == 0) {
        ix = static_cast<int>(x0 >> 16);
        iy = static_cast<int>(y0 >> 16);
        iz = static_cast<int>(z0 >> 16);
    } else {
        const long long den = tQ << 16;
        ix = static_cast<int>(floordiv_pos(x0 * tQ + tN * dx, den));
        iy = static_cast<int>(floordiv_pos(y0 * tQ + tN * dy, den));
        iz = static_cast<int>(floordiv_pos(z0 * tQ + tN * dz, den));
    }
    if ((dx > 0 && ix >= nx) || (dx < 0 && ix < 0)) return 0;
    if ((dy > 0 && iy >= ny) || (dy < 0 && iy < 0)) return 0;
    if ((dz > 0 && iz >= nz) || (dz < 0 && iz < 0)) return 0;

    // per-axis: |D|, next-crossing numerator, remaining valid steps
    long long ax, ay, az, nmx, nmy, nmz;
    int kx, ky, kz;
    {
        const int fx = go[0] >> 16, fy = go[1] >> 16, fz = go[2] >> 16;
        if (dx > 0) { ax = dx; nmx = ((static_cast<long long>(ix) + 1) << 16) - x0; kx = (fx < nx - 1 ? fx : nx - 1) - ix; }
        else if (dx < 0) { ax = -dx; nmx = x0 - (static_cast<long long>(ix) << 16); kx = ix - (fx > 0 ? fx : 0); }
        else { ax = 0; nmx = 1; kx = 0; }
        if (dy > 0) { ay = dy; nmy = ((static_cast<long long>(iy) + 1) << 16) - y0; ky = (fy < ny - 1 ? fy : ny - 1) - iy; }
        else if (dy < 0) { ay = -dy; nmy = y0 - (static_cast<long long>(iy) << 16); ky = iy - (fy > 0 ? fy : 0); }
        else { ay = 0; nmy = 1; ky = 0; }
        if (dz > 0) { az = dz; nmz = ((static_cast<long long>(iz) + 1) << 16) - z0; kz = (fz < nz - 1 ? fz : nz - 1) - iz; }
        else if (dz < 0) { az = -dz; nmz = z0 - (static_cast<long long>(iz) << 16); kz = iz - (fz > 0 ? fz : 0); }
        else { az = 0; nmz = 1; kz = 0; }
    }
    long long exy = nmx * ay - nmy * ax;
    long long exz = nmx * az - nmz * ax;
    long long eyz = nmy * az - nmz * ay;
    const long long ax16 = ax << 16, ay16 = ay << 16, az16 = az << 16;
    const int sx = dx > 0 ? 1 : -1, sy = dy > 0 ? 1 : -1, sz = dz > 0 ? 1 : -1;
    const int stx = sx, sty = sy * nx, stz = sz * nx * ny;

    int idx = ix + nx * (iy + ny * iz);
    bool inside = (ix < nx) && (iy < ny) && (iz < nz);
    unsigned count = 0;
    if (inside) {
        visit(static_cast<uint32_t>(idx));
        ++count;
    }
    // a single point (entry = exit) has no crossings; otherwise at least one
    // axis moves, and the earliest crossing always belongs to a moving axis,
    // so every pass of the loop below steps or stops
    if ((ax | ay | az) == 0) return count;

    for (;;) {
        int first;
        if (exy < 0) first = exz < 0 ? 0 : (exz > 0 ? 2 : -1);
        else if (exy > 0) first = eyz < 0 ? 1 : (eyz > 0 ? 2 : -1);
        else first = -1;
        if (first == 0) {
            if (kx == 0) break;
            --kx; ix += sx; idx += stx; exy += ay16; exz += az16;
        } else if (first == 1) {
            if (ky == 0) break;
            --ky; iy += sy; idx += sty; exy -= ax16; eyz += az16;
        } else if (first == 2) {
            if (kz == 0) break;
            --kz; iz += sz; idx += stz; exz -= ax16; eyz -= ay16;
        } else {
            // several axes cross at the same parameter
            const bool inx = ax != 0 && exy <= 0 && exz <= 0;
            const bool iny = ay != 0 && exy >= 0 && eyz <= 0;
            const bool inz = az != 0 && exz >= 0 && eyz >= 0;
            const bool px = inx && dx > 0, py = iny && dy > 0, pz = inz && dz > 0;
            const bool mx = inx && dx < 0, my = iny && dy < 0, mz = inz && dz < 0;
            if ((px && kx == 0) || (py && ky == 0) || (pz && kz == 0)) break;
            if (px || py || pz) {
                if (px) { --kx; ix += sx; idx += stx; exy += ay16; exz += az16; }
                if (py) { --ky; iy += sy; idx += sty; exy -= ax16; eyz += az16; }
                if (pz) { --kz; iz += sz; idx += stz; exz -= ax16; eyz -= ay16; }
                if (!inside) inside = (ix < nx) && (iy < ny) && (iz < nz);
                if (inside) { visit(static_cast<uint32_t>(idx)); ++count; }
            }
            if (mx || my || mz) {
                if ((mx && kx == 0) || (my && ky == 0) || (mz && kz == 0)) break;
                if (mx) { --kx; ix += sx; idx += stx; exy += ay16; exz += az16; }
                if (my) { --ky; iy += sy; idx += sty; exy -= ax16; eyz += az16; }
                if (mz) { --kz; iz += sz; idx += stz; exz -= ax16; eyz -= ay16; }
                if (!inside) inside = (ix < nx) && (iy < ny) && (iz < nz);
                if (inside) { visit(static_cast<uint32_t>(idx)); ++count; }
            }
            continue;
        }
        if (!inside) inside = (ix < nx) && (iy < ny) && (iz < nz);
        if (inside) {
            visit(static_cast<uint32_t>(idx));
            ++count;
        }
    }
    return count;
}

__global__ void __launch_bounds__(256) trace_kernel(Records rec, const Ctrl *cc, Ctrl *stats,
                                                    GeomQ g, uint32_t *N, uint32_t *M,
                                                    uint32_t *carve)
{
    const unsigned nm = cc->rec_miss, nh = cc->rec_hit;
    const int64_t total = static_cast<int64_t>(nm) + nh;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned steps_m = 0, steps_h = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += stride) {
        const bool miss = i < nm;
        const int64_t slot = miss ? i : rec.cap - 1 - (i - nm);
        const int32_t gi[3] = {rec.g[0][slot], rec.g[1][slot], rec.g[2][slot]};
        const int32_t go[3] = {rec.g[3][slot], rec.g[4][slot], rec.g[5][slot]};
        Visit v;
        v.vol = miss ? N : M;
        v.bits = carve;
        const unsigned c = walk(gi, go, g.nx, g.ny, g.nz, v);
        if (miss) steps_m += c; else steps_h += c;
    }
    const unsigned sm_ = warp_sum_u32(steps_m), sh_ = warp_sum_u32(steps_h);
    if ((threadIdx.x & 31u) == 0) {
        if (sm_) atomicAdd(&stats->steps_miss, static_cast<unsigned long long>(sm_));
        if (sh_) atomicAdd(&stats->steps_hit, static_cast<unsigned long long>(sh_));
    }
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
                          float tau_l, float tau_h, int use_miss, int use_hit,
                          const Records &rec, Ctrl *ctrl, int sm_count, cudaStream_t s)
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
    if (vec)
        ingest_kernel<true><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
            in, n, g, cordic, tau_l, tau_h, use_miss, use_hit, rec, ctrl);
    else
        ingest_kernel<false><<<static_cast<unsigned>(blocks), 256, 0, s>>>(
            in, n, g, cordic, tau_l, tau_h, use_miss, use_hit, rec, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_trace(const Records &rec, const Ctrl *ctrl_counts, Ctrl *ctrl_stats,
                         int64_t miss_upper, int64_t hit_upper, const GeomQ &g, uint32_t *N,
                         uint32_t *M, uint32_t *carve, int sm_count, cudaStream_t s)
{
    const int64_t total = miss_upper + hit_upper;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap_blocks = static_cast<int64_t>(sm_count) * 8;
    if (blocks > cap_blocks) blocks = cap_blocks;
    trace_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(rec, ctrl_counts, ctrl_stats, g, N,
                                                                M, carve);
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
