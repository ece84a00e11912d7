// Thick rays by the Euclidean distance of Eq. 3.2 (d_0 > 0, d the distance
// from a voxel's centre to the closed segment L_i, Sec. 2.1): A_i(d_0) = the
// voxels whose centre lies within d_0 mm of L_i.  Counted into N and M like
// the thin paths, once per history for every voxel of its A_i(d_0).
//
// Exactness.  Coordinates are doubled world mm * 2^16 (the fixed-point
// frame of the thin paths, doubled so that voxel centres (2 i + 1 - n) s / 2
// are integers): A, B the doubled entry and exit points, R = 2 q16(d_0).
// They stay below 2^30 in magnitude, so with u = B - A and w = C - A every
// component fits 32 bits, products 64 bits, and the squared distance times
// |u|^2 fits unsigned 128 bits:
//   F = |w|^2 |u|^2        when w.u <= 0      (nearest point A)
//   F = |C - B|^2 |u|^2    when w.u >= |u|^2  (nearest point B)
//   F = |w x u|^2          otherwise          (the line between them)
// and C is in the set iff F <= R^2 |u|^2 (for A = B: F = |w|^2 <= R^2).
//
// Work.  A warp takes one history at a time (histories handed out in runs
// of consecutive ones, so the gantry cos/sin rarely change); its lanes take
// the rows of voxels along the segment's major in-plane axis that cross the
// box bounding the capsule (segment grown by d_0).  Along a row the squared
// distance is convex, so the row's part of the set is one interval: a float
// estimate of the capsule's cross-section gives starting indices, and exact
// evaluations of F settle both ends (a boundary i with i inside and the
// neighbour outside), or, when the estimate finds no voxel, an exact descent
// to F's minimum along the row decides whether the row has any.  The float
// arithmetic only chooses where the exact tests start, never a result.  Each
// nonempty row adds +1 / -1 to a difference array along the major axis (the
// thick rays' workspace), and row prefix sums add them to N and M.
#include <cmath>
#include <cstdint>

#include "hd_geom.cuh"
#include "hd_thick.cuh"

namespace hd {
namespace {

constexpr int kEuThreads = 256;
constexpr int kEuRunHistories = 16;  // consecutive histories a warp takes at once

typedef unsigned __int128 u128;

// Full product of two 64-bit unsigned values (two multiplies, not a
// general 128 x 128 one).
__device__ __forceinline__ u128 mul64(unsigned long long a, unsigned long long b)
{
    return (static_cast<u128>(__umul64hi(a, b)) << 64) | static_cast<u128>(a * b);
}

__device__ __forceinline__ u128 sq64(long long a)
{
    const unsigned long long m = static_cast<unsigned long long>(a < 0 ? -a : a);
    return mul64(m, m);
}

// One history's capsule in the permuted frame (axis 0 the major in-plane
// axis, 1 the other in-plane axis, 2 z), exact and in float mm.
struct Capsule {
    long long A[3], B[3], u[3];
    unsigned long long uu;  // |u|^2 (< 3 2^62)
    u128 T;                 // the threshold R^2 |u|^2 (or R^2 when u = 0)
    unsigned long long RR;  // R^2
    unsigned long long uu2; // u_1^2 + u_2^2: the segment projected along axis 0
    u128 T2;                // R^2 uu2
    float Af[3], df[3], L2f, Rf;
    float inv_L2, inv_d0, inv_s0;  // 1 / L2f, 1 / df[0], 1 / sf[0] (estimates only)
    int n[3];
    long long s2[3];  // voxel sizes, mm * 2^16 (centres are (2 i + 1 - n) s2)
    float sf[3];      // voxel sizes, mm
};

// The constants of one row (fixed indices a on axis 1 and k on axis 2).
struct Row {
    long long wc, wz, wbc, wbz;  // C - A and C - B on axes 1 and 2
    __int128 dot0;               // (C - A).u restricted to axes 1, 2
    unsigned long long hA, hB;   // |C - A|^2, |C - B|^2 restricted to axes 1, 2
    long long k0;                // cross component without the major axis
};

__device__ __forceinline__ Row row_of(const Capsule &cp, int a, int k)
{
    Row r;
    const long long cc = (2LL * a + 1 - cp.n[1]) * cp.s2[1];
    const long long cz = (2LL * k + 1 - cp.n[2]) * cp.s2[2];
    r.wc = cc - cp.A[1];
    r.wz = cz - cp.A[2];
    r.wbc = cc - cp.B[1];
    r.wbz = cz - cp.B[2];
    r.dot0 = static_cast<__int128>(r.wc) * cp.u[1] + static_cast<__int128>(r.wz) * cp.u[2];
    r.hA = static_cast<unsigned long long>(r.wc * r.wc) + static_cast<unsigned long long>(r.wz * r.wz);
    r.hB = static_cast<unsigned long long>(r.wbc * r.wbc) +
           static_cast<unsigned long long>(r.wbz * r.wbz);
    r.k0 = r.wc * cp.u[2] - r.wz * cp.u[1];
    return r;
}

// F at index i of the row (see the file comment).  Out of line: one copy of
// the 128-bit arithmetic serves every test of the row search (inlined at
// each of them, the kernel's code outgrew the instruction cache: 35 % slower).
__device__ __noinline__ u128 F_at(const Capsule &cp, const Row &r, int i)
{
    const long long cm = (2LL * i + 1 - cp.n[0]) * cp.s2[0];
    const long long wm = cm - cp.A[0];
    if (cp.uu == 0) return static_cast<u128>(static_cast<unsigned long long>(wm * wm) + r.hA);
    const __int128 dot = r.dot0 + static_cast<__int128>(wm) * cp.u[0];
    if (dot <= 0) return mul64(static_cast<unsigned long long>(wm * wm) + r.hA, cp.uu);
    if (dot >= static_cast<__int128>(cp.uu)) {
        const long long wbm = cm - cp.B[0];
        return mul64(static_cast<unsigned long long>(wbm * wbm) + r.hB, cp.uu);
    }
    const long long k1 = r.wz * cp.u[0] - wm * cp.u[2];
    const long long k2 = wm * cp.u[1] - r.wc * cp.u[0];
    return sq64(r.k0) + sq64(k1) + sq64(k2);
}

__device__ __forceinline__ bool in_at(const Capsule &cp, const Row &r, int i)
{
    return F_at(cp, r, i) <= cp.T;
}

// Does the row meet the capsule at all?  The row is a line along axis 0, so
// it does iff its point in the plane of axes 1 and 2 lies within R of the
// segment's projection onto that plane (the projection of the capsule is the
// disc-swept projected segment): the same three cases in two dimensions,
// with the row's constants (dot0 and k0 are that plane's dot and cross).
__device__ __forceinline__ bool row_meets(const Capsule &cp, const Row &r)
{
    if (cp.uu2 == 0 || r.dot0 <= 0) return r.hA <= cp.RR;
    if (r.dot0 >= static_cast<__int128>(cp.uu2)) return r.hB <= cp.RR;
    return sq64(r.k0) <= cp.T2;
}

// Float estimate of the row's cross-section of the capsule, as a range of
// major indices (lo > hi when the estimate finds none); also a float guess
// of where along the row the distance is smallest.
__device__ __forceinline__ void estimate(const Capsule &cp, int a, int k, int &ilo, int &ihi,
                                         int &imin)
{
    // approximate arithmetic throughout (fast square roots and quotients):
    // these numbers only choose where the exact tests start
    const float cc = 0.5f * static_cast<float>(2 * a + 1 - cp.n[1]) * cp.sf[1];
    const float cz = 0.5f * static_cast<float>(2 * k + 1 - cp.n[2]) * cp.sf[2];
    const float wc = cc - cp.Af[1], wz = cz - cp.Af[2];
    const float R2 = cp.Rf * cp.Rf;
    float lo = INFINITY, hi = -INFINITY;
    // the caps: balls around A and B
    const float hA = wc * wc + wz * wz;
    if (hA <= R2) {
        const float s = __fsqrt_rz(R2 - hA);
        lo = fminf(lo, -s);
        hi = fmaxf(hi, s);
    }
    const float bc = wc - cp.df[1], bz = wz - cp.df[2];
    const float hB = bc * bc + bz * bz;
    if (hB <= R2) {
        const float s = __fsqrt_rz(R2 - hB);
        lo = fminf(lo, cp.df[0] - s);
        hi = fmaxf(hi, cp.df[0] + s);
    }
    // sigma = (major coordinate) - A_0 of the point nearest the segment's line
    float smin = 0.0f;
    if (cp.L2f > 0.0f) {
        const float g = wc * cp.df[1] + wz * cp.df[2];
        const float a2 = 1.0f - cp.df[0] * cp.df[0] * cp.inv_L2;
        const float b = -cp.df[0] * g * cp.inv_L2;
        const float c0 = hA - g * g * cp.inv_L2;
        // the parameter along the segment stays in [0, 1]
        float tlo = -INFINITY, thi = INFINITY;
        if (cp.df[0] != 0.0f) {
            const float t0 = -g * cp.inv_d0, t1 = (cp.L2f - g) * cp.inv_d0;
            tlo = fminf(t0, t1);
            thi = fmaxf(t0, t1);
        } else if (g < 0.0f || g > cp.L2f) {
            tlo = INFINITY;  // the row never faces the segment's interior
        }
        if (a2 > 1e-6f) {
            const float ia = __frcp_rz(a2);
            smin = -b * ia;
            const float disc = b * b - a2 * (c0 - R2);
            if (disc >= 0.0f) {
                const float q = __fsqrt_rz(disc);
                const float s1 = fmaxf((-b - q) * ia, tlo), s2 = fminf((-b + q) * ia, thi);
                if (s1 <= s2) {
                    lo = fminf(lo, s1);
                    hi = fmaxf(hi, s2);
                }
            }
        } else {
            smin = 0.5f * cp.df[0];
            if (c0 <= R2 && tlo <= thi) {
                lo = fminf(lo, tlo);
                hi = fmaxf(hi, thi);
            }
        }
        smin = fminf(fmaxf(smin, fminf(0.0f, cp.df[0])), fmaxf(0.0f, cp.df[0]));
    }
    // index of a major coordinate x: x = (2 i + 1 - n) s / 2
    const float off = 0.5f * static_cast<float>(cp.n[0] - 1);
    const float inv = cp.inv_s0;
    const float flo = (lo + cp.Af[0]) * inv + off, fhi = (hi + cp.Af[0]) * inv + off;
    const float fm = (smin + cp.Af[0]) * inv + off;
    const float top = static_cast<float>(cp.n[0] - 1);
    ilo = static_cast<int>(ceilf(fminf(fmaxf(flo, -1.0f), top + 1.0f)));
    ihi = static_cast<int>(floorf(fminf(fmaxf(fhi, -1.0f), top + 1.0f)));
    if (!(lo <= hi)) {
        ilo = 1;
        ihi = 0;
    }
    imin = static_cast<int>(rintf(fminf(fmaxf(fm, 0.0f), top)));
}

// The exact interval [lo, hi] of voxels of a row whose line meets the
// capsule (false when no voxel centre of the row lies inside: the row's
// chord can fall between two centres).
__device__ __forceinline__ bool row_interval(const Capsule &cp, int a, int k, int &lo, int &hi)
{
    const int n = cp.n[0];
    const Row r = row_of(cp, a, k);
    int elo, ehi, emin;
    estimate(cp, a, k, elo, ehi, emin);
    elo = max(0, min(elo, n - 1));
    ehi = max(0, min(ehi, n - 1));
    int m = -1;
    if (elo <= ehi) {
        // the usual case: both estimated ends inside, their outer
        // neighbours outside (convexity: exactly [elo, ehi]); otherwise
        // settle the ends below from an inside point
        const bool in_lo = in_at(cp, r, elo);
        const bool in_hi = in_lo && (ehi == elo || in_at(cp, r, ehi));
        if (in_hi) {
            if ((elo == 0 || !in_at(cp, r, elo - 1)) && (ehi + 1 >= n || !in_at(cp, r, ehi + 1))) {
                lo = elo;
                hi = ehi;
                return true;
            }
            m = elo;
        } else if (in_lo) {
            m = elo;
        } else {
            const int mid = (elo + ehi) >> 1;
            if (in_at(cp, r, mid)) m = mid;
            else emin = mid;
        }
    }
    if (m < 0) {
        // exact descent to F's minimum along the row (F is convex in i)
        int i = emin;
        u128 f = F_at(cp, r, i);
        if (i > 0 && F_at(cp, r, i - 1) < f) {
            for (--i, f = F_at(cp, r, i); i > 0;) {
                const u128 g = F_at(cp, r, i - 1);
                if (!(g < f)) break;
                --i;
                f = g;
            }
        } else {
            for (; i + 1 < n;) {
                const u128 g = F_at(cp, r, i + 1);
                if (!(g < f)) break;
                ++i;
                f = g;
            }
        }
        if (f > cp.T) return false;  // no voxel centre of the row is inside
        m = i;
        elo = ehi = i;
    }
    // both ends, starting from the estimates (in_at(m) holds)
    lo = min(max(elo, 0), m);
    if (in_at(cp, r, lo)) {
        while (lo > 0 && in_at(cp, r, lo - 1)) --lo;
    } else {
        do ++lo;
        while (!in_at(cp, r, lo));
    }
    hi = max(min(ehi, n - 1), m);
    if (in_at(cp, r, hi)) {
        while (hi + 1 < n && in_at(cp, r, hi + 1)) ++hi;
    } else {
        do --hi;
        while (!in_at(cp, r, hi));
    }
    return true;
}

struct EuCounts {
    unsigned n_in = 0, n_miss = 0, n_hit = 0, n_none = 0, n_reject = 0;
};

__global__ void __launch_bounds__(kEuThreads, 3) euclid_kernel(Inputs in, int64_t n, GeomQ g,
                                                            Cordic cd, float tau_l, float tau_h,
                                                            int use_miss, int use_hit,
                                                            long long R2, float d0, ThickDiff td,
                                                            unsigned long long *stats,
                                                            unsigned long long *next)
{
    const unsigned lane = threadIdx.x & 31u;
    // per warp: a queue of rows to process (at most 31 left + 32 new)
    __shared__ int s_queue[kEuThreads / 32][64];
    int *const queue = s_queue[threadIdx.x >> 5];
    EuCounts nc;
    unsigned long long vox[2] = {0, 0}, rows = 0;
    bool tc_valid = false;
    float tc_ang = 0.0f;
    long long tc_c = 0, tc_s = 0;
    const long long s2g[3] = {g.sx, g.sy, g.sz};
    const int ng[3] = {g.nx, g.ny, g.nz};
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(next, static_cast<unsigned long long>(kEuRunHistories));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= static_cast<unsigned long long>(n)) break;
        const int64_t end = min(static_cast<int64_t>(base) + kEuRunHistories, n);
        for (int64_t i = static_cast<int64_t>(base); i < end; ++i) {
            // every lane classifies and sets up the same history
            const float w = in.wepl[i];
            const int cls = w < tau_l ? 0 : (w > tau_h ? 1 : -1);
            if (lane == 0) {
                nc.n_in += 1;
                nc.n_miss += cls == 0;
                nc.n_hit += cls == 1;
                nc.n_none += cls < 0;
            }
            if (cls < 0 || (cls == 0 && !use_miss) || (cls == 1 && !use_hit)) continue;
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
                if (lane == 0) nc.n_reject += 1;
                continue;
            }
            long long W[6];
            world_cs(g, tc_c, tc_s, ui, vi, uo, vo, W);
            long long A[3], B[3];
            for (int q = 0; q < 3; ++q) {
                A[q] = 2 * W[q];
                B[q] = 2 * W[q + 3];
            }
            // the major in-plane axis (rows run along it): frame axes 0, 1, 2
            // are (x, y, z) or (y, x, z), chosen with selects (a runtime
            // array index would put the arrays in local memory)
            const bool mj = llabs(B[1] - A[1]) > llabs(B[0] - A[0]);
            Capsule cp;
            cp.A[0] = mj ? A[1] : A[0];
            cp.A[1] = mj ? A[0] : A[1];
            cp.A[2] = A[2];
            cp.B[0] = mj ? B[1] : B[0];
            cp.B[1] = mj ? B[0] : B[1];
            cp.B[2] = B[2];
            cp.n[0] = mj ? ng[1] : ng[0];
            cp.n[1] = mj ? ng[0] : ng[1];
            cp.n[2] = ng[2];
            cp.s2[0] = mj ? s2g[1] : s2g[0];
            cp.s2[1] = mj ? s2g[0] : s2g[1];
            cp.s2[2] = s2g[2];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                cp.u[q] = cp.B[q] - cp.A[q];
                cp.sf[q] = static_cast<float>(cp.s2[q]) * (1.0f / 65536.0f);
                cp.Af[q] = static_cast<float>(cp.A[q]) * (1.0f / 131072.0f);
                cp.df[q] = static_cast<float>(cp.u[q]) * (1.0f / 131072.0f);
            }
            cp.uu = static_cast<unsigned long long>(cp.u[0] * cp.u[0]) +
                    static_cast<unsigned long long>(cp.u[1] * cp.u[1]) +
                    static_cast<unsigned long long>(cp.u[2] * cp.u[2]);
            cp.RR = static_cast<unsigned long long>(R2 * R2);
            cp.T = cp.uu == 0 ? static_cast<u128>(cp.RR) : mul64(cp.RR, cp.uu);
            cp.uu2 = static_cast<unsigned long long>(cp.u[1] * cp.u[1]) +
                     static_cast<unsigned long long>(cp.u[2] * cp.u[2]);
            cp.T2 = mul64(cp.RR, cp.uu2);
            cp.L2f = cp.df[0] * cp.df[0] + cp.df[1] * cp.df[1] + cp.df[2] * cp.df[2];
            cp.Rf = d0;
            cp.inv_L2 = cp.L2f > 0.0f ? __frcp_rz(cp.L2f) : 0.0f;
            cp.inv_d0 = cp.df[0] != 0.0f ? __frcp_rz(cp.df[0]) : 0.0f;
            cp.inv_s0 = __frcp_rz(cp.sf[0]);
            // index box of the capsule on axes 1 and 2: centres within
            // [min(A, B) - R, max(A, B) + R], widened by one
            int blo[3], bhi[3];
            for (int q = 1; q < 3; ++q) {
                const long long mn = min(cp.A[q], cp.B[q]) - R2, mx = max(cp.A[q], cp.B[q]) + R2;
                const long long fl = mn >= 0 ? mn / cp.s2[q] : -((-mn + cp.s2[q] - 1) / cp.s2[q]);
                const long long fh = mx >= 0 ? mx / cp.s2[q] : -((-mx + cp.s2[q] - 1) / cp.s2[q]);
                const long long l = (fl + cp.n[q] - 1) / 2 - 1, h = (fh + cp.n[q] + 1) / 2 + 1;
                blo[q] = static_cast<int>(max(l, 0LL));
                bhi[q] = static_cast<int>(min(h, static_cast<long long>(cp.n[q] - 1)));
            }
            if (blo[1] > bhi[1] || blo[2] > bhi[2]) continue;
            const int na = bhi[1] - blo[1] + 1;
            const int nrows = na * (bhi[2] - blo[2] + 1);
            int32_t *diff = mj ? td.dy[cls] : td.dx[cls];
            // the rows of the box that meet the capsule (cheap exact test)
            // queue up in shared memory; whenever 32 are queued all lanes take
            // one each, so the costly interval search runs with full warps
            int qn = 0;
            for (int base = 0; base < nrows; base += 32) {
                const int rw = base + static_cast<int>(lane);
                bool meets = false;
                int a = 0, k = 0;
                if (rw < nrows) {
                    a = blo[1] + rw % na;
                    k = blo[2] + rw / na;
                    meets = row_meets(cp, row_of(cp, a, k));
                }
                const unsigned bal = __ballot_sync(0xffffffffu, meets);
                if (meets) queue[qn + __popc(bal & ((1u << lane) - 1u))] = a | (k << 16);
                qn += __popc(bal);
                const bool last = base + 32 >= nrows;
                while (qn >= 32 || (last && qn > 0)) {
                    __syncwarp();
                    int lo, hi;
                    if (static_cast<int>(lane) < qn &&
                        row_interval(cp, queue[lane] & 0xffff, queue[lane] >> 16, lo, hi)) {
                        const int ra = queue[lane] & 0xffff, rk = queue[lane] >> 16;
                        // x-major rows: (nx + 1) entries per (y, z); y-major:
                        // (ny + 1) per (x, z)
                        int32_t *row = diff + (static_cast<int64_t>(ra) +
                                               static_cast<int64_t>(cp.n[1]) * rk) *
                                                  (cp.n[0] + 1);
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
            }
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
        int64_t blocks = int64_t(sm_count > 0 ? sm_count : 1) * 8;  // persistent warps
        const int64_t want = (n + kEuRunHistories * (kEuThreads / 32) - 1) /
                             (kEuRunHistories * (kEuThreads / 32));
        if (blocks > want) blocks = want;
        euclid_kernel<<<static_cast<unsigned>(blocks), kEuThreads, 0, st>>>(
            in, n, g, cd, tau_l, tau_h, use_miss, use_hit, R2, d0, td, cnt, cnt + 8);
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
