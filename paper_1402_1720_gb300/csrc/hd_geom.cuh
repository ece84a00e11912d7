// Fixed-point geometry and the exact voxel traversal (host and device).
//
// Geometry (Sec. 2.1-2.2): the path L_i is the closed segment from the entry
// point -T b + u_in e_u + v_in e_v to the exit point +T b + u_out e_u +
// v_out e_v, b = (cos phi, sin phi, 0), e_u = (-sin phi, cos phi, 0).  Each
// float32 input is rounded once to 16 fractional bits (ties to even); cos
// and sin come from an integer CORDIC with 30 fractional bits; world and
// grid coordinates follow by integer floor division.  After that every step
// is exact.
//
// Voxel set (Eq. 3.2 with d_0 = 0 against half-open voxel cubes): the voxels
// floor(P(t) / 2^16), t in [0, 1], of P(t) = G_in + t D inside the box.  The
// walk orders plane crossings with the three cross-multiplied terms
// E_ab = num_a |D_b| - num_b |D_a| (num_a / |D_a| is the parameter of axis
// a's next crossing) and updates them with additions only.  At equal
// parameters an axis moving + enters its next voxel at the crossing itself
// and an axis moving - leaves its voxel just after it, so a mixed tie visits
// the corner voxel between the two.  The walk starts at the exact rational
// parameter where the segment enters the box.
//
// Magnitudes: |G| < 2^30 + 2^28 (grid coordinates, possibly shifted to a
// tile origin), |D| < 2^31, so every product below stays under 2^62.
#pragma once

#include <cmath>
#include <cstdint>

#include "hd_internal.cuh"

#define HD_HD __host__ __device__ __forceinline__

namespace hd {

HD_HD unsigned long long umulhi64(unsigned long long a, unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return static_cast<unsigned long long>((static_cast<unsigned __int128>(a) * b) >> 64);
#endif
}

HD_HD unsigned umulhi32(unsigned a, unsigned b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return static_cast<unsigned>((static_cast<unsigned long long>(a) * b) >> 32);
#endif
}

// floor(n / d) for d >= 2, |n| < 2^62, with m = floor(2^64 / d): the
// multiply-high quotient is low by at most one, fixed by one comparison.
HD_HD long long floordiv_magic(long long n, unsigned long long d, unsigned long long m)
{
    const bool neg = n < 0;
    const unsigned long long u =
        neg ? static_cast<unsigned long long>(-(n + 1)) : static_cast<unsigned long long>(n);
    unsigned long long q = umulhi64(u, m);
    if (u - q * d >= d) ++q;
    return neg ? -1 - static_cast<long long>(q) : static_cast<long long>(q);
}

// Q16 of a value known to satisfy |x| < 4096: the 32-bit conversion rounds
// exactly as the 64-bit one does.
HD_HD int q16_small(float x)
{
#ifdef __CUDA_ARCH__
    return __float2int_rn(x * 65536.0f);
#else
    return static_cast<int>(lrintf(x * 65536.0f));
#endif
}

HD_HD long long q16_of(float x)
{
    // x * 2^16 is exact in float32 for |x| < 2^20 * ..., so the conversion
    // is the only rounding (to nearest, ties to even).
#ifdef __CUDA_ARCH__
    return __float2ll_rn(x * 65536.0f);
#else
    return llrintf(x * 65536.0f);
#endif
}

HD_HD long long floordiv_pos(long long a, long long b)
{
    long long q = a / b;
    if (a - q * b != 0 && a < 0) --q;
    return q;
}

// Float value of a 64-bit integer (relative error below 2^-22) built from
// two 32-bit conversions.
HD_HD float float_of(long long a)
{
    return static_cast<float>(static_cast<int>(a >> 32)) * 4294967296.0f +
           static_cast<float>(static_cast<unsigned>(a & 0xffffffffLL));
}

// floor(a / b), b > 0, for quotients known to be small (|a / b| < 2^20 and
// |a| < 2^62): a float estimate corrected with exact integer arithmetic, so
// no 64-bit division is needed.
HD_HD long long floordiv_small(long long a, long long b)
{
    // an approximate float quotient: the integer steps below make it exact
#ifdef __CUDA_ARCH__
    long long q = static_cast<long long>(static_cast<int>(floorf(__fdividef(float_of(a), float_of(b)))));
#else
    long long q = static_cast<long long>(static_cast<int>(floorf(float_of(a) / float_of(b))));
#endif
    long long r = a - q * b;
    while (r < 0) {
        --q;
        r += b;
    }
    while (r >= b) {
        ++q;
        r -= b;
    }
    return q;
}

// floor(a / b) for b > 0 and |a / b| < 2^20: a correctly rounded float
// quotient estimate (relative error below 2^-21) is within one of the
// floor, so one correction step each way settles it; unlike floordiv_small
// it needs no loop, which keeps the lanes of a warp together.
HD_HD long long fdiv_small(long long a, long long b)
{
#ifdef __CUDA_ARCH__
    long long q = static_cast<long long>(
        static_cast<int>(floorf(__fdividef(__ll2float_rn(a), __ll2float_rn(b)))));
#else
    long long q = static_cast<long long>(
        static_cast<int>(std::floor(static_cast<float>(a) / static_cast<float>(b))));
#endif
    long long r = a - q * b;
    if (r < 0) {
        --q;
        r += b;
    }
    if (r >= b) ++q;
    return q;
}
// Rotation-mode CORDIC of an angle in degrees * 2^16: cos and sin * 2^30.
HD_HD void cordic_cs(long long a_q16, const Cordic &cd, long long &c, long long &s)
{
    const long long full = 360LL * kQ16, quarter = 90LL * kQ16;
    long long a = a_q16 % full;
    if (a < 0) a += full;
    const int k = static_cast<int>(a / quarter);
    const long long r = a - k * quarter;
    long long z = r << 14;
    // |x|, |y| stay below 2^31 (unit vector scaled by 2^30)
    int x = static_cast<int>(cd.K), y = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int xs = x >> i, ys = y >> i;
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

// Grid coordinate (voxel units, Q16) of a world coordinate w (mm, Q16):
// floor((2 w + n s) 2^16 / (2 s)), the division done by multiply-high.
HD_HD long long to_grid(long long w, int n, long long s_q, unsigned long long m)
{
    return floordiv_magic((2 * w + static_cast<long long>(n) * s_q) * kQ16,
                          static_cast<unsigned long long>(2 * s_q), m);
}

// Host-side construction of the fixed-point geometry.
inline GeomQ make_geomq(int nx, int ny, int nz, float sx, float sy, float sz, float T)
{
    GeomQ g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.sx = llrint(static_cast<double>(sx) * 65536.0);
    g.sy = llrint(static_cast<double>(sy) * 65536.0);
    g.sz = llrint(static_cast<double>(sz) * 65536.0);
    g.T = llrint(static_cast<double>(T) * 65536.0);
    auto magic = [](long long s) {
        const unsigned __int128 one = static_cast<unsigned __int128>(1) << 64;
        return static_cast<unsigned long long>(one / static_cast<unsigned long long>(2 * s));
    };
    g.mx = magic(g.sx);
    g.my = magic(g.sy);
    g.mz = magic(g.sz);
    return g;
}

// World entry and exit points (mm, Q16) of one history from its gantry
// cos/sin: W = (x_in, y_in, z_in, x_out, y_out, z_out).  The inputs must
// satisfy |u|, |v| < 4096 mm (endpoints_cs checks it).
HD_HD void world_cs(const GeomQ &g, long long c, long long s, float ui, float vi, float uo,
                    float vo, long long W[6])
{
    // every factor fits 32 bits (T < 2^28 since the tracker distance is below
    // 4096 mm, |c|, |s| <= 2^30, |u| Q16 < 2^28): exact 32 x 32 -> 64 products
    const int T = static_cast<int>(g.T);
    const int ci = static_cast<int>(c), si = static_cast<int>(s);
    const int qui = q16_small(ui), quo = q16_small(uo);
    auto mul = [](int a, int b) { return static_cast<long long>(a) * static_cast<long long>(b); };
    W[0] = (-mul(T, ci) - mul(qui, si)) >> 30;
    W[1] = (-mul(T, si) + mul(qui, ci)) >> 30;
    W[2] = q16_small(vi);
    W[3] = (mul(T, ci) - mul(quo, si)) >> 30;
    W[4] = (mul(T, si) + mul(quo, ci)) >> 30;
    W[5] = q16_small(vo);
}

// Grid Q16 endpoints of one history from its gantry cos/sin; false when the
// history is rejected.
HD_HD bool endpoints_cs(const GeomQ &g, long long c, long long s, float ui, float vi, float uo,
                        float vo, int32_t out[6])
{
    if (!(fabsf(ui) < 4096.0f) || !(fabsf(vi) < 4096.0f) || !(fabsf(uo) < 4096.0f) ||
        !(fabsf(vo) < 4096.0f))
        return false;
    long long W[6];
    world_cs(g, c, s, ui, vi, uo, vo, W);
    const long long G[6] = {to_grid(W[0], g.nx, g.sx, g.mx), to_grid(W[1], g.ny, g.sy, g.my),
                            to_grid(W[2], g.nz, g.sz, g.mz), to_grid(W[3], g.nx, g.sx, g.mx),
                            to_grid(W[4], g.ny, g.sy, g.my), to_grid(W[5], g.nz, g.sz, g.mz)};
    const long long lim = 1LL << 30;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (G[a] >= lim || G[a] <= -lim) return false;
        out[a] = static_cast<int32_t>(G[a]);
    }
    return true;
}

// Grid Q16 endpoints of one history; false when the history is rejected.
HD_HD bool endpoints(const GeomQ &g, const Cordic &cd, float ang, float ui, float vi, float uo,
                     float vo, int32_t out[6])
{
    if (!(fabsf(ang) < 1048576.0f)) return false;
    long long c, s;
    cordic_cs(q16_of(ang), cd, c, s);
    return endpoints_cs(g, c, s, ui, vi, uo, vo, out);
}

// The slices the part of a segment inside the grid's x-y extent can touch:
// the parameter interval [t_lo, t_hi] of the segment r (grid Q16) inside
// [0, nx) x [0, ny) (closed at its ends, exact rationals), and the z
// indices at its two ends, ordered and clamped to the grid.  A superset of
// the slices that hold voxels of the segment (z is monotone along it);
// false when the segment misses the grid.
HD_HD bool grid_z_range(const TilePlan &tp, const int32_t r[6], int &zlo, int &zhi)
{
    // t_lo = nl / dl, t_hi = nh / dh (den > 0)
    long long nl = 0, dl = 1, nh = 1, dh = 1;
    const int H[2] = {tp.nx << 16, tp.ny << 16};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const long long p = r[a], d = static_cast<long long>(r[a + 3]) - r[a];
        long long en = 0, ed = 1, xn = 1, xd = 1;  // entry and exit parameters
        if (d > 0) {
            if (p >= H[a] || p + d < 0) return false;
            if (p < 0) { en = -p; ed = d; }
            if (p + d > H[a]) { xn = H[a] - p; xd = d; }
        } else if (d < 0) {
            if (p < 0 || p + d >= H[a]) return false;
            if (p >= H[a]) { en = p - H[a]; ed = -d; }
            if (p + d < 0) { xn = p; xd = -d; }
        } else if (p < 0 || p >= H[a]) {
            return false;
        }
        if (en * dl > nl * ed) { nl = en; dl = ed; }
        if (xn * dh < nh * xd) { nh = xn; dh = xd; }
    }
    if (nl * dh > nh * dl) return false;
    const long long z = r[2], dz = static_cast<long long>(r[5]) - r[2];
    int z0 = static_cast<int>(floordiv_small(z * dl + nl * dz, dl << 16));
    int z1 = static_cast<int>(floordiv_small(z * dh + nh * dz, dh << 16));
    if (z0 > z1) { const int t = z0; z0 = z1; z1 = t; }
    if (z1 < 0 || z0 >= tp.nz) return false;
    zlo = z0 < 0 ? 0 : z0;
    zhi = z1 >= tp.nz ? tp.nz - 1 : z1;
    return true;
}

// Tiles a record can touch, given its slices zlo..zhi (grid_z_range): in x
// and y the bounding box of its segment clamped to the grid, in z those
// slices, in tile units.  Returns the number of tiles (0 when the box
// misses the grid).
HD_HD int tile_range_z(const TilePlan &tp, const int32_t r[6], int zlo, int zhi, int lo[3],
                       int hi[3])
{
    const int n[3] = {tp.nx, tp.ny, tp.nz};
    const unsigned m[3] = {tp.mtx, tp.mty, tp.mtz};
    int cnt = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int a0 = r[a] >> 16, a1 = r[a + 3] >> 16;
        int mn = a0 < a1 ? a0 : a1, mx = a0 < a1 ? a1 : a0;
        if (a == 2) {
            mn = zlo;
            mx = zhi;
        }
        if (mx < 0 || mn >= n[a]) return 0;
        mn = mn < 0 ? 0 : mn;
        mx = mx >= n[a] ? n[a] - 1 : mx;
        // floor(v / t) = umulhi(v, floor(2^32 / t) + 1) for v, t <= 4096;
        // m = 0 stands for t = 1
        lo[a] = m[a] ? static_cast<int>(umulhi32(static_cast<unsigned>(mn), m[a])) : mn;
        hi[a] = m[a] ? static_cast<int>(umulhi32(static_cast<unsigned>(mx), m[a])) : mx;
        cnt *= hi[a] - lo[a] + 1;
    }
    return cnt;
}

// tile_range_z with the slices of grid_z_range; 0 when the segment misses
// the grid (it then has no voxel at all).
HD_HD int tile_range(const TilePlan &tp, const int32_t r[6], int lo[3], int hi[3])
{
    int zlo, zhi;
    if (!grid_z_range(tp, r, zlo, zhi)) return 0;
    return tile_range_z(tp, r, zlo, zhi, lo, hi);
}

// A record's status word: bits 0-1 the path (0 no record, 1 tiled, 2
// global), bit 2 the class (0 missed, 1 hit), bits 8-19 and 20-31 its first
// and last slice (grid_z_range, computed once).
HD_HD int32_t record_status(int path, int cls, int zlo, int zhi)
{
    return static_cast<int32_t>(static_cast<uint32_t>(path) | (static_cast<uint32_t>(cls) << 2) |
                                (static_cast<uint32_t>(zlo) << 8) |
                                (static_cast<uint32_t>(zhi) << 20));
}
HD_HD int status_path(int32_t s) { return s & 3; }
HD_HD int status_cls(int32_t s) { return (s >> 2) & 1; }
HD_HD int status_zlo(int32_t s) { return (static_cast<uint32_t>(s) >> 8) & 0xfff; }
HD_HD int status_zhi(int32_t s) { return static_cast<uint32_t>(s) >> 20; }

// ------------------------------------------------------------------ walk

// Resumable traversal state of one segment inside a box of nx*ny*nz voxels.
struct Walk {
    long long exy, exz, eyz;     // crossing-order terms
    long long ax16, ay16, az16;  // |D_a| * 2^16
    int idx;                     // linear index (x fastest) of the current voxel
    int kx, ky, kz;              // remaining valid crossings per axis
    int stx, sty, stz;           // signed index strides
    int flags;                   // bits 0-2: axis moves +; bits 4-6: pending - group
};

HD_HD void walk_apply(Walk &w, int mask)
{
    if (mask & 1) { --w.kx; w.idx += w.stx; w.exy += w.ay16; w.exz += w.az16; }
    if (mask & 2) { --w.ky; w.idx += w.sty; w.exy -= w.ax16; w.eyz += w.az16; }
    if (mask & 4) { --w.kz; w.idx += w.stz; w.exz -= w.ax16; w.eyz -= w.ay16; }
}

HD_HD bool walk_exhausted(const Walk &w, int mask)
{
    return ((mask & 1) && w.kx == 0) || ((mask & 2) && w.ky == 0) || ((mask & 4) && w.kz == 0);
}

// Advance to the next voxel of the set; false when the set is exhausted.
HD_HD bool walk_next(Walk &w)
{
    const int pend = (w.flags >> 4) & 7;
    if (pend) {
        // the - half of a tie: those axes leave their voxels just after the
        // crossing, before any later event
        w.flags &= 7;
        if (walk_exhausted(w, pend)) return false;
        walk_apply(w, pend);
        return true;
    }
    if (w.exy != 0 && w.exz != 0 && w.eyz != 0) {
        // one axis crosses strictly first (the common case, branch-free)
        const bool cxy = w.exy < 0, cxz = w.exz < 0, cyz = w.eyz < 0;
        const bool sx = cxy && cxz;
        const bool sy = !cxy && cyz;
        const int k = sx ? w.kx : (sy ? w.ky : w.kz);
        if (k == 0) return false;
        w.kx -= sx;
        w.ky -= sy;
        w.kz -= (!sx && !sy);
        w.idx += sx ? w.stx : (sy ? w.sty : w.stz);
        w.exy += sx ? w.ay16 : (sy ? -w.ax16 : 0);
        w.exz += sx ? w.az16 : (sy ? 0 : -w.ax16);
        w.eyz += sx ? 0 : (sy ? w.az16 : -w.ay16);
        return true;
    }
    // several axes cross at the same parameter
    const int in = ((w.ax16 != 0 && w.exy <= 0 && w.exz <= 0) ? 1 : 0) |
                   ((w.ay16 != 0 && w.exy >= 0 && w.eyz <= 0) ? 2 : 0) |
                   ((w.az16 != 0 && w.exz >= 0 && w.eyz >= 0) ? 4 : 0);
    const int plus = in & w.flags & 7, minus = in & ~w.flags & 7;
    if (plus) {
        if (walk_exhausted(w, plus)) return false;
        walk_apply(w, plus);
        w.flags |= minus << 4;
        return true;
    }
    if (walk_exhausted(w, minus)) return false;
    walk_apply(w, minus);
    return true;
}

// Set up the walk of segment gi -> go (grid Q16, relative to the box
// origin) through the box [0, nx) x [0, ny) x [0, nz).  Returns false when
// the segment has no voxel in the box; otherwise w.idx is its first voxel.
HD_HD bool walk_begin(Walk &w, const int32_t gi[3], const int32_t go[3], int nx, int ny, int nz,
                      int *ijk = nullptr)
{
    const long long hx = static_cast<long long>(nx) << 16, hy = static_cast<long long>(ny) << 16,
                    hz = static_cast<long long>(nz) << 16;
    const long long x0 = gi[0], y0 = gi[1], z0 = gi[2];
    const long long dx = static_cast<long long>(go[0]) - x0;
    const long long dy = static_cast<long long>(go[1]) - y0;
    const long long dz = static_cast<long long>(go[2]) - z0;

    // t_enter = tN / tQ: the largest per-axis entry parameter
    long long tN = 0, tQ = 1;
    bool ok = true;
    auto entry = [&](long long p0, long long d, long long hi) {
        long long cN = -1, cQ = 1;
        if (d > 0) {
            if (p0 >= hi) ok = false;
            else if (p0 < 0) { cN = -p0; cQ = d; }
        } else if (d < 0) {
            if (p0 < 0) ok = false;
            else if (p0 >= hi) { cN = p0 - hi; cQ = -d; }
        } else if (p0 < 0 || p0 >= hi) {
            ok = false;
        }
        if (cN >= 0 && cN * tQ > tN * cQ) { tN = cN; tQ = cQ; }
    };
    entry(x0, dx, hx);
    entry(y0, dy, hy);
    entry(z0, dz, hz);
    if (!ok || tN > tQ) return false;

    int ix, iy, iz;
    if (tN == 0) {
        ix = static_cast<int>(x0 >> 16);
        iy = static_cast<int>(y0 >> 16);
        iz = static_cast<int>(z0 >> 16);
    } else {
        const long long den = tQ << 16;
        // voxel indices at the entry parameter: quotients below 2^15
        ix = static_cast<int>(floordiv_small(x0 * tQ + tN * dx, den));
        iy = static_cast<int>(floordiv_small(y0 * tQ + tN * dy, den));
        iz = static_cast<int>(floordiv_small(z0 * tQ + tN * dz, den));
    }
    if ((dx > 0 && ix >= nx) || (dx < 0 && ix < 0)) return false;
    if ((dy > 0 && iy >= ny) || (dy < 0 && iy < 0)) return false;
    if ((dz > 0 && iz >= nz) || (dz < 0 && iz < 0)) return false;

    long long ax, ay, az, nmx, nmy, nmz;
    {
        const int fx = go[0] >> 16, fy = go[1] >> 16, fz = go[2] >> 16;
        if (dx > 0) { ax = dx; nmx = ((static_cast<long long>(ix) + 1) << 16) - x0; w.kx = (fx < nx - 1 ? fx : nx - 1) - ix; }
        else if (dx < 0) { ax = -dx; nmx = x0 - (static_cast<long long>(ix) << 16); w.kx = ix - (fx > 0 ? fx : 0); }
        else { ax = 0; nmx = 1; w.kx = 0; }
        if (dy > 0) { ay = dy; nmy = ((static_cast<long long>(iy) + 1) << 16) - y0; w.ky = (fy < ny - 1 ? fy : ny - 1) - iy; }
        else if (dy < 0) { ay = -dy; nmy = y0 - (static_cast<long long>(iy) << 16); w.ky = iy - (fy > 0 ? fy : 0); }
        else { ay = 0; nmy = 1; w.ky = 0; }
        if (dz > 0) { az = dz; nmz = ((static_cast<long long>(iz) + 1) << 16) - z0; w.kz = (fz < nz - 1 ? fz : nz - 1) - iz; }
        else if (dz < 0) { az = -dz; nmz = z0 - (static_cast<long long>(iz) << 16); w.kz = iz - (fz > 0 ? fz : 0); }
        else { az = 0; nmz = 1; w.kz = 0; }
    }
    w.exy = nmx * ay - nmy * ax;
    w.exz = nmx * az - nmz * ax;
    w.eyz = nmy * az - nmz * ay;
    // two axes that never move never cross: give their term a fixed sign so
    // it is never read as a tie
    if (ax == 0 && ay == 0) w.exy = 1;
    if (ax == 0 && az == 0) w.exz = 1;
    if (ay == 0 && az == 0) w.eyz = 1;
    w.ax16 = ax << 16;
    w.ay16 = ay << 16;
    w.az16 = az << 16;
    w.stx = dx > 0 ? 1 : -1;
    w.sty = dy > 0 ? nx : -nx;
    w.stz = dz > 0 ? nx * ny : -(nx * ny);
    w.flags = (dx > 0 ? 1 : 0) | (dy > 0 ? 2 : 0) | (dz > 0 ? 4 : 0);
    w.idx = ix + nx * (iy + ny * iz);
    // an axis moving - that enters through the box's upper face starts one
    // voxel outside; its first crossing brings it in
    int out = (ix >= nx ? 1 : 0) | (iy >= ny ? 2 : 0) | (iz >= nz ? 4 : 0);
    const int k0x = w.kx, k0y = w.ky, k0z = w.kz;
    while (out) {
        if (!walk_next(w)) return false;
        if ((out & 1) && w.kx < k0x) out &= ~1;
        if ((out & 2) && w.ky < k0y) out &= ~2;
        if ((out & 4) && w.kz < k0z) out &= ~4;
    }
    if (ijk) {
        ijk[0] = ix + (dx > 0 ? 1 : -1) * (k0x - w.kx);
        ijk[1] = iy + (dy > 0 ? 1 : -1) * (k0y - w.ky);
        ijk[2] = iz + (dz > 0 ? 1 : -1) * (k0z - w.kz);
    }
    return true;
}

// ------------------------------------------------------------- run walk
//
// The same voxel set, produced as runs along the major in-plane axis m (x
// or y, the one with the larger |D|): only crossings of the two minor axes
// (the other in-plane axis and z) are explicit events.  For a minor axis c,
// D_c = num_c |D_m| - num_m |D_c| orders m's pending crossings against c's:
// m crosses ceil(D_c / S_c) times strictly before c does (S_c = |D_c| 2^16),
// and exactly when c does if D_c is a multiple of S_c.  D_c is kept as
// q S_c + rh 2^16 + rl: every update adds a multiple of 2^16, so rl (the low
// 16 bits) never changes and q, rh are 32-bit, updated Bresenham-style with
// no division after the set-up.  A quotient of 2^29 or more stands for
// "after the major axis has run out" (a box has at most 4096 crossings per
// axis), so q saturates there.  Events are processed in exactly the order
// and with exactly the tie rules of walk_next; crossings of m alone are
// batched.
constexpr int kQBig = 1 << 29;

struct RunWalk {
    long long e12;       // crossing order of the two minors (num_0 |D_1| - num_1 |D_0|)
    int q[2];            // D_c = q S_c + rh 2^16 + rl (q saturated at kQBig)
    unsigned rh[2];      // 0 <= rh < ad
    unsigned ad[2];      // |D_c|, so S_c = ad 2^16
    int Qu[2];           // |D_m| = Qu |D_c| + Ru (Qu saturated at kQBig)
    unsigned Ru[2];
    int km, kc[2];       // remaining valid crossings
    int im, run_start;   // major index now and where the current run began
    int row;             // row of the current run in the major axis' layout
    int rstride[2];      // signed row change when minor c crosses
    int nmaj;            // box size along the major axis
    int flags;           // bit 0: major moves +, bits 1-2: minor moves +, bits 3-4: minor
                         // moves at all, bit 5: major is y, bits 6-8: pending part,
                         // bit 9: done, bits 10-11: rl of minor c is nonzero
};

HD_HD int sat_add(int q, int d)
{
    const int v = q + d;  // both <= kQBig, so no overflow
    return v > kQBig ? kQBig : v;
}

HD_HD bool run_rpos(const RunWalk &w, int c)  // r > 0 for minor c
{
    return w.rh[c] != 0 || ((w.flags >> (10 + c)) & 1);
}

// Minor c crosses: D_c grows by |D_m| 2^16.
HD_HD void run_minor_step(RunWalk &w, int c)
{
    unsigned rh = w.rh[c] + w.Ru[c];
    int q = sat_add(w.q[c], w.Qu[c]);
    if (rh >= w.ad[c]) {
        rh -= w.ad[c];
        q = sat_add(q, 1);
    }
    w.rh[c] = rh;
    w.q[c] = q;
    --w.kc[c];
    w.row += w.rstride[c];
    if (c == 0) w.e12 += static_cast<long long>(w.ad[1]) << 16;
    else w.e12 -= static_cast<long long>(w.ad[0]) << 16;
}

// Apply one part (a set of axes crossing together) of an event: bit 0 the
// major axis, bits 1-2 the minors.  Returns 1 and the finished run when a
// minor crossed (a new row begins), 0 when only the major moved, and -1 with
// the last run when an axis in the part has no valid crossing left (end).
HD_HD int run_apply(RunWalk &w, int part, int &row, int &lo, int &hi)
{
    if (((part & 1) && w.km == 0) || ((part & 2) && w.kc[0] == 0) ||
        ((part & 4) && w.kc[1] == 0)) {
        row = w.row;
        lo = w.run_start < w.im ? w.run_start : w.im;
        hi = w.run_start < w.im ? w.im : w.run_start;
        w.flags |= 1 << 9;
        return -1;
    }
    const int im_before = w.im;
    if (part & 1) {
        w.im += (w.flags & 1) ? 1 : -1;
        --w.km;
        w.q[0] -= (w.q[0] < kQBig) ? 1 : 0;
        w.q[1] -= (w.q[1] < kQBig) ? 1 : 0;
    }
    if (!(part & 6)) return 0;
    row = w.row;
    lo = w.run_start < im_before ? w.run_start : im_before;
    hi = w.run_start < im_before ? im_before : w.run_start;
    if (part & 2) run_minor_step(w, 0);
    if (part & 4) run_minor_step(w, 1);
    w.run_start = w.im;
    return 1;
}

// General step of the run walk (every case, including ties and the end).
HD_HD bool run_next_general(RunWalk &w, int &row, int &lo, int &hi)
{
    if (w.flags & (1 << 9)) return false;
    for (;;) {
        const int pend = (w.flags >> 6) & 7;
        if (pend) {
            w.flags &= ~(7 << 6);
            const int res = run_apply(w, pend, row, lo, hi);
            if (res != 0) return true;
            continue;
        }
        const bool act0 = (w.flags >> 3) & 1, act1 = (w.flags >> 4) & 1;
        int g;  // minors in the event (bits 1-2 of a part)
        if (act0 && act1) g = w.e12 < 0 ? 2 : (w.e12 > 0 ? 4 : 6);
        else g = act0 ? 2 : (act1 ? 4 : 0);
        const bool c0 = (g & 2) != 0;  // minor 0 takes part (else minor 1)
        int j;
        if (g == 0) {
            j = kQBig;
        } else {
            const int qc = c0 ? w.q[0] : w.q[1];
            const bool rp = c0 ? run_rpos(w, 0) : run_rpos(w, 1);
            j = (qc > 0 || (qc == 0 && rp)) ? qc + (rp ? 1 : 0) : 0;
        }
        if (j > w.km) {
            // the major axis runs out before any minor crossing: last run
            w.im += (w.flags & 1) ? w.km : -w.km;
            w.km = 0;
            row = w.row;
            lo = w.run_start < w.im ? w.run_start : w.im;
            hi = w.run_start < w.im ? w.im : w.run_start;
            w.flags |= 1 << 9;
            return true;
        }
        if (j > 0) {
            w.im += (w.flags & 1) ? j : -j;
            w.km -= j;
            w.q[0] -= (w.q[0] < kQBig) ? j : 0;
            w.q[1] -= (w.q[1] < kQBig) ? j : 0;
        }
        if (g != 0 && (c0 ? (w.q[0] == 0 && !run_rpos(w, 0)) : (w.q[1] == 0 && !run_rpos(w, 1))))
            g |= 1;  // the major crosses at the same parameter
        const int posmask = w.flags & 7;
        const int plus = g & posmask, minus = g & ~posmask & 7;
        if (plus) {
            const int res = run_apply(w, plus, row, lo, hi);
            if (res < 0) return true;
            if (minus) w.flags |= minus << 6;
            if (res > 0) return true;
            continue;
        }
        const int res = run_apply(w, minus, row, lo, hi);
        if (res != 0) return true;
    }
}

// Next run of the set: returns false when there is none.  row indexes the
// run's line in the major axis' layout (x-major: y + ny z, y-major:
// x + nx z); lo..hi is the inclusive range of major indices.  The common
// case (one minor axis crossing alone after j major crossings, or the end
// of the walk) is done inline without branching on which minor crossed;
// ties and the parts they leave go to run_next_general.
HD_HD bool run_next(RunWalk &w, int &row, int &lo, int &hi)
{
    const int fl = w.flags;
    if (fl & (1 << 9)) return false;
    const bool act0 = (fl >> 3) & 1, act1 = (fl >> 4) & 1;
    if ((fl & (7 << 6)) == 0 && !(act0 && act1 && w.e12 == 0)) {
        const bool cz = !(act0 && (!act1 || w.e12 < 0));  // minor 1 crosses first
        const int qc = cz ? w.q[1] : w.q[0];
        const bool rp = cz ? run_rpos(w, 1) : run_rpos(w, 0);
        const int kcc = cz ? w.kc[1] : w.kc[0];
        const bool any = act0 || act1;
        const int j = !any ? kQBig : ((qc > 0 || (qc == 0 && rp)) ? qc + (rp ? 1 : 0) : 0);
        const bool runs_out = j > w.km;
        const bool major_tie = any && !rp && qc >= 0;
        if (runs_out || !major_tie) {
            const int ji = runs_out ? w.km : j;
            const int end = w.im + ((fl & 1) ? ji : -ji);
            row = w.row;
            lo = w.run_start < end ? w.run_start : end;
            hi = w.run_start < end ? end : w.run_start;
            if (runs_out || kcc == 0) {
                w.flags = fl | (1 << 9);
                return true;
            }
            w.km -= ji;
            w.q[0] -= (w.q[0] < kQBig) ? ji : 0;
            w.q[1] -= (w.q[1] < kQBig) ? ji : 0;
            // minor cz crosses alone
            const unsigned adc = cz ? w.ad[1] : w.ad[0];
            unsigned rh = (cz ? w.rh[1] : w.rh[0]) + (cz ? w.Ru[1] : w.Ru[0]);
            int qn = sat_add(cz ? w.q[1] : w.q[0], cz ? w.Qu[1] : w.Qu[0]);
            if (rh >= adc) {
                rh -= adc;
                qn = sat_add(qn, 1);
            }
            w.q[1] = cz ? qn : w.q[1];
            w.rh[1] = cz ? rh : w.rh[1];
            w.q[0] = cz ? w.q[0] : qn;
            w.rh[0] = cz ? w.rh[0] : rh;
            w.kc[1] -= cz ? 1 : 0;
            w.kc[0] -= cz ? 0 : 1;
            w.row += cz ? w.rstride[1] : w.rstride[0];
            w.e12 += cz ? -(static_cast<long long>(w.ad[0]) << 16)
                        : (static_cast<long long>(w.ad[1]) << 16);
            w.im = end;
            w.run_start = end;
            return true;
        }
    }
    return run_next_general(w, row, lo, hi);
}

// Set up the run walk of segment gi -> go in the box (see walk_begin).
HD_HD bool run_begin(RunWalk &rw, const int32_t gi[3], const int32_t go[3], int nx, int ny,
                     int nz)
{
    Walk w;
    int ijk[3];
    if (!walk_begin(w, gi, go, nx, ny, nz, ijk)) return false;
    const bool ymaj = w.ay16 > w.ax16;
    // axes: major m, minor 0 (the other in-plane axis), minor 1 (z)
    const unsigned am = static_cast<unsigned>((ymaj ? w.ay16 : w.ax16) >> 16);
    const unsigned a0 = static_cast<unsigned>((ymaj ? w.ax16 : w.ay16) >> 16);
    const unsigned a1 = static_cast<unsigned>(w.az16 >> 16);
    // D_c = -E_mc
    const long long d0 = ymaj ? w.exy : -w.exy;
    const long long d1 = ymaj ? -w.eyz : -w.exz;
    rw.e12 = ymaj ? w.exz : w.eyz;
    const int fl = w.flags;
    const int pm = ymaj ? ((fl >> 1) & 1) : (fl & 1);
    const int p0 = ymaj ? (fl & 1) : ((fl >> 1) & 1);
    const int p1 = (fl >> 2) & 1;
    int flags = pm | (p0 << 1) | (p1 << 2) | ((a0 != 0) << 3) | ((a1 != 0) << 4) | (ymaj << 5);
    const int pend = (fl >> 4) & 7;  // pending - part of walk_begin, in x,y,z bits
    if (pend) {
        const int bm = ymaj ? ((pend >> 1) & 1) : (pend & 1);
        const int b0 = ymaj ? (pend & 1) : ((pend >> 1) & 1);
        const int b1 = (pend >> 2) & 1;
        flags |= (bm | (b0 << 1) | (b1 << 2)) << 6;
    }
    rw.km = ymaj ? w.ky : w.kx;
    rw.kc[0] = ymaj ? w.kx : w.ky;
    rw.kc[1] = w.kz;
    const unsigned A[2] = {a0, a1};
    const long long Dc[2] = {d0, d1};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (A[c] != 0) {
            rw.ad[c] = A[c];
            const unsigned qu = am / A[c];
            rw.Qu[c] = qu >= (1u << 20) ? kQBig : static_cast<int>(qu);
            rw.Ru[c] = am - qu * A[c];
            // D = Dh 2^16 + Dl with 0 <= Dl < 2^16, q = floor(Dh / ad)
            const long long dh = Dc[c] >> 16;
            const unsigned dl = static_cast<unsigned>(Dc[c] & 0xffff);
            if (float_of(dh) >= 1048576.0f * static_cast<float>(A[c])) {
                rw.q[c] = kQBig;
                rw.rh[c] = 1;  // any remainder > 0: never a tie
            } else {
                const long long q = floordiv_small(dh, static_cast<long long>(A[c]));
                rw.q[c] = static_cast<int>(q);
                rw.rh[c] = static_cast<unsigned>(dh - q * static_cast<long long>(A[c]));
            }
            if (dl != 0) flags |= 1 << (10 + c);
        } else {
            rw.ad[c] = 1;
            rw.Qu[c] = kQBig;
            rw.Ru[c] = 0;
            rw.q[c] = kQBig;
            rw.rh[c] = 0;
            flags |= 1 << (10 + c);
        }
    }
    rw.flags = flags;
    if (!ymaj) {
        rw.im = ijk[0];
        rw.row = ijk[1] + ny * ijk[2];
        rw.rstride[0] = (fl & 2) ? 1 : -1;
        rw.rstride[1] = (fl & 4) ? ny : -ny;
        rw.nmaj = nx;
    } else {
        rw.im = ijk[1];
        rw.row = ijk[0] + nx * ijk[2];
        rw.rstride[0] = (fl & 1) ? 1 : -1;
        rw.rstride[1] = (fl & 4) ? nx : -nx;
        rw.nmaj = ny;
    }
    rw.run_start = rw.im;
    return true;
}

// Calls visit(v) for the voxels of the walk gi -> go over the whole grid in
// path order: runs come in order, and a run is expanded in the direction
// the major axis moves.
template <class VisitT>
HD_HD void walk_path(const int32_t r[6], int nx, int ny, int nz, VisitT &visit)
{
    const int32_t gi[3] = {r[0], r[1], r[2]};
    const int32_t go[3] = {r[3], r[4], r[5]};
    RunWalk w;
    if (!run_begin(w, gi, go, nx, ny, nz)) return;
    const bool ymaj = (w.flags >> 5) & 1;
    const bool plus = w.flags & 1;
    int row, lo, hi;
    // a run's voxels are base + m stride: x-major rows are y + ny z (stride
    // 1), y-major rows x + nx z (stride nx)
    const int stride = ymaj ? nx : 1;
    const int step = plus ? stride : -stride;
    while (run_next(w, row, lo, hi)) {
        const int base = ymaj ? row % nx + nx * ny * (row / nx) : nx * row;
        int v = base + (plus ? lo : hi) * stride;
        for (int k = hi - lo; k >= 0; --k, v += step) visit(static_cast<uint32_t>(v));
    }
}

// ---------------------------------------------------------- lean run walk
//
// Most walks inside a one-voxel-deep tile are "lean": the in-plane minor
// axis (minor 0) never crosses at the same parameter as the major axis
// (rl_0 != 0: D_0 is never a multiple of S_0), z never ties with the major
// axis (rl_1 != 0) nor with minor 0 (e12 is never a multiple of 2^16, and
// every update adds one), no tie is pending at the start, and z has no valid
// crossing inside the box, so its first crossing (if any) ends the walk.
// Then every event is a lone crossing and the runs have a closed form.
// Counting major crossings from the start, minor 0's k-th crossing (k >= 1)
// comes after J_k = q_0 + 1 + (k - 1) Qu_0 + floor((rh_0 + (k - 1) Ru_0) / ad_0)
// of them (so J_1 = q_0 + 1, and J_{k+1} = J_k + Qu_0 + carry, Bresenham
// style); z crosses after j_z = q_1 + 1; the major axis runs out after km.
// Crossing k of minor 0 happens iff k <= K = min(kc_0, K_z), K_z being the
// number of minor-0 crossings before z's (from the sign of
// e12 + k ad_1 2^16), and J_k <= km.  Run k (k = 0, 1, ...) covers major
// counts J_k .. J_{k+1} (J_0 = 0) in row row_0 + k s_0 (s_0 the signed
// minor-0 row stride), the last ending at min(J_{k+1}, km, j_z) instead.
// These are exactly the runs run_next produces.  With kmz = min(km, j_z),
// run k is the last iff k = K or J_{k+1} > kmz (a crossing k + 1 <= K_z comes
// no later than z's), and it ends at min(J_{k+1}, kmz).
struct LeanWalk {
    unsigned ad, Ru, rem;  // |D_0|, |D_m| mod |D_0|, (rh_0 + k Ru_0) mod ad_0
    int jn;                // J_{k+1} (capped: any value above kmz acts alike)
    int Qu;                // floor(|D_m| / |D_0|), capped at kLeanQuCap
    int kmz;               // min(km, j_z)
    int kleft, K;          // crossings of minor 0 left, and in all
    int s;                 // J_k: where the current run starts
    int im0;               // major index of the first voxel
    int row;               // row of the current run (major axis' layout)
    int fl;                // bit 0 major +, bit 1 minor 0 +, bit 2 major is y, bit 3 empty
};
constexpr int kLeanWords = 8;   // packed size (32 bytes)
constexpr int kLeanQuCap = 8192;  // > any box extent (4096): one step beyond the box suffices
constexpr int kLeanJCap = 16383;

// The lean form of a freshly begun walk, when it has one.
HD_HD bool lean_of(const RunWalk &w, LeanWalk &L)
{
    const int fl = w.flags;
    if (fl & ((7 << 6) | (1 << 9))) return false;  // a tie pending, or empty
    const bool act0 = (fl >> 3) & 1, act1 = (fl >> 4) & 1;
    if (w.kc[1] != 0) return false;                            // z crosses inside the box
    if (!((fl >> 10) & 1) || !((fl >> 11) & 1)) return false;  // a tie with the major axis
    if (w.q[0] < -1 || w.q[1] < -1) return false;
    int kz;  // minor-0 crossings before z's
    if (!act0) {
        kz = 0;
    } else if (!act1) {
        kz = w.kc[0];
    } else {
        if ((w.e12 & 0xffff) == 0) return false;  // minor 0 and z may tie
        if (w.e12 > 0) {
            kz = 0;
        } else {
            // ceil(-e12 / step) = floor((-e12 - 1) / step) + 1 (e12 < 0), needed
            // only up to kc_0 <= 4096: a float estimate settles larger ones
            const long long step = static_cast<long long>(w.ad[1]) << 16;
            const long long num = -w.e12 - 1;
            if (float_of(num) >= (static_cast<float>(w.kc[0]) + 2.0f) * float_of(step)) {
                kz = w.kc[0];
            } else {
                const long long n = floordiv_small(num, step) + 1;
                kz = n < w.kc[0] ? static_cast<int>(n) : w.kc[0];
            }
        }
    }
    L.K = act0 ? (kz < w.kc[0] ? kz : w.kc[0]) : 0;
    L.kleft = L.K;
    const int jz = act1 ? w.q[1] + 1 : kQBig;
    L.kmz = w.km < jz ? w.km : jz;
    const int j1 = act0 ? w.q[0] + 1 : kQBig;
    L.jn = j1 < kLeanJCap ? j1 : kLeanJCap;
    L.Qu = w.Qu[0] < kLeanQuCap ? w.Qu[0] : kLeanQuCap;
    L.ad = w.ad[0];
    L.Ru = w.Ru[0];
    L.rem = w.rh[0];
    L.s = 0;
    L.im0 = w.im;
    L.row = w.row;
    L.fl = (fl & 3) | (((fl >> 5) & 1) << 2);
    return true;
}

HD_HD void lean_pack(const LeanWalk &L, uint32_t o[kLeanWords])
{
    o[0] = L.ad;
    o[1] = L.Ru;
    o[2] = L.rem;
    o[3] = static_cast<uint32_t>(L.jn) | (static_cast<uint32_t>(L.Qu) << 16);
    o[4] = static_cast<uint32_t>(L.kmz) | (static_cast<uint32_t>(L.K) << 16);
    o[5] = static_cast<uint32_t>(L.im0) | (static_cast<uint32_t>(L.fl) << 16);
    o[6] = static_cast<uint32_t>(L.row);
    o[7] = 0;
}

// The lean walk of the segment gi -> go (grid Q16, relative to the box
// origin) in a one-slice box [0, nx) x [0, ny) x [0, 1), computed directly:
// the same LeanWalk as lean_of(run_begin(...)) gives, without the general
// set-up's machinery.  In a one-slice box z never crosses inside (its only
// crossing ends the walk), the z index at the entry point is 0 or 1 (one
// comparison), the axis that sets the entry parameter needs no division,
// and z's crossing matters only through j_z, so its major-step quotient is
// not needed.  An axis moving - that enters through its upper face starts
// one voxel outside and takes that crossing first (as walk_begin does);
// when another axis moving - is exactly on a plane at the entry (a tie) or
// two axes enter that way, and for walks without in-plane motion, it
// returns -1 and the caller takes the general set-up.  Returns 1 (lean, L
// filled), 0 (no voxel in the box) or -1 (use run_begin and lean_of).
HD_HD int slab_lean(const int32_t gi[3], const int32_t go[3], int nx, int ny, LeanWalk &L)
{
    // 32-bit storage throughout (|P| < 2^30, |D| < 2^31, plane distances
    // below 2^31); only products are 64-bit
    const int P[3] = {gi[0], gi[1], gi[2]};
    const int D[3] = {go[0] - gi[0], go[1] - gi[1], go[2] - gi[2]};
    const int n[3] = {nx, ny, 1};
    const int H[3] = {nx << 16, ny << 16, 1 << 16};
    if (D[0] == 0 && D[1] == 0) return -1;
    // entry parameter tN / tQ (the largest per-axis entry) and its axis
    unsigned tN = 0, tQ = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        unsigned cN = 0, cQ = 1;
        bool cand = false;
        if (D[a] > 0) {
            if (P[a] >= H[a]) return 0;
            if (P[a] < 0) { cN = static_cast<unsigned>(-P[a]); cQ = static_cast<unsigned>(D[a]); cand = true; }
        } else if (D[a] < 0) {
            if (P[a] < 0) return 0;
            if (P[a] >= H[a]) { cN = static_cast<unsigned>(P[a] - H[a]); cQ = static_cast<unsigned>(-D[a]); cand = true; }
        } else if (P[a] < 0 || P[a] >= H[a]) {
            return 0;
        }
        if (cand && static_cast<unsigned long long>(cN) * tQ > static_cast<unsigned long long>(tN) * cQ) {
            tN = cN;
            tQ = cQ;
        }
    }
    if (tN > tQ) return 0;
    // voxel indices at the entry point, and whether that point lies on a
    // plane of each axis (remainder 0)
    int idx[3];
    bool onp[3];
    const long long den = static_cast<long long>(tQ) << 16;
    // the entry point's coordinate along each axis, P tQ + tN D over den
    // (also right for the entry axis and when the segment starts inside)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long num = static_cast<long long>(P[a]) * tQ + static_cast<long long>(tN) * D[a];
        if (a == 2) {
            idx[2] = num < 0 ? -1 : (num >= den ? 1 : 0);
            onp[2] = num == 0 || num == den;
        } else {
            const long long q = fdiv_small(num >> 16, static_cast<long long>(tQ));
            idx[a] = static_cast<int>(q);
            onp[a] = num == q * den;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if ((D[a] > 0 && idx[a] >= n[a]) || (D[a] < 0 && idx[a] < 0)) return 0;
    // an axis moving - that enters through its upper face starts one voxel
    // outside; its crossing at the entry parameter comes first unless another
    // axis moving - is on a plane there too (a tie: general set-up)
    int out = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (idx[a] >= n[a]) {
            if (out >= 0) return -1;
            out = a;
        }
    }
    if (out >= 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a != out && D[a] < 0 && onp[a]) return -1;
            if (a == out) idx[a] -= 1;
        }
    }
    // distances from the segment's start to each axis' next plane, and the
    // crossings left inside the box
    int nm[3], k[3];
    unsigned A[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int f = go[a] >> 16;
        const bool pos = D[a] > 0, neg = D[a] < 0;
        A[a] = pos ? static_cast<unsigned>(D[a]) : (neg ? static_cast<unsigned>(-D[a]) : 0u);
        nm[a] = pos ? ((idx[a] + 1) << 16) - P[a] : (neg ? P[a] - (idx[a] << 16) : 1);
        k[a] = pos ? (f < n[a] - 1 ? f : n[a] - 1) - idx[a] : (neg ? idx[a] - (f > 0 ? f : 0) : 0);
    }
    if (k[0] < 0 || k[1] < 0 || k[2] < 0) return 0;  // the walk ends where it enters
    if (k[2] != 0) return -1;
    // axes: major m, minor 0 (the other in-plane axis), minor 1 (z); every
    // array is read at constant indices (a runtime index would put it in
    // local memory)
    const bool ymaj = A[1] > A[0];
    const unsigned am = ymaj ? A[1] : A[0];
    const unsigned a0 = ymaj ? A[0] : A[1];
    const unsigned a1 = A[2];
    const long long nmm = ymaj ? nm[1] : nm[0], nmc = ymaj ? nm[0] : nm[1];
    const long long nmz = nm[2];
    // crossing-order terms against the major axis (D_c of run_begin), and
    // between the minors (e12); two axes that never move never cross
    const long long d0 = a0 == 0 ? -1 : nmc * am - nmm * a0;
    const long long d1 = a1 == 0 ? -1 : nmz * am - nmm * a1;
    const long long e12 = (a0 == 0 && a1 == 0) ? 1 : nmc * a1 - nmz * a0;
    const bool act0 = a0 != 0, act1 = a1 != 0;
    int q0 = kQBig, q1 = kQBig;
    unsigned rh0 = 0, Ru0 = 0;
    int Qu0 = kQBig;
    if (act0) {
        if ((d0 & 0xffff) == 0) return -1;  // minor 0 may tie with the major axis
        const unsigned qu = am / a0;
        Qu0 = qu >= (1u << 20) ? kQBig : static_cast<int>(qu);
        Ru0 = am - qu * a0;
        const long long dh = d0 >> 16;
        if (float_of(dh) >= 1048576.0f * static_cast<float>(a0)) {
            q0 = kQBig;
            rh0 = 1;
        } else {
            const long long q = fdiv_small(dh, static_cast<long long>(a0));
            q0 = static_cast<int>(q);
            rh0 = static_cast<unsigned>(dh - q * static_cast<long long>(a0));
        }
    }
    if (act1) {
        if ((d1 & 0xffff) == 0) return -1;  // z may tie with the major axis
        const long long dh = d1 >> 16;
        if (float_of(dh) >= 1048576.0f * static_cast<float>(a1)) {
            q1 = kQBig;
        } else {
            q1 = static_cast<int>(fdiv_small(dh, static_cast<long long>(a1)));
        }
    }
    if (q0 < -1 || q1 < -1) return -1;
    const int km = ymaj ? k[1] : k[0], kc0 = ymaj ? k[0] : k[1];
    int kz;  // minor-0 crossings before z's
    if (!act0) {
        kz = 0;
    } else if (!act1) {
        kz = kc0;
    } else {
        if ((e12 & 0xffff) == 0) return -1;  // minor 0 and z may tie
        if (e12 > 0) {
            kz = 0;
        } else {
            const long long step = static_cast<long long>(a1) << 16;
            const long long num = -e12 - 1;
            if (float_of(num) >= (static_cast<float>(kc0) + 2.0f) * float_of(step)) {
                kz = kc0;
            } else {
                const long long q = fdiv_small(num, step) + 1;
                kz = q < kc0 ? static_cast<int>(q) : kc0;
            }
        }
    }
    L.K = act0 ? (kz < kc0 ? kz : kc0) : 0;
    L.kleft = L.K;
    const int jz = act1 ? q1 + 1 : kQBig;
    L.kmz = km < jz ? km : jz;
    const int j1 = act0 ? q0 + 1 : kQBig;
    L.jn = j1 < kLeanJCap ? j1 : kLeanJCap;
    L.Qu = Qu0 < kLeanQuCap ? Qu0 : kLeanQuCap;
    L.ad = act0 ? a0 : 1u;
    L.Ru = Ru0;
    L.rem = rh0;
    L.s = 0;
    L.im0 = ymaj ? idx[1] : idx[0];
    L.row = ymaj ? idx[0] : idx[1];
    const bool pm = (ymaj ? D[1] : D[0]) > 0, pc = (ymaj ? D[0] : D[1]) > 0;
    L.fl = (pm ? 1 : 0) | ((pc ? 1 : 0) << 1) | ((ymaj ? 1 : 0) << 2);
    return 1;
}

// A packed walk with no voxel.
HD_HD void lean_pack_empty(uint32_t o[kLeanWords])
{
    for (int i = 0; i < kLeanWords; ++i) o[i] = 0;
    o[5] = 8u << 16;
}

HD_HD void lean_unpack(const uint32_t o[kLeanWords], LeanWalk &L)
{
    L.ad = o[0];
    L.Ru = o[1];
    L.rem = o[2];
    L.jn = static_cast<int>(o[3] & 0xffffu);
    L.Qu = static_cast<int>(o[3] >> 16);
    L.kmz = static_cast<int>(o[4] & 0xffffu);
    L.K = static_cast<int>(o[4] >> 16);
    L.kleft = L.K;
    L.im0 = static_cast<int>(o[5] & 0xffffu);
    L.fl = static_cast<int>(o[5] >> 16);
    L.row = static_cast<int>(o[6]);
    L.s = 0;
}

HD_HD bool lean_empty(const LeanWalk &L) { return (L.fl >> 3) & 1; }

// The traversal kernel's form of a lean walk: the same runs, with the row
// offset (row * nmaj), the run's start and the direction kept as signed
// increments so that a run costs a few integer operations.
struct LeanCursor {
    unsigned ad, Ru, rem;  // as in LeanWalk
    int jn, Qu, kmz, kleft;
    int im0, sg;  // major index of the first voxel, major direction (+1 or -1)
    int ms;       // major index where the current run starts
    int rb;       // row * nmaj of the current run
    int rstep;    // change of rb per minor-0 crossing (+nmaj or -nmaj)
};

// A packed lean walk as a cursor over rows of nmaj voxels (nmaj: the box's
// extent along the walk's major axis).  Returns false for an empty walk.
HD_HD bool lean_start(const uint32_t o[kLeanWords], int nmaj, LeanCursor &c)
{
    const int fl = static_cast<int>(o[5] >> 16);
    c.ad = o[0];
    c.Ru = o[1];
    c.rem = o[2];
    c.jn = static_cast<int>(o[3] & 0xffffu);
    c.Qu = static_cast<int>(o[3] >> 16);
    c.kmz = static_cast<int>(o[4] & 0xffffu);
    c.kleft = static_cast<int>(o[4] >> 16);
    c.im0 = static_cast<int>(o[5] & 0xffffu);
    c.sg = (fl & 1) ? 1 : -1;
    c.ms = c.im0;
    c.rb = static_cast<int>(o[6]) * nmaj;
    c.rstep = (fl & 2) ? nmaj : -nmaj;
    return !((fl >> 3) & 1);
}

// The current run: *rb its row offset, lo..hi its major range (inclusive).
// Returns whether more runs follow.  With the last run it adds e (the major
// count where the walk ends) to `ends`: the walk's voxel count is e plus its
// number of runs (see lean_step), so a caller that counts the runs gets the
// voxels as runs + ends.  Branch-free: the cursor also advances past the
// last run, where it is not used again.
HD_HD bool lean_run(LeanCursor &c, int &rb, int &lo, int &hi, unsigned &ends)
{
    const int jn = c.jn;
    const int e = jn < c.kmz ? jn : c.kmz;
    const int b = c.im0 + c.sg * e;
    lo = c.ms < b ? c.ms : b;
    hi = c.ms < b ? b : c.ms;
    rb = c.rb;
    const bool last = c.kleft == 0 || jn > c.kmz;
    ends += last ? static_cast<unsigned>(e) : 0u;
    c.ms = b;  // before the last run e = jn: the next run starts where this one ends
    const unsigned rem = c.rem + c.Ru;
    const bool carry = rem >= c.ad;
    c.rem = carry ? rem - c.ad : rem;
    c.jn = jn + c.Qu + (carry ? 1 : 0);
    --c.kleft;
    c.rb += c.rstep;
    return !last;
}

// The current run of a non-empty lean walk: row, and the inclusive range
// lo..hi of major indices.  Returns whether more runs follow; with the last
// run it adds the walk's voxel count (e + K + 1: the major cells covered
// plus one per row change) to `steps`.
HD_HD bool lean_step(LeanWalk &L, int &row, int &lo, int &hi, unsigned &steps)
{
    const int jn = L.jn;
    const int e = jn < L.kmz ? jn : L.kmz;
    const int a = (L.fl & 1) ? L.im0 + L.s : L.im0 - L.s;
    const int b = (L.fl & 1) ? L.im0 + e : L.im0 - e;
    lo = a < b ? a : b;
    hi = a < b ? b : a;
    row = L.row;
    if (L.kleft == 0 || jn > L.kmz) {
        steps += static_cast<unsigned>(e + (L.K - L.kleft) + 1);
        return false;
    }
    L.s = jn;
    const unsigned rem = L.rem + L.Ru;
    const bool carry = rem >= L.ad;
    L.rem = carry ? rem - L.ad : rem;
    L.jn = jn + L.Qu + (carry ? 1 : 0);
    --L.kleft;
    L.row += (L.fl & 2) ? 1 : -1;
    return true;
}

// The tiled traversal's form of a lean walk: the same runs as lean_run, as
// byte offsets into a tile box of dx x dy x dz voxels stored one 32-bit
// word per voxel, x fastest, with one padding column and one padding row:
// word(x, y, z) = x + Wx (y + Hy z), Wx = dx + 1, Hy = dy + 1.  A run adds
// inc (1 for runs along x, 65536 for runs along y: the two halves of a
// word) at its first voxel and subtracts it just past its last one, which
// for a run ending at the box's edge lies in the padding.  Consecutive runs
// share a major index (the walk changes row there), so a run is fixed by
// the major positions b_prev (where it starts in walk order) and b (where
// it ends): with the major axis moving +, inc goes at b_prev and -inc just
// past b; moving -, inc goes at b and -inc just past b_prev.  The cursor
// keeps the row base and the positions as byte offsets (plus a base the
// caller chooses, such as the tile's shared-memory address) and the two
// per-walk offsets and values that this choice implies, so a run costs a
// few integer steps and no comparison of its ends.
struct TileCursor {
    unsigned ad, Ru, rem;  // Bresenham state of minor 0 (as in LeanWalk)
    int jn, Qu, kmz, kleft;
    int m0b;    // byte offset of the first voxel's major index within its row
    int sgm;    // signed bytes per major step
    int bprev;  // byte offset of the current run's start (walk order) in its row
    int rowb;   // base + byte offset of the current row's major index 0
    int rstep;  // change of rowb per minor-0 crossing
    int oprev, ocur;     // byte offsets added to the run's ends: 0 or one major step
    uint32_t vprev, vcur;  // values added there: inc and -inc, in walk order
};

// Start a packed lean walk (lean_pack's form) in a box of dx x dy x dz
// voxels whose word 0 is at byte address `base`; false for an empty walk.
HD_HD bool tile_cursor_start(const uint32_t o[kLeanWords], int dx, int dy, int dz, int base,
                             TileCursor &c)
{
    const int fl = static_cast<int>(o[5] >> 16);
    const bool ymaj = (fl >> 2) & 1;
    const bool plus = fl & 1;
    const int Wx = dx + 1, Hy = dy + 1;
    c.ad = o[0];
    c.Ru = o[1];
    c.rem = o[2];
    c.jn = static_cast<int>(o[3] & 0xffffu);
    c.Qu = static_cast<int>(o[3] >> 16);
    c.kmz = static_cast<int>(o[4] & 0xffffu);
    c.kleft = static_cast<int>(o[4] >> 16);
    const int im0 = static_cast<int>(o[5] & 0xffffu);
    // the row in the major axis' layout of the box: x-major y + dy z,
    // y-major x + dx z; a lean walk never changes z
    const int row = static_cast<int>(o[6]);
    const int nminor = ymaj ? dx : dy;
    const int z = dz == 1 ? 0 : row / nminor;
    const int a = row - z * nminor;  // the minor-0 index (y for x-major, x for y-major)
    const int mstep = ymaj ? 4 * Wx : 4;
    c.sgm = plus ? mstep : -mstep;
    c.m0b = im0 * mstep;
    c.bprev = c.m0b;
    c.rowb = base + (ymaj ? 4 * (a + Wx * Hy * z) : 4 * Wx * (a + Hy * z));
    const int rs = ymaj ? 4 : 4 * Wx;
    c.rstep = (fl & 2) ? rs : -rs;
    const uint32_t inc = ymaj ? 65536u : 1u;
    c.oprev = plus ? 0 : mstep;
    c.ocur = plus ? mstep : 0;
    c.vprev = plus ? inc : 0u - inc;
    c.vcur = plus ? 0u - inc : inc;
    return !((fl >> 3) & 1);
}

// The current run: vprev is added at byte address `at_prev` and vcur at
// `at_cur`.  Returns whether more runs follow.  Past its last run the
// cursor holds kleft = (crossings left at the start) - (runs walked).
HD_HD bool tile_cursor_run(TileCursor &c, int &at_prev, int &at_cur)
{
    const int jn = c.jn;
    const int e = jn < c.kmz ? jn : c.kmz;
    const int b = c.m0b + c.sgm * e;
    at_prev = c.rowb + c.bprev + c.oprev;
    at_cur = c.rowb + b + c.ocur;
    const bool last = c.kleft == 0 || jn > c.kmz;
    c.bprev = b;  // the next run starts where this one ends (in the next row)
    const unsigned rem = c.rem + c.Ru;
    const bool carry = rem >= c.ad;
    c.rem = carry ? rem - c.ad : rem;
    c.jn = jn + c.Qu + (carry ? 1 : 0);
    --c.kleft;
    c.rowb += c.rstep;
    return !last;
}

// Packed run-walk state: 16 32-bit words, so a walk prepared by one kernel
// can be resumed by another.  The row strides and the major size follow
// from the box (nx, ny) and the flags.
constexpr int kPackedWords = 16;

HD_HD void run_pack(const RunWalk &w, uint32_t o[kPackedWords])
{
    o[0] = static_cast<uint32_t>(static_cast<unsigned long long>(w.e12) & 0xffffffffull);
    o[1] = static_cast<uint32_t>(static_cast<unsigned long long>(w.e12) >> 32);
    o[2] = static_cast<uint32_t>(w.q[0]);
    o[3] = static_cast<uint32_t>(w.q[1]);
    o[4] = w.rh[0];
    o[5] = w.rh[1];
    o[6] = w.ad[0];
    o[7] = w.ad[1];
    o[8] = static_cast<uint32_t>(w.Qu[0]);
    o[9] = static_cast<uint32_t>(w.Qu[1]);
    o[10] = w.Ru[0];
    o[11] = w.Ru[1];
    o[12] = static_cast<uint32_t>(w.row);
    o[13] = (static_cast<uint32_t>(w.im) & 0xffffu) | (static_cast<uint32_t>(w.km) << 16);
    o[14] = (static_cast<uint32_t>(w.kc[0]) & 0xffffu) | (static_cast<uint32_t>(w.kc[1]) << 16);
    o[15] = static_cast<uint32_t>(w.flags);
}

// A packed state that yields no run.
HD_HD void run_pack_empty(uint32_t o[kPackedWords])
{
    for (int i = 0; i < kPackedWords; ++i) o[i] = 0;
    o[15] = 1u << 9;
}

HD_HD void run_unpack(const uint32_t o[kPackedWords], int nx, int ny, RunWalk &w)
{
    w.e12 = static_cast<long long>((static_cast<unsigned long long>(o[1]) << 32) | o[0]);
    w.q[0] = static_cast<int>(o[2]);
    w.q[1] = static_cast<int>(o[3]);
    w.rh[0] = o[4];
    w.rh[1] = o[5];
    w.ad[0] = o[6];
    w.ad[1] = o[7];
    w.Qu[0] = static_cast<int>(o[8]);
    w.Qu[1] = static_cast<int>(o[9]);
    w.Ru[0] = o[10];
    w.Ru[1] = o[11];
    w.row = static_cast<int>(o[12]);
    w.im = static_cast<int>(o[13] & 0xffffu);
    w.km = static_cast<int>(o[13] >> 16);
    w.kc[0] = static_cast<int>(o[14] & 0xffffu);
    w.kc[1] = static_cast<int>(o[14] >> 16);
    w.flags = static_cast<int>(o[15]);
    const bool ymaj = (w.flags >> 5) & 1;
    w.run_start = w.im;
    w.rstride[0] = (w.flags & 2) ? 1 : -1;
    w.rstride[1] = (w.flags & 4) ? (ymaj ? nx : ny) : -(ymaj ? nx : ny);
    w.nmaj = ymaj ? ny : nx;
}

// Call visit(v) for every voxel of the set in traversal order; returns |A_i|.
template <class VisitT>
HD_HD unsigned walk_all(const int32_t gi[3], const int32_t go[3], int nx, int ny, int nz,
                        const VisitT &visit)
{
    Walk w;
    if (!walk_begin(w, gi, go, nx, ny, nz)) return 0;
    unsigned c = 0;
    do {
        visit(static_cast<uint32_t>(w.idx));
        ++c;
    } while (walk_next(w));
    return c;
}

}  // namespace hd
