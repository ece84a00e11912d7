// Thick rays by the Euclidean distance of Eq. 3.2 (d_0 > 0, d the distance
// from a voxel's centre to the closed segment L_i, Sec. 2.1): the row search
// of one history's capsule (host and device, so that the host test suite can
// check it against a voxel-by-voxel search).
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
// Float filter.  Most membership tests are settled in float32 with bounds
// that make the answer certain; the exact test above runs only for centres
// whose float distance falls in a narrow band around R.  In float, t is the
// clamped parameter of the point of the segment nearest C and e = w - t u:
//  * |e| bounds the distance from above for any t in [0, 1] (A + t u is a
//    point of the segment), and the computed |e| differs from the exact one
//    by at most 3.02 eps S (eps = 2^-24; S the sum over the axes of the
//    largest |w| a tested centre can have, the grid's doubled extent along
//    the row axis and |u|), so a computed |e|^2 below (R - 2^-19 S)^2
//    (1 - 2^-19) certifies C inside;
//  * the exact distance is at least |w - t u|^2 - G^2 with G <= 10.5 eps S
//    (t is within 6.1 eps S / |u| of the nearest point's parameter: its dot
//    product is off by at most 6.1 eps S |u|), so a computed |e|^2 above
//    (R + 2^-19 S)^2 (1 + 2^-19) certifies C outside.
// Float coordinates are formed without conversions of wide integers: the
// coordinate of index j along an axis is w at index 0 (rounded once) plus
// j times the exact step 2 s2, in one fused multiply-add.
// The margins 2^-19 S = 32 eps S cover both bounds and the rounding of the
// thresholds themselves.
//
// Rows.  A row is the line of voxel centres along the capsule's major
// in-plane axis (axis 0) at fixed indices a (axis 1) and k (z).  Along it F
// is convex, so the row's part of the set is one interval: a float estimate
// of the capsule's cross-section gives starting indices, and membership tests
// settle both ends (a boundary i with i inside and the neighbour outside),
// or, when the estimate finds no voxel, an exact descent to F's minimum along
// the row decides whether the row has any.  The float estimate only chooses
// where the tests start, never a result.
#pragma once

#include <cmath>
#include <cstdint>

#include "hd_geom.cuh"

namespace hd {
namespace {

typedef unsigned __int128 u128;

// Full product of two 64-bit unsigned values (two multiplies, not a general
// 128 x 128 one).
HD_HD u128 mul64(unsigned long long a, unsigned long long b)
{
    return (static_cast<u128>(umulhi64(a, b)) << 64) | static_cast<u128>(a * b);
}

HD_HD u128 sq64(long long a)
{
    const unsigned long long m = static_cast<unsigned long long>(a < 0 ? -a : a);
    return mul64(m, m);
}

// j as a float for |j| < 2^22, exact, with integer and float additions only
// (no conversion instruction).
HD_HD float float_small(int j)
{
#ifdef __CUDA_ARCH__
    return __int_as_float(0x4B400000 + j) - 12582912.0f;
#else
    return static_cast<float>(j);
#endif
}

// Approximate square root and reciprocal: they only place the estimate.
HD_HD float sqrt_est(float x)
{
#ifdef __CUDA_ARCH__
    return __fsqrt_rz(x);
#else
    return std::sqrt(x);
#endif
}

HD_HD float rcp_est(float x)
{
#ifdef __CUDA_ARCH__
    return __frcp_rz(x);
#else
    return 1.0f / x;
#endif
}

// Correctly rounded reciprocal (the filter's bound on t assumes it).
HD_HD float rcp_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __frcp_rn(x);
#else
    return 1.0f / x;
#endif
}

// One history's capsule in the permuted frame (axis 0 the major in-plane
// axis, 1 the other in-plane axis, 2 z), in two parts: the exact values,
// read only by the exact tests (kept once per warp in shared memory on the
// device), and the float values of the filter and the estimate (kept in
// registers).  All in doubled Q16 units.
struct CapX {
    long long A[3], B[3], u[3];
    unsigned long long uu;   // |u|^2 (< 3 2^62)
    unsigned long long uu2;  // u_1^2 + u_2^2: the segment projected along axis 0
    unsigned long long RR;   // R^2
    u128 T;                  // the threshold R^2 |u|^2 (or R^2 when u = 0)
    u128 T2;                 // R^2 uu2
    int n[3];
    long long s2[3];  // voxel sizes, mm * 2^16 (centres are (2 i + 1 - n) s2)
};

struct CapF {
    float uf[3];      // u
    float uuf;        // |u|^2
    float inv_uu;     // 1 / |u|^2 (0 when u = 0)
    float inv_uu2;    // 1 / (u_1^2 + u_2^2) (0 when that is 0)
    float inv_u0;     // 1 / u_0 (estimate only; 0 when u_0 = 0)
    float wb[3];      // w at index 0 along each axis: (1 - n) s2 - A
    float step[3];    // 2 s2, the step of w per index (exact)
    float inv_step0;  // 1 / step[0] (estimate only)
    float Rf;         // R (exact)
    float Tin, Tout;  // certain inside at or below Tin, outside above Tout
    float margin;     // 2^-19 S
    int n0;           // centres along a row
    // the band of rows that can meet the capsule (k_range)
    float ratio;      // u_2 / u_1
    float Hk;         // R sqrt(1 + ratio^2) plus the error margin
    float inv_step2;  // 1 / step[2]
    bool kband;       // |u_2| <= 4 |u_1| and u_1 != 0 (else the whole box)
};

// The float constants of row (a, k).
struct RowF {
    float wc, wz, dot;  // w on axes 1 and 2, and w.u restricted to them
    int a, k;
};

HD_HD RowF rowf_of(const CapF &cf, int a, int k)
{
    RowF r;
    r.wc = fmaf(float_small(a), cf.step[1], cf.wb[1]);
    r.wz = fmaf(float_small(k), cf.step[2], cf.wb[2]);
    r.dot = fmaf(r.wc, cf.uf[1], r.wz * cf.uf[2]);
    r.a = a;
    r.k = k;
    return r;
}

// The exact constants of row (a, k): C - A and C - B on axes 1 and 2, the
// plane's dot product with u, the squared distances to A and B in that
// plane, and the cross component without the major axis.
struct RowX {
    long long wc, wz, wbc, wbz;
    __int128 dot0;
    unsigned long long hA, hB;
    long long k0;
};

HD_HD RowX rowx_of(const CapX &cx, int a, int k)
{
    RowX r;
    const long long cc = (2LL * a + 1 - cx.n[1]) * cx.s2[1];
    const long long cz = (2LL * k + 1 - cx.n[2]) * cx.s2[2];
    r.wc = cc - cx.A[1];
    r.wz = cz - cx.A[2];
    r.wbc = cc - cx.B[1];
    r.wbz = cz - cx.B[2];
    r.dot0 = static_cast<__int128>(r.wc) * cx.u[1] + static_cast<__int128>(r.wz) * cx.u[2];
    r.hA = static_cast<unsigned long long>(r.wc * r.wc) + static_cast<unsigned long long>(r.wz * r.wz);
    r.hB = static_cast<unsigned long long>(r.wbc * r.wbc) +
           static_cast<unsigned long long>(r.wbz * r.wbz);
    r.k0 = r.wc * cx.u[2] - r.wz * cx.u[1];
    return r;
}

// F at index i of row (a, k) (see the file comment).  Out of line on the
// device: the exact tests are rare, and one copy of the 128-bit arithmetic
// serves all of them.
__host__ __device__ __noinline__ u128 F_exact(const CapX &cx, int a, int k, int i)
{
    const RowX r = rowx_of(cx, a, k);
    const long long cm = (2LL * i + 1 - cx.n[0]) * cx.s2[0];
    const long long wm = cm - cx.A[0];
    if (cx.uu == 0) return static_cast<u128>(static_cast<unsigned long long>(wm * wm) + r.hA);
    const __int128 dot = r.dot0 + static_cast<__int128>(wm) * cx.u[0];
    if (dot <= 0) return mul64(static_cast<unsigned long long>(wm * wm) + r.hA, cx.uu);
    if (dot >= static_cast<__int128>(cx.uu)) {
        const long long wbm = cm - cx.B[0];
        return mul64(static_cast<unsigned long long>(wbm * wbm) + r.hB, cx.uu);
    }
    const long long k1 = r.wz * cx.u[0] - wm * cx.u[2];
    const long long k2 = wm * cx.u[1] - r.wc * cx.u[0];
    return sq64(r.k0) + sq64(k1) + sq64(k2);
}

// Does row (a, k) meet the capsule at all?  The row is a line along axis 0,
// so it does iff its point in the plane of axes 1 and 2 lies within R of
// the segment's projection onto that plane (the projection of the capsule is
// the disc-swept projected segment): the same three cases in two dimensions,
// with the row's constants (dot0 and k0 are that plane's dot and cross).
__host__ __device__ __noinline__ bool meets_exact(const CapX &cx, int a, int k)
{
    const RowX r = rowx_of(cx, a, k);
    if (cx.uu2 == 0 || r.dot0 <= 0) return r.hA <= cx.RR;
    if (r.dot0 >= static_cast<__int128>(cx.uu2)) return r.hB <= cx.RR;
    return sq64(r.k0) <= cx.T2;
}

// The float filter's squared distance of centre i of the row, and the
// component e_0 along the row (see the file comment for its bounds).
HD_HD float d2_filter(const CapF &cf, const RowF &r, int i, float &e0)
{
    const float w0 = fmaf(float_small(i), cf.step[0], cf.wb[0]);
    const float dot = fmaf(w0, cf.uf[0], r.dot);
    const float t = fminf(fmaxf(dot * cf.inv_uu, 0.0f), 1.0f);
    e0 = fmaf(-t, cf.uf[0], w0);
    const float e1 = fmaf(-t, cf.uf[1], r.wc);
    const float e2 = fmaf(-t, cf.uf[2], r.wz);
    return fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
}

// Is centre i of the row inside?  Exact: the float filter answers where its
// bounds make the answer certain, the exact F otherwise.
HD_HD bool in_at(const CapF &cf, const CapX &cx, const RowF &r, int i)
{
    float e0;
    const float d2 = d2_filter(cf, r, i, e0);
    if (d2 <= cf.Tin) return true;
    if (d2 > cf.Tout) return false;
    return F_exact(cx, r.a, r.k, i) <= cx.T;
}

// Certifies from the float filter alone that no centre of the row is inside,
// looking at centres j - 1, j, j + 1 (those in the row): all three outside,
// and the distance falling at the first and rising at the last (unless it is
// the row's end).  Along the row the squared distance to the segment is
// convex and continuously differentiable, its slope of the sign of e_0 (the
// row component of C minus its nearest point), and the computed e_0 is
// within 9.1 eps S of the exact one (the filter's bounds on w and on t), so
// |e_0| above the margin fixes the sign; then every centre beyond the three
// is farther out than the nearest of them.  False means not certified.
HD_HD bool row_empty(const CapF &cf, const RowF &r, int j)
{
    const int n = cf.n0;
    const int lo = j > 0 ? j - 1 : 0, hi = j + 1 < n ? j + 1 : n - 1;
    float e_lo = 0.0f, e_hi = 0.0f;
    for (int i = lo; i <= hi; ++i) {
        float e0;
        if (!(d2_filter(cf, r, i, e0) > cf.Tout)) return false;
        if (i == lo) e_lo = e0;
        if (i == hi) e_hi = e0;
    }
    return (lo == 0 || e_lo < -cf.margin) && (hi == n - 1 || e_hi > cf.margin);
}

// meets_exact with the float filter in front: the same bounds hold in the
// plane of axes 1 and 2 (the terms of axis 0 dropped), and the exact test
// runs only inside the band.
HD_HD bool row_meets_at(const CapF &cf, const CapX &cx, int a, int k)
{
    const RowF r = rowf_of(cf, a, k);
    const float t = fminf(fmaxf(r.dot * cf.inv_uu2, 0.0f), 1.0f);
    const float e1 = fmaf(-t, cf.uf[1], r.wc);
    const float e2 = fmaf(-t, cf.uf[2], r.wz);
    const float d2 = fmaf(e2, e2, e1 * e1);
    if (d2 <= cf.Tin) return true;
    if (d2 > cf.Tout) return false;
    return meets_exact(cx, a, k);
}

// Float estimate of the row's cross-section of the capsule, as a range of
// major indices (lo > hi when the estimate finds none); also a float guess
// of where along the row the distance is smallest.  Positions x along the
// row are measured from A_0.
HD_HD void estimate(const CapF &cf, const RowF &r, int &ilo, int &ihi, int &imin)
{
    // approximate arithmetic throughout (fast square roots and quotients):
    // these numbers only choose where the membership tests start
    const float wc = r.wc, wz = r.wz;
    const float R2 = cf.Rf * cf.Rf;
    float lo = INFINITY, hi = -INFINITY;
    // the caps: balls around A and B
    const float hA = wc * wc + wz * wz;
    if (hA <= R2) {
        const float s = sqrt_est(R2 - hA);
        lo = fminf(lo, -s);
        hi = fmaxf(hi, s);
    }
    const float bc = wc - cf.uf[1], bz = wz - cf.uf[2];
    const float hB = bc * bc + bz * bz;
    if (hB <= R2) {
        const float s = sqrt_est(R2 - hB);
        lo = fminf(lo, cf.uf[0] - s);
        hi = fmaxf(hi, cf.uf[0] + s);
    }
    // the position of the point nearest the segment's line
    float smin = 0.0f;
    if (cf.uuf > 0.0f) {
        const float g = r.dot;
        const float a2 = 1.0f - cf.uf[0] * cf.uf[0] * cf.inv_uu;
        const float b = -cf.uf[0] * g * cf.inv_uu;
        const float c0 = hA - g * g * cf.inv_uu;
        // the parameter along the segment stays in [0, 1]
        float tlo = -INFINITY, thi = INFINITY;
        if (cf.uf[0] != 0.0f) {
            const float t0 = -g * cf.inv_u0, t1 = (cf.uuf - g) * cf.inv_u0;
            tlo = fminf(t0, t1);
            thi = fmaxf(t0, t1);
        } else if (g < 0.0f || g > cf.uuf) {
            tlo = INFINITY;  // the row never faces the segment's interior
        }
        if (a2 > 1e-6f) {
            const float ia = rcp_est(a2);
            smin = -b * ia;
            const float disc = b * b - a2 * (c0 - R2);
            if (disc >= 0.0f) {
                const float q = sqrt_est(disc);
                const float s1 = fmaxf((-b - q) * ia, tlo), s2 = fminf((-b + q) * ia, thi);
                if (s1 <= s2) {
                    lo = fminf(lo, s1);
                    hi = fmaxf(hi, s2);
                }
            }
        } else {
            smin = 0.5f * cf.uf[0];
            if (c0 <= R2 && tlo <= thi) {
                lo = fminf(lo, tlo);
                hi = fmaxf(hi, thi);
            }
        }
        smin = fminf(fmaxf(smin, fminf(0.0f, cf.uf[0])), fmaxf(0.0f, cf.uf[0]));
    }
    // index of a position x: x = wb_0 + i step_0
    const float flo = (lo - cf.wb[0]) * cf.inv_step0, fhi = (hi - cf.wb[0]) * cf.inv_step0;
    const float fm = (smin - cf.wb[0]) * cf.inv_step0;
    const float top = float_small(cf.n0 - 1);
    ilo = static_cast<int>(ceilf(fminf(fmaxf(flo, -1.0f), top + 1.0f)));
    ihi = static_cast<int>(floorf(fminf(fmaxf(fhi, -1.0f), top + 1.0f)));
    if (!(lo <= hi)) {
        ilo = 1;
        ihi = 0;
    }
    imin = static_cast<int>(rintf(fminf(fmaxf(fm, 0.0f), top)));
}

// The exact interval [lo, hi] of voxels of row (a, k) inside the capsule
// (false when no voxel centre of the row lies inside: the row may miss the
// capsule, or its chord fall between two centres).
HD_HD bool row_interval(const CapF &cf, const CapX &cx, int a, int k, int &lo, int &hi)
{
    const int n = cf.n0;
    const RowF r = rowf_of(cf, a, k);
    int elo, ehi, emin;
    estimate(cf, r, elo, ehi, emin);
    elo = elo < 0 ? 0 : (elo > n - 1 ? n - 1 : elo);
    ehi = ehi < 0 ? 0 : (ehi > n - 1 ? n - 1 : ehi);
    int m = -1;
    if (elo <= ehi) {
        // the usual case: both estimated ends inside, their outer
        // neighbours outside (convexity: exactly [elo, ehi]); otherwise
        // settle the ends below from an inside point
        const bool in_lo = in_at(cf, cx, r, elo);
        const bool in_hi = in_lo && (ehi == elo || in_at(cf, cx, r, ehi));
        if (in_hi) {
            if ((elo == 0 || !in_at(cf, cx, r, elo - 1)) &&
                (ehi + 1 >= n || !in_at(cf, cx, r, ehi + 1))) {
                lo = elo;
                hi = ehi;
                return true;
            }
            m = elo;
        } else if (in_lo) {
            m = elo;
        } else {
            const int mid = (elo + ehi) >> 1;
            if (in_at(cf, cx, r, mid)) m = mid;
            else emin = mid;
        }
    }
    if (m < 0) {
        if (row_empty(cf, r, emin)) return false;
        // exact descent to F's minimum along the row (F is convex in i)
        int i = emin;
        u128 f = F_exact(cx, a, k, i);
        if (i > 0 && F_exact(cx, a, k, i - 1) < f) {
            for (--i, f = F_exact(cx, a, k, i); i > 0;) {
                const u128 g = F_exact(cx, a, k, i - 1);
                if (!(g < f)) break;
                --i;
                f = g;
            }
        } else {
            for (; i + 1 < n;) {
                const u128 g = F_exact(cx, a, k, i + 1);
                if (!(g < f)) break;
                ++i;
                f = g;
            }
        }
        if (f > cx.T) return false;  // no voxel centre of the row is inside
        m = i;
        elo = ehi = i;
    }
    // both ends, starting from the estimates (centre m is inside)
    lo = elo < m ? (elo < 0 ? 0 : elo) : m;
    if (in_at(cf, cx, r, lo)) {
        while (lo > 0 && in_at(cf, cx, r, lo - 1)) --lo;
    } else {
        do ++lo;
        while (!in_at(cf, cx, r, lo));
    }
    hi = ehi > m ? (ehi > n - 1 ? n - 1 : ehi) : m;
    if (in_at(cf, cx, r, hi)) {
        while (hi + 1 < n && in_at(cf, cx, r, hi + 1)) ++hi;
    } else {
        do --hi;
        while (!in_at(cf, cx, r, hi));
    }
    return true;
}

HD_HD long long abs_ll(long long v) { return v < 0 ? -v : v; }
HD_HD int max_i(int a, int b) { return a > b ? a : b; }
HD_HD int min_i(int a, int b) { return a < b ? a : b; }

// floor(v / s) for s > 0 (|v| < 2^62).
HD_HD long long floor_div(long long v, long long s)
{
    return v >= 0 ? v / s : -((-v + s - 1) / s);
}

// The frame of one history's capsule from its world endpoints W (mm * 2^16,
// as world_cs gives them) and R = 2 q16(d_0): the doubled endpoints A, B in
// the permuted frame, whether rows run along y (else x), the index box of
// the rows that can meet the capsule on axes 1 and 2 ([blo, bhi]; false when
// empty), and S of the float filter.
HD_HD bool capsule_frame(const GeomQ &g, const long long W[6], long long R, long long A[3],
                         long long B[3], bool &ymaj, int blo[3], int bhi[3], float &S)
{
    long long P[3], Q[3];
    for (int q = 0; q < 3; ++q) {
        P[q] = 2 * W[q];
        Q[q] = 2 * W[q + 3];
    }
    // the major in-plane axis (rows run along it): frame axes 0, 1, 2 are
    // (x, y, z) or (y, x, z), chosen with selects (a runtime array index
    // would put the arrays in local memory)
    const bool mj = abs_ll(Q[1] - P[1]) > abs_ll(Q[0] - P[0]);
    ymaj = mj;
    A[0] = mj ? P[1] : P[0];
    A[1] = mj ? P[0] : P[1];
    A[2] = P[2];
    B[0] = mj ? Q[1] : Q[0];
    B[1] = mj ? Q[0] : Q[1];
    B[2] = Q[2];
    const int n[3] = {mj ? g.ny : g.nx, mj ? g.nx : g.ny, g.nz};
    const long long s2[3] = {mj ? g.sy : g.sx, mj ? g.sx : g.sy, g.sz};
    // S: per axis the largest |w| over the grid's centres, plus |u|, plus
    // the row axis' doubled extent
    long long s = 2LL * n[0] * s2[0];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const long long c0 = (1LL - n[q]) * s2[q], c1 = (n[q] - 1LL) * s2[q];
        const long long w0 = abs_ll(c0 - A[q]), w1 = abs_ll(c1 - A[q]);
        s += (w0 > w1 ? w0 : w1) + abs_ll(B[q] - A[q]);
    }
    S = static_cast<float>(s);
    // index box of the capsule on axes 1 and 2: centres within
    // [min(A, B) - R, max(A, B) + R], widened by one
#pragma unroll
    for (int q = 1; q < 3; ++q) {
        const long long mn = (A[q] < B[q] ? A[q] : B[q]) - R;
        const long long mx = (A[q] > B[q] ? A[q] : B[q]) + R;
        const long long fl = floor_div(mn, s2[q]), fh = floor_div(mx, s2[q]);
        const long long l = (fl + n[q] - 1) / 2 - 1, h = (fh + n[q] + 1) / 2 + 1;
        blo[q] = static_cast<int>(l > 0 ? l : 0LL);
        bhi[q] = static_cast<int>(h < n[q] - 1 ? h : static_cast<long long>(n[q] - 1));
    }
    return blo[1] <= bhi[1] && blo[2] <= bhi[2];
}

// The exact part of the capsule of endpoints A, B (capsule_frame's frame).
HD_HD void capx_of(const GeomQ &g, const long long A[3], const long long B[3], bool ymaj,
                   long long R, CapX &cx)
{
    cx.n[0] = ymaj ? g.ny : g.nx;
    cx.n[1] = ymaj ? g.nx : g.ny;
    cx.n[2] = g.nz;
    cx.s2[0] = ymaj ? g.sy : g.sx;
    cx.s2[1] = ymaj ? g.sx : g.sy;
    cx.s2[2] = g.sz;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        cx.A[q] = A[q];
        cx.B[q] = B[q];
        cx.u[q] = B[q] - A[q];
    }
    cx.uu = static_cast<unsigned long long>(cx.u[0] * cx.u[0]) +
            static_cast<unsigned long long>(cx.u[1] * cx.u[1]) +
            static_cast<unsigned long long>(cx.u[2] * cx.u[2]);
    cx.RR = static_cast<unsigned long long>(R * R);
    cx.T = cx.uu == 0 ? static_cast<u128>(cx.RR) : mul64(cx.RR, cx.uu);
    cx.uu2 = static_cast<unsigned long long>(cx.u[1] * cx.u[1]) +
             static_cast<unsigned long long>(cx.u[2] * cx.u[2]);
    cx.T2 = mul64(cx.RR, cx.uu2);
}

// The float part of the capsule: from its exact part, S and R.
HD_HD CapF capf_of(const CapX &cx, float S, long long R)
{
    CapF cf;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        cf.uf[q] = static_cast<float>(cx.u[q]);
        cf.wb[q] = static_cast<float>((1LL - cx.n[q]) * cx.s2[q] - cx.A[q]);
        cf.step[q] = static_cast<float>(2 * cx.s2[q]);
    }
    cf.uuf = static_cast<float>(cx.uu);
    cf.inv_uu = cx.uu == 0 ? 0.0f : rcp_rn(cf.uuf);
    cf.inv_uu2 = cx.uu2 == 0 ? 0.0f : rcp_rn(static_cast<float>(cx.uu2));
    cf.inv_u0 = cx.u[0] != 0 ? rcp_est(cf.uf[0]) : 0.0f;
    cf.inv_step0 = rcp_est(cf.step[0]);
    cf.n0 = cx.n[0];
    cf.Rf = static_cast<float>(R);  // exact (R < 2^24)
    const float m = S * (1.0f / 524288.0f);  // 2^-19 S
    const float lo = cf.Rf - m, hi = cf.Rf + m;
    cf.margin = m;
    cf.Tin = lo > 0.0f ? (lo * lo) * (1.0f - 1.0f / 524288.0f) : -1.0f;
    cf.Tout = (hi * hi) * (1.0f + 1.0f / 524288.0f);
    const float au1 = fabsf(cf.uf[1]), au2 = fabsf(cf.uf[2]);
    cf.kband = cx.u[1] != 0 && au2 <= 4.0f * au1;
    cf.ratio = cf.kband ? cf.uf[2] * rcp_est(cf.uf[1]) : 0.0f;
    cf.Hk = cf.Rf * sqrt_est(1.0f + cf.ratio * cf.ratio) + (S + cf.Rf) * (1.0f / 65536.0f);
    cf.inv_step2 = rcp_est(cf.step[2]);
    return cf;
}

// The rows (a, k) of the capsule's index box that can meet it, for one a:
// k in [klo, khi] (empty when klo > khi).  A row meets the capsule only if
// its point lies within R of the projected segment's line in the plane of
// axes 1 and 2, that is within R sqrt(1 + r^2) of it along axis 2 (r the
// line's slope u_2 / u_1).  In float, with |r| <= 4, the line's height at
// the row, that distance and the division into indices are off by less
// than 100 eps (S + R) together, so widening the distance by 2^-16 (S + R)
// makes [klo, khi] a superset of the meeting rows; steeper or axis-parallel
// projections take the whole box.
HD_HD void k_range(const CapF &cf, int a, int blo2, int bhi2, int &klo, int &khi)
{
    if (!cf.kband) {
        klo = blo2;
        khi = bhi2;
        return;
    }
    const float wc = fmaf(float_small(a), cf.step[1], cf.wb[1]);
    const float zc = wc * cf.ratio;
    const float fb = float_small(blo2 - 1), ft = float_small(bhi2 + 1);
    const float lo = fminf(fmaxf((zc - cf.Hk - cf.wb[2]) * cf.inv_step2, fb), ft);
    const float hi = fminf(fmaxf((zc + cf.Hk - cf.wb[2]) * cf.inv_step2, fb), ft);
    klo = max_i(blo2, static_cast<int>(ceilf(lo)));
    khi = min_i(bhi2, static_cast<int>(floorf(hi)));
}

}  // namespace
}  // namespace hd
