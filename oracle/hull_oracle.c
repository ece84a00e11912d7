/*
 * CPU oracle for proton-CT hull detection (SC, MSC, SM).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the hull-detection path computes.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline arm may load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What is computed, and where it comes from:
 *   - Classification of a history as missed (WEPL below a cutoff) or hit
 *     (WEPL above a cutoff): Eq. 3.1 and Eq. 3.7, with the paper's cutoffs
 *     1.0 mm and 5.0 mm on individual WEPL values and no angular cutoff
 *     (Sec. 3.2 last paragraph, Sec. 3.3 last paragraph, Sec. 3.4 last
 *     paragraph).
 *   - The path L_i is the straight segment joining the entry and exit points
 *     (Sec. 2.1 and the definition of L_i before Eq. 3.2).  The voxel set
 *     A_i = {v : d(L_i, v) <= d_0} (Eq. 3.2) is read with d_0 = 0 against the
 *     half-open voxel cube: A_i is the set of voxels whose cube
 *     [k, k+1)^3 (in voxel units) contains a point of the closed segment.
 *     This matches the 0/1 system-matrix rows of "intersected voxels"
 *     (Sec. 2.1).  Geometry is made exact by one rounding of the float32
 *     inputs to 16 fractional bits, an integer CORDIC for the gantry
 *     rotation, and integer floor divisions; after that every step is exact.
 *   - N(v) = |C(v)| over missed histories (Eq. 3.4), M(v) = |C(v)| over hit
 *     histories (Eq. 3.9), H_1 = V minus the union of A_i (Eq. 3.3, Alg. 1),
 *     H_2 by the neighbour-difference threshold N_t (Eq. 3.5, Eq. 3.6,
 *     Alg. 2), H_3 by the steepest-edge threshold M_t (Eq. 3.10, Alg. 3,
 *     made per slice as Sec. 3.4 describes).
 *
 * The voxel set is enumerated from its definition: the voxel function
 * floor(P(t)) of the segment P(t) = G_in + t (G_out - G_in), t in [0, 1], is
 * constant between consecutive parameters at which some coordinate crosses a
 * grid plane, so the set is the voxels at those parameters and at the
 * midpoints between them.  All parameters are exact rationals.  A second,
 * independent statement (the per-voxel slab test) checks it on small grids.
 *
 * Reported only (not a parity reference): the same set definition on
 * unquantised FP64 geometry, to measure how many voxel memberships and
 * hull voxels the fixed-point geometry changes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef __int128 i128;

#define Q16 65536LL

/* ------------------------------------------------------------ quantisation */

/* Round a float32 to 16 fractional bits, ties to even.  The float32 -> double
 * conversion and the multiplication by 2^16 are exact, so the only rounding
 * is the final one. */
static int64_t q16_of(float x) { return (int64_t)llrint((double)x * 65536.0); }

static int64_t floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static i128 floordiv128(i128 a, i128 b) /* b > 0 */
{
    i128 q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

/* ----------------------------------------------------------------- CORDIC */

/* Rotation-mode CORDIC (Volder 1959) of the angle a (degrees, 16 fractional
 * bits).  theta[i] = round(atan(2^-i) * 180/pi * 2^30) and
 * K = round(2^30 * prod_i (1 + 2^-2i)^(-1/2)) are supplied by the caller.
 * Returns cos and sin with 30 fractional bits. */
void oracle_cordic(int64_t a_q16, const int64_t *theta, int64_t K,
                   int64_t *cos_q30, int64_t *sin_q30)
{
    const int64_t full = 360LL * Q16, quarter = 90LL * Q16;
    int64_t a = a_q16 % full;
    if (a < 0) a += full;
    int64_t k = a / quarter;
    int64_t r = a - k * quarter;
    int64_t z = r << 14; /* degrees, 30 fractional bits */
    int64_t x = K, y = 0;
    for (int i = 0; i < 32; ++i) {
        int64_t xs = x >> i, ys = y >> i; /* arithmetic shifts: floor */
        if (z >= 0) {
            x = x - ys;
            y = y + xs;
            z = z - theta[i];
        } else {
            x = x + ys;
            y = y - xs;
            z = z + theta[i];
        }
    }
    int64_t c, s;
    switch (k) {
    case 0: c = x; s = y; break;
    case 1: c = -y; s = x; break;
    case 2: c = -x; s = -y; break;
    default: c = y; s = -x; break;
    }
    *cos_q30 = c;
    *sin_q30 = s;
}

/* ---------------------------------------------------------------- geometry */

typedef struct {
    int32_t nx, ny, nz;
    float sx, sy, sz;
    float T; /* tracker half-separation, mm */
} og_geom;

/* Grid coordinate (voxel units, 16 fractional bits) of a world coordinate w
 * (mm, 16 fractional bits) on an axis with n voxels of size s_q (mm, Q16),
 * the grid centred on the origin:  (w + n s / 2) / s. */
static int64_t to_grid(int64_t w, int32_t n, int64_t s_q)
{
    return floordiv((2 * w + (int64_t)n * s_q) * Q16, 2 * s_q);
}

/* Entry and exit points of one history in grid Q16.  Returns 0 when the
 * history is usable and 1 when it is rejected (a non-finite or out-of-range
 * coordinate: |u|, |v| >= 4096 mm, |angle| >= 2^20 degrees, or a grid
 * coordinate of magnitude >= 2^30). */
/* World entry and exit points of one history in mm with 16 fractional bits
 * (the frame of Sec. 2.1 made exact: CORDIC cos/sin, floor division by 2^30):
 * win = -T b + u_in e_u + v_in e_v, wout = +T b + u_out e_u + v_out e_v. */
static void world_endpoints(const og_geom *g, const int64_t *theta, int64_t K, float angle,
                            float u_in, float v_in, float u_out, float v_out, int64_t *win,
                            int64_t *wout)
{
    int64_t c, s;
    oracle_cordic(q16_of(angle), theta, K, &c, &s);
    int64_t T = q16_of(g->T);
    int64_t ui = q16_of(u_in), vi = q16_of(v_in);
    int64_t uo = q16_of(u_out), vo = q16_of(v_out);
    win[0] = (-T * c - ui * s) >> 30;
    win[1] = (-T * s + ui * c) >> 30;
    win[2] = vi;
    wout[0] = (T * c - uo * s) >> 30;
    wout[1] = (T * s + uo * c) >> 30;
    wout[2] = vo;
}

int oracle_grid_endpoints(const og_geom *g, const int64_t *theta, int64_t K,
                          float angle, float u_in, float v_in, float u_out,
                          float v_out, int64_t *gin, int64_t *gout)
{
    if (!(fabsf(angle) < 1048576.0f)) return 1;
    if (!(fabsf(u_in) < 4096.0f) || !(fabsf(v_in) < 4096.0f) ||
        !(fabsf(u_out) < 4096.0f) || !(fabsf(v_out) < 4096.0f))
        return 1;
    int64_t c, s;
    oracle_cordic(q16_of(angle), theta, K, &c, &s);
    int64_t T = q16_of(g->T);
    int64_t ui = q16_of(u_in), vi = q16_of(v_in);
    int64_t uo = q16_of(u_out), vo = q16_of(v_out);
    /* world point = -/+ T b + u e_u + v e_v, b = (c, s, 0), e_u = (-s, c, 0) */
    int64_t wx_in = (-T * c - ui * s) >> 30;
    int64_t wy_in = (-T * s + ui * c) >> 30;
    int64_t wx_out = (T * c - uo * s) >> 30;
    int64_t wy_out = (T * s + uo * c) >> 30;
    int64_t sx = q16_of(g->sx), sy = q16_of(g->sy), sz = q16_of(g->sz);
    gin[0] = to_grid(wx_in, g->nx, sx);
    gin[1] = to_grid(wy_in, g->ny, sy);
    gin[2] = to_grid(vi, g->nz, sz);
    gout[0] = to_grid(wx_out, g->nx, sx);
    gout[1] = to_grid(wy_out, g->ny, sy);
    gout[2] = to_grid(vo, g->nz, sz);
    const int64_t lim = (int64_t)1 << 30;
    for (int a = 0; a < 3; ++a)
        if (gin[a] >= lim || gin[a] <= -lim || gout[a] >= lim || gout[a] <= -lim) return 1;
    return 0;
}

/* ----------------------------------------------------- voxel set (Eq. 3.2) */

typedef struct { i128 p, q; } rat; /* p / q with q > 0 */

static int rat_cmp(const void *a, const void *b)
{
    const rat *x = (const rat *)a, *y = (const rat *)b;
    i128 l = x->p * y->q, r = y->p * x->q;
    return (l < r) ? -1 : (l > r) ? 1 : 0;
}

static int cmp_u32(const void *a, const void *b)
{
    const uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* Linear index of floor(P(t)) for t = p/q, or -1 when outside the grid. */
static int64_t voxel_at(const int64_t *gin, const int64_t *d, const int32_t *n, i128 p, i128 q)
{
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        i128 num = (i128)gin[a] * q + p * (i128)d[a];
        i128 k = floordiv128(num, q * (i128)Q16);
        if (k < 0 || k >= n[a]) return -1;
        idx[a] = (int64_t)k;
    }
    return idx[0] + (int64_t)n[0] * (idx[1] + (int64_t)n[1] * idx[2]);
}

/* The voxel set A_i of the closed segment gin -> gout (grid Q16) as sorted
 * unique linear indices (x fastest).  Writes at most `cap` indices and
 * returns the set's size, or -1 on allocation failure. */
int64_t oracle_voxel_set(const int64_t *gin, const int64_t *gout, int32_t nx, int32_t ny,
                         int32_t nz, int64_t *out, int64_t cap)
{
    const int32_t n[3] = {nx, ny, nz};
    int64_t d[3];
    int64_t maxbp = 2;
    for (int a = 0; a < 3; ++a) {
        d[a] = gout[a] - gin[a];
        maxbp += (int64_t)n[a] + 1;
    }
    rat *bp = (rat *)malloc(sizeof(rat) * (size_t)maxbp);
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * maxbp + 1));
    if (!bp || !cand) {
        free(bp);
        free(cand);
        return -1;
    }
    int64_t nb = 0;
    bp[nb].p = 0; bp[nb].q = 1; ++nb;
    bp[nb].p = 1; bp[nb].q = 1; ++nb;
    /* parameters at which coordinate a sits on grid plane k (0 <= k <= n_a) */
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0) continue;
        for (int64_t k = 0; k <= n[a]; ++k) {
            i128 p = (i128)(k * Q16 - gin[a]);
            i128 q = (i128)d[a];
            if (q < 0) { p = -p; q = -q; }
            if (p < 0 || p > q) continue; /* outside [0, 1] */
            bp[nb].p = p; bp[nb].q = q; ++nb;
        }
    }
    qsort(bp, (size_t)nb, sizeof(rat), rat_cmp);
    int64_t nc = 0;
    for (int64_t j = 0; j < nb; ++j) {
        int64_t v = voxel_at(gin, d, n, bp[j].p, bp[j].q);
        if (v >= 0) cand[nc++] = v;
        if (j + 1 < nb && rat_cmp(&bp[j], &bp[j + 1]) != 0) {
            /* midpoint of (bp[j], bp[j+1]) */
            i128 p = bp[j].p * bp[j + 1].q + bp[j + 1].p * bp[j].q;
            i128 q = 2 * bp[j].q * bp[j + 1].q;
            v = voxel_at(gin, d, n, p, q);
            if (v >= 0) cand[nc++] = v;
        }
    }
    qsort(cand, (size_t)nc, sizeof(int64_t), cmp_i64);
    int64_t m = 0;
    for (int64_t j = 0; j < nc; ++j) {
        if (j > 0 && cand[j] == cand[j - 1]) continue;
        if (m < cap) out[m] = cand[j];
        ++m;
    }
    free(bp);
    free(cand);
    return m;
}

/* Independent statement of the same membership: does the closed segment
 * gin -> gout meet the half-open cube of voxel (x, y, z)?  Per axis the
 * parameters with k <= P_a(t) / 2^16 < k + 1 form an interval whose open and
 * closed ends depend on the direction of travel; the voxel is a member when
 * the intersection of the three intervals with [0, 1] is not empty. */
int oracle_segment_meets_voxel(const int64_t *gin, const int64_t *gout, int64_t x, int64_t y,
                               int64_t z)
{
    const int64_t v[3] = {x, y, z};
    /* running lower bound lo (closed unless lo_open) and upper bound hi */
    i128 lo_p = 0, lo_q = 1, hi_p = 1, hi_q = 1;
    int lo_open = 0, hi_open = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t d = gout[a] - gin[a];
        int64_t lo_plane = v[a] * Q16, hi_plane = (v[a] + 1) * Q16;
        if (d == 0) {
            if (!(gin[a] >= lo_plane && gin[a] < hi_plane)) return 0;
            continue;
        }
        i128 lp, lq, hp, hq;
        int l_open, h_open;
        if (d > 0) { /* lo_plane <= gin + t d  <=>  t >= (lo_plane - gin)/d, closed */
            lp = lo_plane - gin[a]; lq = d; l_open = 0;
            hp = hi_plane - gin[a]; hq = d; h_open = 1; /* strict upper */
        } else {     /* decreasing coordinate */
            lp = gin[a] - hi_plane; lq = -d; l_open = 1; /* gin + t d < hi  <=>  t > ... */
            hp = gin[a] - lo_plane; hq = -d; h_open = 0; /* gin + t d >= lo  <=>  t <= ... */
        }
        /* lower = max(lower, (lp/lq)); open wins on equality */
        i128 c = lp * lo_q - lo_p * lq;
        if (c > 0 || (c == 0 && l_open)) { lo_p = lp; lo_q = lq; lo_open = l_open || (c == 0 && lo_open); }
        c = hp * hi_q - hi_p * hq;
        if (c < 0 || (c == 0 && h_open)) { hi_p = hp; hi_q = hq; hi_open = h_open || (c == 0 && hi_open); }
    }
    i128 c = lo_p * hi_q - hi_p * lo_q;
    if (c < 0) return 1;
    if (c == 0 && !lo_open && !hi_open) return 1;
    return 0;
}

/* -------------------------------------------------- classification (3.1/3.7) */

/* 1 = missed (WEPL < tau_l, Eq. 3.1), 2 = hit (WEPL > tau_h, Eq. 3.7),
 * 0 = neither (including NaN).  Plain IEEE float32 comparisons. */
int oracle_classify(float wepl, float tau_l, float tau_h)
{
    if (wepl < tau_l) return 1;
    if (wepl > tau_h) return 2;
    return 0;
}

/* ------------------------------------------------ accumulation (Alg. 1-3) */

enum { OM_SC = 1, OM_MSC = 2, OM_SM = 4 };

/* stats: [0] histories in, [1] missed, [2] hit, [3] neither,
 *        [4] rejected (missed or hit, but unusable geometry),
 *        [5] voxel memberships added from missed histories,
 *        [6] voxel memberships added from hit histories.
 * N counts missed histories per voxel (Eq. 3.4), M hit ones (Eq. 3.9),
 * H1 starts at 1 and is carved to 0 along missed paths (Alg. 1).
 * N, M and H1 may each be NULL when not wanted.  Returns 0, or -1 when out
 * of memory. */
int oracle_accumulate(const og_geom *g, float tau_l, float tau_h, int32_t methods,
                      const int64_t *theta, int64_t K, const float *angle, const float *u_in,
                      const float *v_in, const float *u_out, const float *v_out,
                      const float *wepl, int64_t n, uint32_t *N, uint32_t *M, uint8_t *H1,
                      int64_t *stats)
{
    int64_t cap = (int64_t)g->nx + g->ny + g->nz + 8;
    int64_t *set = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!set) return -1;
    int use_miss = (methods & (OM_SC | OM_MSC)) != 0;
    int use_hit = (methods & OM_SM) != 0;
    for (int64_t i = 0; i < n; ++i) {
        stats[0] += 1;
        int cls = oracle_classify(wepl[i], tau_l, tau_h);
        if (cls == 1) stats[1] += 1;
        else if (cls == 2) stats[2] += 1;
        else stats[3] += 1;
        if (!((cls == 1 && use_miss) || (cls == 2 && use_hit))) continue;
        int64_t gin[3], gout[3];
        if (oracle_grid_endpoints(g, theta, K, angle[i], u_in[i], v_in[i], u_out[i], v_out[i],
                                  gin, gout)) {
            stats[4] += 1;
            continue;
        }
        int64_t m = oracle_voxel_set(gin, gout, g->nx, g->ny, g->nz, set, cap);
        if (m < 0 || m > cap) {
            free(set);
            return -1;
        }
        for (int64_t j = 0; j < m; ++j) {
            int64_t v = set[j];
            if (cls == 1) {
                if (N) N[v] += 1;
                if (H1) H1[v] = 0;
            } else {
                if (M) M[v] += 1;
            }
        }
        stats[cls == 1 ? 5 : 6] += m;
    }
    free(set);
    return 0;
}

/* ------------------------------------- thick rays (next row f4) */

/* Thick rays (Eq. 3.2 with d_0 > 0; the paper leaves the distance measure
 * open): A_i(k) = the voxels within k voxels of a voxel of A_i in the same
 * slice, by the in-plane Chebyshev distance (|dx| <= k and |dy| <= k, same
 * z), k = floor(d_0 / in-plane voxel size).  k = 0 is A_i itself.  Counts
 * N and M as oracle_accumulate does, one per history for every voxel of its
 * A_i(k): the dilated set of each history is formed voxel by voxel and
 * stamped, so a voxel reached from several voxels of A_i counts once.
 * stats as oracle_accumulate ([5], [6]: the voxels of the thick sets). */
int oracle_accumulate_thick(const og_geom *g, float tau_l, float tau_h, int32_t methods,
                            const int64_t *theta, int64_t K, int32_t k, const float *angle,
                            const float *u_in, const float *v_in, const float *u_out,
                            const float *v_out, const float *wepl, int64_t n, uint32_t *N,
                            uint32_t *M, int64_t *stats)
{
    const int64_t V = (int64_t)g->nx * g->ny * g->nz;
    const int64_t cap = (int64_t)g->nx + g->ny + g->nz + 8;
    int64_t *set = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    if (!set || !stamp) {
        free(set);
        free(stamp);
        return -1;
    }
    for (int64_t v = 0; v < V; ++v) stamp[v] = -1;
    const int use_miss = (methods & (OM_SC | OM_MSC)) != 0;
    const int use_hit = (methods & OM_SM) != 0;
    for (int64_t i = 0; i < n; ++i) {
        stats[0] += 1;
        const int cls = oracle_classify(wepl[i], tau_l, tau_h);
        if (cls == 1) stats[1] += 1;
        else if (cls == 2) stats[2] += 1;
        else stats[3] += 1;
        if (!((cls == 1 && use_miss) || (cls == 2 && use_hit))) continue;
        int64_t gin[3], gout[3];
        if (oracle_grid_endpoints(g, theta, K, angle[i], u_in[i], v_in[i], u_out[i], v_out[i],
                                  gin, gout)) {
            stats[4] += 1;
            continue;
        }
        const int64_t m = oracle_voxel_set(gin, gout, g->nx, g->ny, g->nz, set, cap);
        if (m < 0 || m > cap) {
            free(set);
            free(stamp);
            return -1;
        }
        int64_t count = 0;
        for (int64_t j = 0; j < m; ++j) {
            const int64_t v = set[j];
            const int64_t x = v % g->nx, y = (v / g->nx) % g->ny, z = v / ((int64_t)g->nx * g->ny);
            for (int64_t dy = -k; dy <= k; ++dy)
                for (int64_t dx = -k; dx <= k; ++dx) {
                    const int64_t X = x + dx, Y = y + dy;
                    if (X < 0 || X >= g->nx || Y < 0 || Y >= g->ny) continue;
                    const int64_t w = X + g->nx * (Y + g->ny * z);
                    if (stamp[w] == i) continue;
                    stamp[w] = i;
                    ++count;
                    if (cls == 1) {
                        if (N) N[w] += 1;
                    } else if (M) {
                        M[w] += 1;
                    }
                }
        }
        stats[cls == 1 ? 5 : 6] += count;
    }
    free(set);
    free(stamp);
    return 0;
}

/* ---------------------------- thick rays, Euclidean distance (next row f4) */

/* Thick rays as Eq. 3.2 states them with d_0 > 0 and d the Euclidean
 * distance: A_i(d_0) = the voxels whose centre lies within d_0 mm of the
 * closed segment L_i (entry to exit point, Sec. 2.1).  Exact in integers:
 * with every coordinate doubled from mm * 2^16 (so voxel centres
 * ((2 i + 1 - n) s / 2) are integers too), A = 2 win, B = 2 wout, the centre
 * C = ((2 i + 1 - nx) sx, (2 j + 1 - ny) sy, (2 k + 1 - nz) sz) (s in mm *
 * 2^16, rounded once as all inputs are) and R = 2 q16(d_0), u = B - A,
 * w = C - A:
 *   w.u <= 0      : |w|^2 <= R^2            (nearest point A)
 *   w.u >= |u|^2  : |C - B|^2 <= R^2        (nearest point B)
 *   otherwise     : |w x u|^2 <= R^2 |u|^2  (the line between them).
 * |coordinates| < 2^30, so |u|, |w| < 2^31, products of two < 2^62, cross
 * components < 2^63 and |w x u|^2 < 3 2^126 fit unsigned 128 bits. */
typedef unsigned __int128 u128;

static u128 sq64(int64_t a) { return (u128)((i128)a * (i128)a); }

int oracle_in_capsule(const int64_t *A, const int64_t *B, const int64_t *C, int64_t R)
{
    int64_t u[3], w[3], wb[3];
    for (int a = 0; a < 3; ++a) {
        u[a] = B[a] - A[a];
        w[a] = C[a] - A[a];
        wb[a] = C[a] - B[a];
    }
    i128 dot = 0, uu = 0;
    for (int a = 0; a < 3; ++a) {
        dot += (i128)w[a] * u[a];
        uu += (i128)u[a] * u[a];
    }
    const u128 RR = (u128)((i128)R * R);
    if (dot <= 0) return (sq64(w[0]) + sq64(w[1]) + sq64(w[2])) <= RR;
    if (dot >= uu) return (sq64(wb[0]) + sq64(wb[1]) + sq64(wb[2])) <= RR;
    const int64_t cx = w[1] * u[2] - w[2] * u[1];
    const int64_t cy = w[2] * u[0] - w[0] * u[2];
    const int64_t cz = w[0] * u[1] - w[1] * u[0];
    return (sq64(cx) + sq64(cy) + sq64(cz)) <= RR * (u128)uu;
}

/* Doubled world endpoints of a usable history and the doubled radius; 1 when
 * the history is rejected (the thin path's rule, oracle_grid_endpoints). */
int oracle_capsule_of(const og_geom *g, const int64_t *theta, int64_t K, float d0, float angle,
                      float u_in, float v_in, float u_out, float v_out, int64_t *A, int64_t *B,
                      int64_t *R)
{
    int64_t gin[3], gout[3];
    if (oracle_grid_endpoints(g, theta, K, angle, u_in, v_in, u_out, v_out, gin, gout)) return 1;
    int64_t win[3], wout[3];
    world_endpoints(g, theta, K, angle, u_in, v_in, u_out, v_out, win, wout);
    for (int a = 0; a < 3; ++a) {
        A[a] = 2 * win[a];
        B[a] = 2 * wout[a];
    }
    *R = 2 * q16_of(d0);
    return 0;
}

/* N and M over the Euclidean thick sets: for every usable missed (hit)
 * history, every voxel of the grid box bounding its capsule (segment grown
 * by d_0) is tested with oracle_in_capsule and counted once when inside.
 * stats as oracle_accumulate ([5], [6]: the voxels of the thick sets). */
int oracle_accumulate_euclid(const og_geom *g, float tau_l, float tau_h, int32_t methods,
                             const int64_t *theta, int64_t K, float d0, const float *angle,
                             const float *u_in, const float *v_in, const float *u_out,
                             const float *v_out, const float *wepl, int64_t n, uint32_t *N,
                             uint32_t *M, int64_t *stats)
{
    const int32_t nn[3] = {g->nx, g->ny, g->nz};
    const int64_t sq[3] = {q16_of(g->sx), q16_of(g->sy), q16_of(g->sz)};
    const int use_miss = (methods & (OM_SC | OM_MSC)) != 0;
    const int use_hit = (methods & OM_SM) != 0;
    for (int64_t i = 0; i < n; ++i) {
        stats[0] += 1;
        const int cls = oracle_classify(wepl[i], tau_l, tau_h);
        if (cls == 1) stats[1] += 1;
        else if (cls == 2) stats[2] += 1;
        else stats[3] += 1;
        if (!((cls == 1 && use_miss) || (cls == 2 && use_hit))) continue;
        int64_t A[3], B[3], R;
        if (oracle_capsule_of(g, theta, K, d0, angle[i], u_in[i], v_in[i], u_out[i], v_out[i], A,
                              B, &R)) {
            stats[4] += 1;
            continue;
        }
        /* index range of each axis: centres (2 i + 1 - n) s within
         * [min(A, B) - R, max(A, B) + R], widened by one and clipped */
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            const int64_t mn = (A[a] < B[a] ? A[a] : B[a]) - R;
            const int64_t mx = (A[a] < B[a] ? B[a] : A[a]) + R;
            lo[a] = (floordiv(mn, sq[a]) + nn[a] - 1) / 2 - 1;
            hi[a] = (floordiv(mx, sq[a]) + nn[a] + 1) / 2 + 1;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > nn[a] - 1) hi[a] = nn[a] - 1;
        }
        int64_t count = 0;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    const int64_t C[3] = {(2 * x + 1 - nn[0]) * sq[0], (2 * y + 1 - nn[1]) * sq[1],
                                          (2 * z + 1 - nn[2]) * sq[2]};
                    if (!oracle_in_capsule(A, B, C, R)) continue;
                    ++count;
                    const int64_t v = x + (int64_t)nn[0] * (y + (int64_t)nn[1] * z);
                    if (cls == 1) {
                        if (N) N[v] += 1;
                    } else if (M) {
                        M[v] += 1;
                    }
                }
        stats[cls == 1 ? 5 : 6] += count;
    }
    return 0;
}

/* Does the closed segment gin -> gout (grid Q16) meet the half-open box
 * [lo, hi) (voxel units)?  The slab test of oracle_segment_meets_voxel on a
 * box: a voxel v is in A_i(k) exactly when the segment meets the box of
 * voxels within k of v in-plane, clipped to the grid. */
int oracle_segment_meets_box(const int64_t *gin, const int64_t *gout, const int64_t *lo,
                             const int64_t *hi)
{
    i128 lo_p = 0, lo_q = 1, hi_p = 1, hi_q = 1;
    int lo_open = 0, hi_open = 0;
    for (int a = 0; a < 3; ++a) {
        const int64_t d = gout[a] - gin[a];
        const int64_t lo_plane = lo[a] * Q16, hi_plane = hi[a] * Q16;
        if (d == 0) {
            if (!(gin[a] >= lo_plane && gin[a] < hi_plane)) return 0;
            continue;
        }
        i128 lp, lq, hp, hq;
        int l_open, h_open;
        if (d > 0) {
            lp = lo_plane - gin[a]; lq = d; l_open = 0;
            hp = hi_plane - gin[a]; hq = d; h_open = 1;
        } else {
            lp = gin[a] - hi_plane; lq = -d; l_open = 1;
            hp = gin[a] - lo_plane; hq = -d; h_open = 0;
        }
        i128 c = lp * lo_q - lo_p * lq;
        if (c > 0 || (c == 0 && l_open)) { lo_p = lp; lo_q = lq; lo_open = l_open || (c == 0 && lo_open); }
        c = hp * hi_q - hi_p * hq;
        if (c < 0 || (c == 0 && h_open)) { hi_p = hp; hi_q = hq; hi_open = h_open || (c == 0 && hi_open); }
    }
    const i128 c = lo_p * hi_q - hi_p * lo_q;
    if (c < 0) return 1;
    if (c == 0 && !lo_open && !hi_open) return 1;
    return 0;
}

/* Thick-ray counts of chosen voxels by testing every history: counts[b]
 * (zeroed by the caller) = histories of class cls (1 missed, 2 hit) whose
 * thick set A_i(k) holds voxel vox[b] (linear index), for nb voxels. */
void oracle_count_thick_voxels(const og_geom *g, float tau_l, float tau_h, const int64_t *theta,
                               int64_t K, int32_t k, const float *angle, const float *u_in,
                               const float *v_in, const float *u_out, const float *v_out,
                               const float *wepl, int64_t n, int32_t cls, const int64_t *vox,
                               int64_t nb, int64_t *counts)
{
    for (int64_t i = 0; i < n; ++i) {
        if (oracle_classify(wepl[i], tau_l, tau_h) != cls) continue;
        int64_t gin[3], gout[3];
        if (oracle_grid_endpoints(g, theta, K, angle[i], u_in[i], v_in[i], u_out[i], v_out[i],
                                  gin, gout))
            continue;
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t x = vox[b] % g->nx, y = (vox[b] / g->nx) % g->ny;
            const int64_t z = vox[b] / ((int64_t)g->nx * g->ny);
            const int64_t lo[3] = {x - k < 0 ? 0 : x - k, y - k < 0 ? 0 : y - k, z};
            const int64_t hi[3] = {x + k + 1 > g->nx ? g->nx : x + k + 1,
                                   y + k + 1 > g->ny ? g->ny : y + k + 1, z + 1};
            counts[b] += oracle_segment_meets_box(gin, gout, lo, hi);
        }
    }
}

/* ------------------------------- hull diagnostics (next row f3) */

/* Extra and missing voxels of a hull against the true object (the counts of
 * Tables 1-2, Sec. 4): per slice z, counts[z] = |{v in z : hull, not object}|
 * and counts[nz + z] = |{v in z : object, not hull}|; counts[2 nz] and
 * counts[2 nz + 1] are the totals. */
void oracle_hull_compare(const uint8_t *hull, const uint8_t *object, int32_t nx, int32_t ny,
                         int32_t nz, int64_t *counts)
{
    const int64_t plane = (int64_t)nx * ny;
    for (int64_t i = 0; i < 2 * (int64_t)nz + 2; ++i) counts[i] = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t j = 0; j < plane; ++j) {
            const int h = hull[z * plane + j] != 0, o = object[z * plane + j] != 0;
            if (h && !o) counts[z] += 1;
            if (o && !h) counts[nz + z] += 1;
        }
    for (int64_t z = 0; z < nz; ++z) {
        counts[2 * nz] += counts[z];
        counts[2 * nz + 1] += counts[nz + z];
    }
}

/* The voxels of a mask that it encloses within their slice: out = mask
 * minus every mask voxel joined to the slice's border by a 4-connected path
 * of mask voxels (a breadth-first search from the border).  Applied to the
 * literal MSC hull H_2 (Eq. 3.6), which excludes only a shell of steep
 * drops, it keeps the region the shell encloses.  Returns 0, -1 when out of
 * memory. */
int oracle_fill_enclosed(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, uint8_t *out)
{
    const int64_t plane = (int64_t)nx * ny;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)plane);
    uint8_t *seen = (uint8_t *)malloc((size_t)plane);
    if (!queue || !seen) {
        free(queue);
        free(seen);
        return -1;
    }
    for (int64_t z = 0; z < nz; ++z) {
        const uint8_t *m = mask + z * plane;
        memset(seen, 0, (size_t)plane);
        int64_t head = 0, tail = 0;
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int border = x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
                const int64_t j = x + nx * y;
                if (border && m[j] && !seen[j]) {
                    seen[j] = 1;
                    queue[tail++] = j;
                }
            }
        while (head < tail) {
            const int64_t j = queue[head++];
            const int64_t x = j % nx, y = j / nx;
            const int64_t nb[4][2] = {{x - 1, y}, {x + 1, y}, {x, y - 1}, {x, y + 1}};
            for (int k = 0; k < 4; ++k) {
                const int64_t X = nb[k][0], Y = nb[k][1];
                if (X < 0 || X >= nx || Y < 0 || Y >= ny) continue;
                const int64_t w = X + nx * Y;
                if (m[w] && !seen[w]) {
                    seen[w] = 1;
                    queue[tail++] = w;
                }
            }
        }
        for (int64_t j = 0; j < plane; ++j) out[z * plane + j] = m[j] && !seen[j];
    }
    free(queue);
    free(seen);
    return 0;
}

/* ------------------------- SM threshold by edge detection (next row f3) */

/* A documented form of the "modified Canny" picker of Sec. 4 (the paper
 * names the method, not its modification): per slice of M,
 *   S   = M smoothed with the 3x3 binomial kernel [1 2 1]^T [1 2 1] (edge
 *         values replicated beyond the slice),
 *   G   = Sobel derivatives of S (replicated), magnitude |Gx| + |Gy|,
 *   NMS = a voxel whose magnitude is at least its neighbour's against the
 *         gradient and above its neighbour's along it (the gradient points
 *         to larger M, so a tie keeps the voxel on the object's side);
 *         direction: along x when 5 |Gy| < 2 |Gx|, along y when
 *         5 |Gx| < 2 |Gy|, else the diagonal of sign(Gx Gy); neighbours
 *         outside the slice have magnitude 0,
 *   edge = NMS voxels with 5 mag >= max (weak) joined through weak voxels
 *         (8-connected) to one with 2 mag >= max (strong), max = the
 *         slice's largest NMS magnitude,
 *   M_t = the element of index floor(q (k - 1) / 100) of the sorted M
 *         values of the k edge voxels, H_3 = [M >= M_t]; a slice without
 *         edge voxels (max = 0) gets H_3 = 0 (as the slope picker does).
 * All integer arithmetic.  Intermediate images are returned when their
 * pointers are not NULL.  Returns 0, -1 when out of memory. */
static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_sm_canny(const uint32_t *M, int32_t nx, int32_t ny, int32_t nz, int32_t q_pct,
                    uint32_t *mt, uint8_t *has_edge, uint8_t *H3, int64_t *S_out,
                    int64_t *gx_out, int64_t *gy_out, int64_t *mag_out, uint8_t *nms_out,
                    uint8_t *edge_out)
{
    const int64_t plane = (int64_t)nx * ny;
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)plane);
    int64_t *gx = (int64_t *)malloc(sizeof(int64_t) * (size_t)plane);
    int64_t *gy = (int64_t *)malloc(sizeof(int64_t) * (size_t)plane);
    int64_t *mag = (int64_t *)malloc(sizeof(int64_t) * (size_t)plane);
    uint8_t *nms = (uint8_t *)malloc((size_t)plane);
    uint8_t *edge = (uint8_t *)malloc((size_t)plane);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)plane);
    uint32_t *vals = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)plane);
    if (!S || !gx || !gy || !mag || !nms || !edge || !queue || !vals) {
        free(S); free(gx); free(gy); free(mag); free(nms); free(edge); free(queue); free(vals);
        return -1;
    }
    static const int64_t bw[3] = {1, 2, 1};
    for (int64_t z = 0; z < nz; ++z) {
        const uint32_t *m = M + z * plane;
        for (int64_t y = 0; y < ny; ++y) /* smoothing */
            for (int64_t x = 0; x < nx; ++x) {
                int64_t acc = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int64_t X = clampi(x + dx, 0, nx - 1), Y = clampi(y + dy, 0, ny - 1);
                        acc += bw[dx + 1] * bw[dy + 1] * (int64_t)m[X + nx * Y];
                    }
                S[x + nx * y] = acc;
            }
        for (int64_t y = 0; y < ny; ++y) /* Sobel on S */
            for (int64_t x = 0; x < nx; ++x) {
                int64_t sx = 0, sy = 0;
                for (int k = -1; k <= 1; ++k) {
                    const int64_t Yk = clampi(y + k, 0, ny - 1), Xk = clampi(x + k, 0, nx - 1);
                    const int64_t Xm = clampi(x - 1, 0, nx - 1), Xp = clampi(x + 1, 0, nx - 1);
                    const int64_t Ym = clampi(y - 1, 0, ny - 1), Yp = clampi(y + 1, 0, ny - 1);
                    sx += bw[k + 1] * (S[Xp + nx * Yk] - S[Xm + nx * Yk]);
                    sy += bw[k + 1] * (S[Xk + nx * Yp] - S[Xk + nx * Ym]);
                }
                gx[x + nx * y] = sx;
                gy[x + nx * y] = sy;
                mag[x + nx * y] = llabs(sx) + llabs(sy);
            }
        int64_t mmax = 0;
        for (int64_t y = 0; y < ny; ++y) /* non-maximum suppression */
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t j = x + nx * y, ax = llabs(gx[j]), ay = llabs(gy[j]);
                int64_t dx, dy;
                if (5 * ay < 2 * ax) {
                    dx = gx[j] > 0 ? 1 : -1;
                    dy = 0;
                } else if (5 * ax < 2 * ay) {
                    dx = 0;
                    dy = gy[j] > 0 ? 1 : -1;
                } else {
                    dx = gx[j] > 0 ? 1 : -1;
                    dy = gy[j] > 0 ? 1 : -1;
                }
                int64_t fwd = 0, bwd = 0; /* along and against the gradient */
                if (x + dx >= 0 && x + dx < nx && y + dy >= 0 && y + dy < ny)
                    fwd = mag[(x + dx) + nx * (y + dy)];
                if (x - dx >= 0 && x - dx < nx && y - dy >= 0 && y - dy < ny)
                    bwd = mag[(x - dx) + nx * (y - dy)];
                nms[j] = mag[j] > 0 && mag[j] >= bwd && mag[j] > fwd;
                if (nms[j] && mag[j] > mmax) mmax = mag[j];
            }
        /* hysteresis: weak voxels joined (8-connected) to strong ones */
        int64_t head = 0, tail = 0;
        memset(edge, 0, (size_t)plane);
        for (int64_t j = 0; j < plane; ++j)
            if (nms[j] && mmax > 0 && 2 * mag[j] >= mmax) {
                edge[j] = 1;
                queue[tail++] = j;
            }
        while (head < tail) {
            const int64_t j = queue[head++], x = j % nx, y = j / nx;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int64_t X = x + dx, Y = y + dy;
                    if (X < 0 || X >= nx || Y < 0 || Y >= ny) continue;
                    const int64_t w = X + nx * Y;
                    if (!edge[w] && nms[w] && 5 * mag[w] >= mmax) {
                        edge[w] = 1;
                        queue[tail++] = w;
                    }
                }
        }
        int64_t k = 0; /* the threshold: a quantile of M over the edge */
        for (int64_t j = 0; j < plane; ++j)
            if (edge[j]) vals[k++] = m[j];
        uint8_t *h = H3 + z * plane;
        if (k == 0) {
            mt[z] = 0;
            has_edge[z] = 0;
            memset(h, 0, (size_t)plane);
        } else {
            qsort(vals, (size_t)k, sizeof(uint32_t), cmp_u32);
            mt[z] = vals[((int64_t)q_pct * (k - 1)) / 100];
            has_edge[z] = 1;
            for (int64_t j = 0; j < plane; ++j) h[j] = m[j] >= mt[z];
        }
        if (S_out) memcpy(S_out + z * plane, S, sizeof(int64_t) * (size_t)plane);
        if (gx_out) memcpy(gx_out + z * plane, gx, sizeof(int64_t) * (size_t)plane);
        if (gy_out) memcpy(gy_out + z * plane, gy, sizeof(int64_t) * (size_t)plane);
        if (mag_out) memcpy(mag_out + z * plane, mag, sizeof(int64_t) * (size_t)plane);
        if (nms_out) memcpy(nms_out + z * plane, nms, (size_t)plane);
        if (edge_out) memcpy(edge_out + z * plane, edge, (size_t)plane);
    }
    free(S); free(gx); free(gy); free(mag); free(nms); free(edge); free(queue); free(vals);
    return 0;
}

/* ------------------------------- SC as the paper ran it (next row f2) */

/* Binned SC (Sec. 2.2 data cuts; Sec. 3.2, its implementation paragraphs).
 * Histories are binned by gantry angle and by the lateral and vertical
 * displacement of the path's mid-point, (u_in + u_out) / 2 and
 * (v_in + v_out) / 2, from the centre of the volume.  Angle bins are centred
 * on multiples of the bin size (so a gantry angle falls on a bin centre);
 * displacement bins are [lo + i size, lo + (i + 1) size).  In each bin, a
 * history whose WEPL, lateral slope (u_out - u_in) or vertical slope
 * (v_out - v_in) lies more than k standard deviations from the bin's mean is
 * cut; the slopes over the fixed tracker separation stand for the relative
 * angles.  A bin whose kept histories have mean WEPL below the cutoff is
 * missed: in every slice whose centre height lies in the bin's vertical
 * interval, the straight line along the beam at the bin's centre angle and
 * lateral centre, at that slice's centre height, is carved (the bin's line,
 * one per slice it covers, so that slices thinner than a bin all get lines).
 * The carved image is averaged over a w x w window in each slice (voxels
 * outside the grid count as 0) and a voxel is in the hull when its window
 * holds at least min_count uncarved voxels (the average exceeds
 * (min_count - 1) / w^2).
 *
 * All of it is integer arithmetic: angle, u and v in Q16 as for the paths;
 * WEPL and slopes in 1/256 mm (rounded to nearest even); per-bin sums in 64
 * bits (exact while a bin holds fewer than 2^27 histories); and the cut
 * |x - mean| <= k sigma, with the population sigma, as
 * (n x - S)^2 <= k^2 (n Q - S^2) in 128 bits.  A history is binned when its
 * angle and coordinates are in the path's accepted range, |WEPL| < 1024 mm,
 * both slopes are below 1024 mm and its bin exists. */
typedef struct {
    int32_t n_ang, n_u, n_v;   /* bins per axis; n_ang ang_q = 360 degrees */
    int64_t ang_q, u_q, v_q;   /* bin sizes, Q16 degrees and mm */
    int64_t u_lo_q, v_lo_q;    /* lower edge of the first u and v bin, Q16 mm */
    int32_t k;                 /* cut at k standard deviations */
    int64_t miss_q8;           /* missed: kept mean WEPL below this, 1/256 mm */
    int32_t w;                 /* averaging window, odd */
    int32_t min_count;         /* uncarved voxels a window needs */
} og_binned;

static int64_t q8_of(float x) { return (int64_t)llrint((double)x * 256.0); }

/* Bin of one history, -1 when it is not binned; x receives WEPL, lateral and
 * vertical slope in 1/256 mm. */
static int64_t bin_of(const og_binned *b, float angle, float u_in, float v_in, float u_out,
                      float v_out, float wepl, int64_t x[3])
{
    if (!(fabsf(angle) < 1048576.0f) || !(fabsf(wepl) < 1024.0f)) return -1;
    if (!(fabsf(u_in) < 4096.0f) || !(fabsf(v_in) < 4096.0f) || !(fabsf(u_out) < 4096.0f) ||
        !(fabsf(v_out) < 4096.0f))
        return -1;
    x[0] = q8_of(wepl);
    x[1] = q8_of(u_out) - q8_of(u_in);
    x[2] = q8_of(v_out) - q8_of(v_in);
    if (llabs(x[1]) >= 1024 * 256 || llabs(x[2]) >= 1024 * 256) return -1;
    const int64_t full = 360LL * Q16;
    int64_t a = q16_of(angle) % full;
    if (a < 0) a += full;
    int64_t ia = floordiv(2 * a + b->ang_q, 2 * b->ang_q); /* nearest centre */
    if (ia == b->n_ang) ia = 0;
    const int64_t u2 = q16_of(u_in) + q16_of(u_out), v2 = q16_of(v_in) + q16_of(v_out);
    const int64_t iu = floordiv(u2 - 2 * b->u_lo_q, 2 * b->u_q);
    const int64_t iv = floordiv(v2 - 2 * b->v_lo_q, 2 * b->v_q);
    if (iu < 0 || iu >= b->n_u || iv < 0 || iv >= b->n_v) return -1;
    return ia + (int64_t)b->n_ang * (iu + (int64_t)b->n_u * iv);
}

/* x within k standard deviations of the bin's values (n, S, Q). */
static int within(int64_t n, int64_t S, int64_t Q, int64_t x, int32_t k)
{
    const i128 d = (i128)n * x - S;
    const i128 var_n2 = (i128)n * Q - (i128)S * S; /* n^2 sigma^2 */
    return d * d <= (i128)k * k * var_n2;
}

/* Bin bi's centre angle (degrees) and lateral centre (mm). */
void oracle_bin_line(const og_binned *b, int64_t bi, float *la, float *lu)
{
    const int64_t ia = bi % b->n_ang, iu = (bi / b->n_ang) % b->n_u;
    *la = (float)((double)(ia * b->ang_q) / (double)Q16);
    *lu = (float)((double)(2 * b->u_lo_q + (2 * iu + 1) * b->u_q) / (2.0 * Q16));
}

/* Vertical bin of slice z (its centre height, from the Q16 slice thickness),
 * or -1; *zc receives the centre height in mm. */
int64_t oracle_slice_bin(const og_geom *g, const og_binned *b, int64_t z, float *zc)
{
    const int64_t sz_q = q16_of(g->sz);
    const int64_t c2 = (2 * z + 1 - g->nz) * sz_q; /* twice the centre, Q16 */
    *zc = (float)((double)c2 / (2.0 * Q16));
    const int64_t iv = floordiv(c2 - 2 * b->v_lo_q, 2 * b->v_q);
    return iv >= 0 && iv < b->n_v ? iv : -1;
}

/* Binned SC over n histories.  acc (9 int64 per bin, zeroed by the caller):
 * n, S and Q of WEPL, lateral and vertical slope, then kept n and kept WEPL
 * sum; carved (V bytes): 1 not carved, 0 carved; mask (V bytes): the hull;
 * stats (zeroed by the caller): [0] histories binned, [1] histories cut,
 * [2] bins with histories, [3] missed bins, [4] lines carved (a missed bin
 * times the slices it covers), [5] lines that miss the volume.  Returns 0,
 * -1 when out of memory. */
int oracle_sc_binned(const og_geom *g, const og_binned *b, const int64_t *theta, int64_t K,
                     const float *angle, const float *u_in, const float *v_in,
                     const float *u_out, const float *v_out, const float *wepl, int64_t n,
                     int64_t *acc, uint8_t *carved, uint8_t *mask, int64_t *stats)
{
    const int64_t nb = (int64_t)b->n_ang * b->n_u * b->n_v;
    const int64_t V = (int64_t)g->nx * g->ny * g->nz;
    const int64_t cap = (int64_t)g->nx + g->ny + g->nz + 8;
    int64_t *set = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!set) return -1;
    int64_t x[3];
    for (int64_t i = 0; i < n; ++i) { /* bin statistics */
        const int64_t bi = bin_of(b, angle[i], u_in[i], v_in[i], u_out[i], v_out[i], wepl[i], x);
        if (bi < 0) continue;
        int64_t *a = acc + 9 * bi;
        a[0] += 1;
        for (int q = 0; q < 3; ++q) {
            a[1 + q] += x[q];
            a[4 + q] += x[q] * x[q];
        }
        stats[0] += 1;
    }
    for (int64_t i = 0; i < n; ++i) { /* data cuts; kept WEPL per bin */
        const int64_t bi = bin_of(b, angle[i], u_in[i], v_in[i], u_out[i], v_out[i], wepl[i], x);
        if (bi < 0) continue;
        int64_t *a = acc + 9 * bi;
        int keep = 1;
        for (int q = 0; q < 3; ++q) keep = keep && within(a[0], a[1 + q], a[4 + q], x[q], b->k);
        if (!keep) {
            stats[1] += 1;
            continue;
        }
        a[7] += 1;
        a[8] += x[0];
    }
    memset(carved, 1, (size_t)V);
    for (int64_t bi = 0; bi < nb; ++bi) { /* carve the missed bins' lines */
        const int64_t *a = acc + 9 * bi;
        if (a[0] > 0) stats[2] += 1;
        if (!(a[7] > 0 && a[8] < b->miss_q8 * a[7])) continue;
        stats[3] += 1;
        const int64_t iv = bi / ((int64_t)b->n_ang * b->n_u);
        float la, lu;
        oracle_bin_line(b, bi, &la, &lu);
        for (int64_t z = 0; z < g->nz; ++z) {
            float zc;
            if (oracle_slice_bin(g, b, z, &zc) != iv) continue;
            stats[4] += 1;
            int64_t gin[3], gout[3];
            if (oracle_grid_endpoints(g, theta, K, la, lu, zc, lu, zc, gin, gout)) {
                stats[5] += 1;
                continue;
            }
            const int64_t m = oracle_voxel_set(gin, gout, g->nx, g->ny, g->nz, set, cap);
            if (m < 0 || m > cap) {
                free(set);
                return -1;
            }
            for (int64_t j = 0; j < m; ++j) carved[set[j]] = 0;
        }
    }
    const int64_t r = b->w / 2; /* w x w in-slice window, outside = 0 */
    for (int64_t z = 0; z < g->nz; ++z)
        for (int64_t y = 0; y < g->ny; ++y)
            for (int64_t xx = 0; xx < g->nx; ++xx) {
                int64_t c = 0;
                for (int64_t dy = -r; dy <= r; ++dy)
                    for (int64_t dx = -r; dx <= r; ++dx) {
                        const int64_t X = xx + dx, Y = y + dy;
                        if (X < 0 || X >= g->nx || Y < 0 || Y >= g->ny) continue;
                        c += carved[X + g->nx * (Y + g->ny * z)];
                    }
                mask[xx + g->nx * (y + g->ny * z)] = c >= b->min_count;
            }
    free(set);
    return 0;
}

/* ------------------------- hull-restricted system-matrix rows (next row f1) */

/* The voxels of A_i in the order the path meets them (increasing t): the
 * voxel at each crossing parameter and at each midpoint between two, in
 * parameter order, repeats dropped (a straight segment meets a convex voxel
 * in one parameter interval, so a voxel's candidates are consecutive).
 * Writes at most `cap` indices; returns the count, or -1 when out of memory. */
int64_t oracle_voxel_path(const int64_t *gin, const int64_t *gout, int32_t nx, int32_t ny,
                          int32_t nz, int64_t *out, int64_t cap)
{
    const int32_t n[3] = {nx, ny, nz};
    int64_t d[3];
    int64_t maxbp = 2;
    for (int a = 0; a < 3; ++a) {
        d[a] = gout[a] - gin[a];
        maxbp += (int64_t)n[a] + 1;
    }
    rat *bp = (rat *)malloc(sizeof(rat) * (size_t)maxbp);
    if (!bp) return -1;
    int64_t nb = 0;
    bp[nb].p = 0; bp[nb].q = 1; ++nb;
    bp[nb].p = 1; bp[nb].q = 1; ++nb;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0) continue;
        for (int64_t k = 0; k <= n[a]; ++k) {
            i128 p = (i128)(k * Q16 - gin[a]);
            i128 q = (i128)d[a];
            if (q < 0) { p = -p; q = -q; }
            if (p < 0 || p > q) continue;
            bp[nb].p = p; bp[nb].q = q; ++nb;
        }
    }
    qsort(bp, (size_t)nb, sizeof(rat), rat_cmp);
    int64_t m = 0, last = -1;
    for (int64_t j = 0; j < nb; ++j) {
        int64_t v = voxel_at(gin, d, n, bp[j].p, bp[j].q);
        for (int pass = 0; pass < 2; ++pass) {
            if (v >= 0 && v != last) {
                if (m < cap) out[m] = v;
                ++m;
                last = v;
            }
            if (pass == 0) {
                if (!(j + 1 < nb && rat_cmp(&bp[j], &bp[j + 1]) != 0)) break;
                i128 p = bp[j].p * bp[j + 1].q + bp[j + 1].p * bp[j].q;
                i128 q = 2 * bp[j].q * bp[j + 1].q;
                v = voxel_at(gin, d, n, p, q);
            }
        }
    }
    free(bp);
    return m;
}

/* Rows of the hull-restricted system matrix: row i lists, in path order, the
 * voxels of A_i that are in the hull (hull[v] != 0).  Every input history
 * has a row (a history with unusable geometry has an empty one).  row_nnz[i]
 * receives the row's length; when cols is not NULL the rows are written
 * back to back (cols must hold their total).  Returns 0, -1 when out of
 * memory. */
int oracle_system_rows(const og_geom *g, const int64_t *theta, int64_t K, const float *angle,
                       const float *u_in, const float *v_in, const float *u_out,
                       const float *v_out, int64_t n, const uint8_t *hull, int64_t *row_nnz,
                       int32_t *cols)
{
    int64_t cap = (int64_t)g->nx + g->ny + g->nz + 8;
    int64_t *path = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!path) return -1;
    int64_t at = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t gin[3], gout[3];
        int64_t cnt = 0;
        if (!oracle_grid_endpoints(g, theta, K, angle[i], u_in[i], v_in[i], u_out[i], v_out[i],
                                   gin, gout)) {
            int64_t m = oracle_voxel_path(gin, gout, g->nx, g->ny, g->nz, path, cap);
            if (m < 0 || m > cap) {
                free(path);
                return -1;
            }
            for (int64_t j = 0; j < m; ++j)
                if (hull[path[j]]) {
                    if (cols) cols[at] = (int32_t)path[j];
                    ++at;
                    ++cnt;
                }
        }
        row_nnz[i] = cnt;
    }
    free(path);
    return 0;
}

/* ------------------------------- FP64 geometry comparison (reported only) */

/* The same history with unquantised FP64 geometry: libm cos/sin of the
 * angle, no rounding of u, v, T or the voxel sizes; grid coordinates in
 * voxel units, (w + n s / 2) / s.  The same rejection rules as
 * oracle_grid_endpoints (a grid coordinate of magnitude >= 2^14 voxels,
 * i.e. 2^30 in Q16).  Returns 0 when usable, 1 when rejected. */
int oracle_grid_endpoints_fp64(const og_geom *g, float angle, float u_in, float v_in,
                               float u_out, float v_out, double *gin, double *gout)
{
    if (!(fabsf(angle) < 1048576.0f)) return 1;
    if (!(fabsf(u_in) < 4096.0f) || !(fabsf(v_in) < 4096.0f) ||
        !(fabsf(u_out) < 4096.0f) || !(fabsf(v_out) < 4096.0f))
        return 1;
    const double rad = fmod((double)angle, 360.0) * (acos(-1.0) / 180.0);
    const double c = cos(rad), s = sin(rad), T = g->T;
    const double wx_in = -T * c - (double)u_in * s, wy_in = -T * s + (double)u_in * c;
    const double wx_out = T * c - (double)u_out * s, wy_out = T * s + (double)u_out * c;
    gin[0] = wx_in / g->sx + g->nx / 2.0;
    gin[1] = wy_in / g->sy + g->ny / 2.0;
    gin[2] = (double)v_in / g->sz + g->nz / 2.0;
    gout[0] = wx_out / g->sx + g->nx / 2.0;
    gout[1] = wy_out / g->sy + g->ny / 2.0;
    gout[2] = (double)v_out / g->sz + g->nz / 2.0;
    for (int a = 0; a < 3; ++a)
        if (fabs(gin[a]) >= 16384.0 || fabs(gout[a]) >= 16384.0) return 1;
    return 0;
}

static int cmp_dbl(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* Linear index of floor(P(t)) in double, or -1 outside the grid. */
static int64_t voxel_at_fp64(const double *gin, const double *d, const int32_t *n, double t)
{
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        double k = floor(gin[a] + t * d[a]);
        if (k < 0 || k >= n[a]) return -1;
        idx[a] = (int64_t)k;
    }
    return idx[0] + (int64_t)n[0] * (idx[1] + (int64_t)n[1] * idx[2]);
}

/* The voxel set of the closed segment gin -> gout (grid units, double) by
 * the definition the fixed-point set uses: floor(P(t)) is constant between
 * the parameters at which a coordinate crosses a grid plane, so the set is
 * the voxels at the two ends and at the midpoints between consecutive
 * crossing parameters (at FP64 inputs a segment passes through an edge or a
 * corner with probability zero, so the crossing points themselves add no
 * voxel).  Sorted unique linear indices; returns the size, -1 when out of
 * memory. */
int64_t oracle_voxel_set_fp64(const double *gin, const double *gout, int32_t nx, int32_t ny,
                              int32_t nz, int64_t *out, int64_t cap)
{
    const int32_t n[3] = {nx, ny, nz};
    double d[3];
    int64_t maxbp = 2;
    for (int a = 0; a < 3; ++a) {
        d[a] = gout[a] - gin[a];
        maxbp += (int64_t)n[a] + 1;
    }
    double *bp = (double *)malloc(sizeof(double) * (size_t)maxbp);
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxbp + 2));
    if (!bp || !cand) {
        free(bp);
        free(cand);
        return -1;
    }
    int64_t nb = 0;
    bp[nb++] = 0.0;
    bp[nb++] = 1.0;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        for (int64_t k = 0; k <= n[a]; ++k) {
            const double t = ((double)k - gin[a]) / d[a];
            if (t > 0.0 && t < 1.0) bp[nb++] = t;
        }
    }
    qsort(bp, (size_t)nb, sizeof(double), cmp_dbl);
    int64_t nc = 0;
    int64_t v = voxel_at_fp64(gin, d, n, 0.0);
    if (v >= 0) cand[nc++] = v;
    v = voxel_at_fp64(gin, d, n, 1.0);
    if (v >= 0) cand[nc++] = v;
    for (int64_t j = 0; j + 1 < nb; ++j) {
        if (bp[j + 1] <= bp[j]) continue;
        v = voxel_at_fp64(gin, d, n, 0.5 * (bp[j] + bp[j + 1]));
        if (v >= 0) cand[nc++] = v;
    }
    qsort(cand, (size_t)nc, sizeof(int64_t), cmp_i64);
    int64_t m = 0;
    for (int64_t j = 0; j < nc; ++j) {
        if (j > 0 && cand[j] == cand[j - 1]) continue;
        if (m < cap) out[m] = cand[j];
        ++m;
    }
    free(bp);
    free(cand);
    return m;
}

/* Each traversed history's fixed-point set (the method as built) against its
 * FP64-geometry set, and the FP64 counts N64 (missed) and M64 (hit).
 * cmp: [0] histories traversed with both geometries, [1] their fixed-point
 * memberships, [2] memberships in exactly one of the two sets, [3] histories
 * whose two sets differ, [4] histories traversed with one geometry only.
 * Returns 0, or -1 when out of memory. */
int oracle_compare_fp64(const og_geom *g, float tau_l, float tau_h, int32_t methods,
                        const int64_t *theta, int64_t K, const float *angle,
                        const float *u_in, const float *v_in, const float *u_out,
                        const float *v_out, const float *wepl, int64_t n, uint32_t *N64,
                        uint32_t *M64, int64_t *cmp)
{
    int64_t cap = (int64_t)g->nx + g->ny + g->nz + 8;
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t *b = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!a || !b) {
        free(a);
        free(b);
        return -1;
    }
    int use_miss = (methods & (OM_SC | OM_MSC)) != 0;
    int use_hit = (methods & OM_SM) != 0;
    for (int64_t i = 0; i < n; ++i) {
        int cls = oracle_classify(wepl[i], tau_l, tau_h);
        if (!((cls == 1 && use_miss) || (cls == 2 && use_hit))) continue;
        int64_t gin[3], gout[3];
        double fin[3], fout[3];
        int rej_q = oracle_grid_endpoints(g, theta, K, angle[i], u_in[i], v_in[i], u_out[i],
                                          v_out[i], gin, gout);
        int rej_f = oracle_grid_endpoints_fp64(g, angle[i], u_in[i], v_in[i], u_out[i],
                                               v_out[i], fin, fout);
        int64_t ma = 0, mb = 0;
        if (!rej_q) ma = oracle_voxel_set(gin, gout, g->nx, g->ny, g->nz, a, cap);
        if (!rej_f) mb = oracle_voxel_set_fp64(fin, fout, g->nx, g->ny, g->nz, b, cap);
        if (ma < 0 || mb < 0 || ma > cap || mb > cap) {
            free(a);
            free(b);
            return -1;
        }
        if (!rej_f)
            for (int64_t j = 0; j < mb; ++j) {
                if (cls == 1) N64[b[j]] += 1;
                else M64[b[j]] += 1;
            }
        if (rej_q != rej_f) {
            cmp[4] += 1;
            continue;
        }
        if (rej_q) continue;
        /* symmetric difference of two sorted sets */
        int64_t x = 0, y = 0, only = 0;
        while (x < ma || y < mb) {
            if (y >= mb || (x < ma && a[x] < b[y])) { ++only; ++x; }
            else if (x >= ma || b[y] < a[x]) { ++only; ++y; }
            else { ++x; ++y; }
        }
        cmp[0] += 1;
        cmp[1] += ma;
        cmp[2] += only;
        cmp[3] += only > 0;
    }
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------ decisions (3.3-3.10) */

/* H_1 = V \ U A_i  (Eq. 3.3) from the count of missed paths through v. */
void oracle_sc_from_counts(const uint32_t *N, int64_t V, uint8_t *H1)
{
    for (int64_t v = 0; v < V; ++v) H1[v] = (N[v] == 0) ? 1 : 0;
}

/* Neighbourhood B(v) = {w : d(v, w) <= 1} (Eq. 3.5) with d in voxel-index
 * units: v itself and its face neighbours inside the grid; nbhd = 6 for all
 * three axes, 4 for the in-plane ones only.  Writes up to 7 indices. */
static int neighbours(int64_t x, int64_t y, int64_t z, int32_t nx, int32_t ny, int32_t nz,
                      int nbhd, int64_t *w)
{
    int c = 0;
    int64_t base = x + (int64_t)nx * (y + (int64_t)ny * z);
    w[c++] = base;
    if (x > 0) w[c++] = base - 1;
    if (x + 1 < nx) w[c++] = base + 1;
    if (y > 0) w[c++] = base - nx;
    if (y + 1 < ny) w[c++] = base + nx;
    if (nbhd == 6) {
        if (z > 0) w[c++] = base - (int64_t)nx * ny;
        if (z + 1 < nz) w[c++] = base + (int64_t)nx * ny;
    }
    return c;
}

/* MSC decision (Eq. 3.6, Alg. 2): H_2(v) = 0 when N(v) - N(w) >= N_t for some
 * w in B(v), else 1.  Differences are taken in signed 64-bit arithmetic. */
void oracle_msc_decide(const uint32_t *N, int32_t nx, int32_t ny, int32_t nz, int32_t Nt,
                       int32_t nbhd, uint8_t *H2)
{
    int64_t w[7];
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
                H2[v] = 1;
                int c = neighbours(x, y, z, nx, ny, nz, nbhd, w);
                for (int j = 0; j < c; ++j)
                    if ((int64_t)N[v] - (int64_t)N[w[j]] >= (int64_t)Nt) H2[v] = 0;
            }
}

/* SM threshold and decision (Eq. 3.10, Alg. 3).  With per_slice = 1 each
 * slice z is treated on its own with the in-plane neighbourhood (Sec. 3.4:
 * the steepest edge is found in each slice); with per_slice = 0 the whole
 * volume is one region with neighbourhood nbhd.  In visiting order (x
 * fastest) the steepest drop MaxSlope = max M(v) - M(w) is tracked with the
 * ">=" update of Alg. 3, so the last voxel that reaches the maximum gives
 * index; M_t = M(index).  H_3(v) = [M(v) >= M_t] when ge = 1 (the text of
 * Sec. 3.4), [M(v) > M_t] when ge = 0 (Eq. 3.10).  A region whose MaxSlope is
 * 0 has no edge and gets H_3 = 0.  Outputs per slice: Mt, slope, index (the
 * same values in every slice when per_slice = 0). */
void oracle_sm_decide(const uint32_t *M, int32_t nx, int32_t ny, int32_t nz, int32_t per_slice,
                      int32_t nbhd, int32_t ge, uint32_t *Mt_out, uint32_t *slope_out,
                      int64_t *index_out, uint8_t *H3)
{
    int64_t w[7];
    int64_t plane = (int64_t)nx * ny;
    int32_t nregions = per_slice ? nz : 1;
    int region_nbhd = per_slice ? 4 : nbhd;
    for (int32_t r = 0; r < nregions; ++r) {
        int64_t z0 = per_slice ? r : 0, z1 = per_slice ? r + 1 : nz;
        int64_t max_slope = 0, index = 0;
        for (int64_t z = z0; z < z1; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    int64_t v = x + nx * (y + (int64_t)ny * z);
                    int c = neighbours(x, y, z, nx, ny, nz, region_nbhd, w);
                    for (int j = 0; j < c; ++j) {
                        int64_t diff = (int64_t)M[v] - (int64_t)M[w[j]];
                        if (diff >= max_slope) {
                            max_slope = diff;
                            index = v;
                        }
                    }
                }
        uint32_t Mt = M[index];
        for (int64_t z = z0; z < z1; ++z) {
            Mt_out[z] = Mt;
            slope_out[z] = (uint32_t)max_slope;
            index_out[z] = index;
            for (int64_t q = 0; q < plane; ++q) {
                int64_t v = z * plane + q;
                uint8_t in = ge ? (M[v] >= Mt) : (M[v] > Mt);
                H3[v] = (max_slope == 0) ? 0 : in;
            }
        }
    }
}

/* ------------------------------------------------ per-voxel sampled counts */

/* |C(v)| for one voxel v = (x, y, z) straight from Eq. 3.4 / Eq. 3.9: the
 * number of histories of class `cls` (1 missed, 2 hit) whose path meets v,
 * tested history by history with the slab test.  Independent of the voxel
 * enumeration above; used to check single voxels of full-size volumes. */
int64_t oracle_count_through_voxel(const og_geom *g, float tau_l, float tau_h,
                                   const int64_t *theta, int64_t K, const float *angle,
                                   const float *u_in, const float *v_in, const float *u_out,
                                   const float *v_out, const float *wepl, int64_t n,
                                   int32_t cls, int64_t x, int64_t y, int64_t z)
{
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (oracle_classify(wepl[i], tau_l, tau_h) != cls) continue;
        int64_t gin[3], gout[3];
        if (oracle_grid_endpoints(g, theta, K, angle[i], u_in[i], v_in[i], u_out[i], v_out[i],
                                  gin, gout))
            continue;
        count += oracle_segment_meets_voxel(gin, gout, x, y, z);
    }
    return count;
}
