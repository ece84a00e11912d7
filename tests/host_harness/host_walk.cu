// Test harness: the library's fixed-point geometry and traversal (hd_geom.cuh),
// compiled for the host so the CPU test suite can compare them with the oracle.
#include "../../paper_1402_1720_gb300/csrc/hd_geom.cuh"
#include <vector>
struct HostVisit {
    int32_t *out; int cap; mutable int n = 0;
    void operator()(uint32_t v) const { if (n < cap) out[n] = (int32_t)v; ++n; }
};
extern "C" int hx_walk(const int32_t *gi, const int32_t *go, int nx, int ny, int nz, int32_t *out, int cap)
{
    HostVisit v{out, cap};
    return (int)hd::walk_all(gi, go, nx, ny, nz, v);
}
// union of the walks clipped to tiles of size (tx,ty,tz); returns global indices
extern "C" int hx_walk_tiled(const int32_t *gi, const int32_t *go, int nx, int ny, int nz, int tx, int ty, int tz, int32_t *out, int cap)
{
    int n = 0;
    for (int z0 = 0; z0 < nz; z0 += tz) for (int y0 = 0; y0 < ny; y0 += ty) for (int x0 = 0; x0 < nx; x0 += tx) {
        int dx = std::min(tx, nx - x0), dy = std::min(ty, ny - y0), dz = std::min(tz, nz - z0);
        int32_t a[3] = {gi[0] - (x0 << 16), gi[1] - (y0 << 16), gi[2] - (z0 << 16)};
        int32_t b[3] = {go[0] - (x0 << 16), go[1] - (y0 << 16), go[2] - (z0 << 16)};
        hd::Walk w;
        if (!hd::walk_begin(w, a, b, dx, dy, dz)) continue;
        do {
            int l = w.idx; int lx = l % dx, ly = (l / dx) % dy, lz = l / (dx * dy);
            if (lx < 0 || ly < 0 || lz < 0 || lz >= dz) return -1000000;
            if (n < cap) out[n] = (x0 + lx) + nx * ((y0 + ly) + ny * (z0 + lz));
            ++n;
        } while (hd::walk_next(w));
    }
    return n;
}
extern "C" int hx_endpoints(int nx, int ny, int nz, float sx, float sy, float sz, float T,
                            const long long *theta, long long K, float a, float ui, float vi, float uo, float vo, int32_t *out)
{
    hd::GeomQ g = hd::make_geomq(nx, ny, nz, sx, sy, sz, T);
    hd::Cordic cd; for (int i = 0; i < 32; ++i) cd.theta[i] = theta[i]; cd.K = K;
    return hd::endpoints(g, cd, a, ui, vi, uo, vo, out) ? 1 : 0;
}
// the voxel set produced as major-axis runs, expanded to linear indices
extern "C" int hx_runs(const int32_t *gi, const int32_t *go, int nx, int ny, int nz, int32_t *out, int cap, int *nruns)
{
    hd::RunWalk w;
    int n = 0, runs = 0;
    if (hd::run_begin(w, gi, go, nx, ny, nz)) {
        const bool ymaj = (w.flags >> 5) & 1;
        int row, lo, hi;
        while (hd::run_next(w, row, lo, hi)) {
            ++runs;
            if (lo < 0 || hi >= w.nmaj || lo > hi) return -1000000;
            for (int m = lo; m <= hi; ++m) {
                int v;
                if (!ymaj) v = m + nx * row;
                else v = (row % nx) + nx * (m + ny * (row / nx));
                if (n < cap) out[n] = v;
                ++n;
            }
            if (runs > 100000) return -2000000;
        }
    }
    *nruns = runs;
    return n;
}
// the same, with the walk state packed and unpacked before the first run
extern "C" int hx_runs_packed(const int32_t *gi, const int32_t *go, int nx, int ny, int nz, int32_t *out, int cap)
{
    hd::RunWalk w0, w;
    uint32_t o[hd::kPackedWords];
    if (hd::run_begin(w0, gi, go, nx, ny, nz)) hd::run_pack(w0, o);
    else hd::run_pack_empty(o);
    hd::run_unpack(o, nx, ny, w);
    int n = 0;
    const bool ymaj = (w.flags >> 5) & 1;
    int row, lo, hi;
    while (hd::run_next(w, row, lo, hi)) {
        if (lo < 0 || hi >= w.nmaj || lo > hi) return -1000000;
        for (int m = lo; m <= hi; ++m) {
            int v = !ymaj ? m + nx * row : (row % nx) + nx * (m + ny * (row / nx));
            if (n < cap) out[n] = v;
            ++n;
        }
    }
    return n;
}
// exhaustive check of the tile-index division used when bucketing records:
// floor(v / t) for every v in [0, 4096) and tile size t in [1, 4096];
// returns the number of mismatches
extern "C" long long hx_check_tile_division(void)
{
    long long bad = 0;
    for (int t = 1; t <= 4096; ++t) {
        hd::TilePlan tp{};
        tp.nx = tp.ny = tp.nz = 4096;
        tp.tx = tp.ty = tp.tz = t;
        const unsigned m = t == 1 ? 0u : static_cast<unsigned>((1ull << 32) / static_cast<unsigned>(t)) + 1u;
        tp.mtx = tp.mty = tp.mtz = m;
        for (int v = 0; v < 4096; ++v) {
            const int32_t r[6] = {v << 16, v << 16, v << 16, v << 16, v << 16, v << 16};
            int lo[3], hi[3];
            hd::tile_range(tp, r, lo, hi);
            if (lo[0] != v / t || hi[2] != v / t) ++bad;
        }
    }
    return bad;
}
// the lean form when the walk has one (through pack and unpack, as the
// traversal kernel sees it), else the general run walk; *lean says which
// and *steps is the voxel count the lean walk reports with its last run
extern "C" int hx_runs_lean(const int32_t *gi, const int32_t *go, int nx, int ny, int nz,
                            int32_t *out, int cap, int *lean, unsigned *steps)
{
    hd::RunWalk w;
    *lean = 0;
    *steps = 0;
    int n = 0, runs = 0;
    auto emit = [&](bool ymaj, int nmaj, int row, int lo, int hi) {
        if (lo < 0 || hi >= nmaj || lo > hi) return false;
        for (int m = lo; m <= hi; ++m) {
            int v = !ymaj ? m + nx * row : (row % nx) + nx * (m + ny * (row / nx));
            if (n < cap) out[n] = v;
            ++n;
        }
        return ++runs <= 100000;
    };
    if (!hd::run_begin(w, gi, go, nx, ny, nz)) return 0;
    hd::LeanWalk L0, L;
    if (hd::lean_of(w, L0)) {
        *lean = 1;
        uint32_t o[hd::kLeanWords];
        hd::lean_pack(L0, o);
        hd::lean_unpack(o, L);
        if (hd::lean_empty(L)) return -3000000;
        const bool ymaj = (L.fl >> 2) & 1;
        const int nmaj = ymaj ? ny : nx;
        // the kernel's cursor form must give the same runs as lean_step
        hd::LeanCursor c;
        if (!hd::lean_start(o, nmaj, c)) return -3000000;
        unsigned ends = 0, runs_c = 0;
        int row, lo, hi, rb, lo_c, hi_c;
        bool more;
        do {
            more = hd::lean_step(L, row, lo, hi, *steps);
            const bool more_c = hd::lean_run(c, rb, lo_c, hi_c, ends);
            ++runs_c;
            if (more_c != more || rb != row * nmaj || lo_c != lo || hi_c != hi) return -4000000;
            if (!emit(ymaj, nmaj, row, lo, hi)) return -1000000;
        } while (more);
        if (ends + runs_c != *steps) return -4000000;  // voxels = runs + end count
        return n;
    }
    const bool ymaj = (w.flags >> 5) & 1;
    int row, lo, hi;
    while (hd::run_next(w, row, lo, hi))
        if (!emit(ymaj, w.nmaj, row, lo, hi)) return -1000000;
    return n;
}
// the tiled traversal's byte-offset cursor on a lean walk in a box of
// dx x dy x dz voxels: its +inc / -inc updates are applied to a copy of the
// padded word layout (each half kept as a plain integer), decoded by prefix
// sums along x (low halves) and y (high halves), and the voxels with a
// nonzero count are returned as box-linear indices (x fastest).  Returns
// -1 when the walk has no lean form, -5000000 when an offset falls outside
// the box's words or is not word-aligned, -6000000 when a voxel is counted
// other than once, -7000000 when the run count disagrees with the cursor.
extern "C" int hx_tile_cursor(const int32_t *gi, const int32_t *go, int dx, int dy, int dz,
                              int32_t *out, int cap, int *nruns)
{
    hd::RunWalk w;
    *nruns = 0;
    if (!hd::run_begin(w, gi, go, dx, dy, dz)) return 0;
    hd::LeanWalk L;
    if (!hd::lean_of(w, L)) return -1;
    uint32_t o[hd::kLeanWords];
    hd::lean_pack(L, o);
    hd::TileCursor c;
    if (!hd::tile_cursor_start(o, dx, dy, dz, 0, c)) return 0;
    const int Wx = dx + 1, Hy = dy + 1;
    const long long words = (long long)Wx * Hy * dz;
    std::vector<long long> lo(words, 0), hi(words, 0);
    const int k0 = c.kleft;
    int runs = 0;
    bool more;
    do {
        int p, m;
        const uint32_t vp = c.vprev, vc = c.vcur;
        more = hd::tile_cursor_run(c, p, m);
        ++runs;
        if (p < 0 || m < 0 || (p & 3) || (m & 3) || p / 4 >= words || m / 4 >= words) return -5000000;
        // each value is +-1 in one half of a word
        auto apply = [&](int at, uint32_t v) {
            if (v == 1u) lo[at / 4] += 1;
            else if (v == 0xffffffffu) lo[at / 4] -= 1;
            else if (v == 65536u) hi[at / 4] += 1;
            else if (v == 0xffff0000u) hi[at / 4] -= 1;
            else return false;
            return true;
        };
        if (!apply(p, vp) || !apply(m, vc)) return -5000000;
        if (runs > 100000) return -5000000;
    } while (more);
    if (k0 - c.kleft != runs) return -7000000;
    *nruns = runs;
    int n = 0;
    for (int z = 0; z < dz; ++z)
        for (int y = 0; y < dy; ++y)
            for (int x = 0; x < dx; ++x) {
                long long sx = 0, sy = 0;
                for (int i = 0; i <= x; ++i) sx += lo[i + (long long)Wx * (y + Hy * z)];
                for (int j = 0; j <= y; ++j) sy += hi[x + (long long)Wx * (j + Hy * z)];
                const long long v = sx + sy;
                if (v != 0 && v != 1) return -6000000;
                if (v) {
                    if (n < cap) out[n] = x + dx * (y + dy * z);
                    ++n;
                }
            }
    return n;
}
// the direct one-slice set-up against the general one: returns 1 when both
// give the same packed lean walk, 2 when both find no voxel, 3 when the
// direct one declines (-1) and the general one is lean or not, 4 when both
// decline; negative on a disagreement (-10: emptiness differs, -11: the
// direct one is lean where the general one is not, -12: packed words differ)
extern "C" int hx_slab_lean(const int32_t *gi, const int32_t *go, int nx, int ny)
{
    hd::LeanWalk Ld;
    const int rd = hd::slab_lean(gi, go, nx, ny, Ld);
    hd::RunWalk w;
    const bool nonempty = hd::run_begin(w, gi, go, nx, ny, 1);
    hd::LeanWalk Lg;
    const bool lean = nonempty && hd::lean_of(w, Lg);
    if (rd == 0) return nonempty ? -10 : 2;
    if (rd < 0) return lean ? 3 : 4;
    if (!nonempty) return -10;
    if (!lean) return -11;
    uint32_t a[hd::kLeanWords], b[hd::kLeanWords];
    hd::lean_pack(Ld, a);
    hd::lean_pack(Lg, b);
    for (int i = 0; i < hd::kLeanWords; ++i)
        if (a[i] != b[i]) return -12;
    return 1;
}
// tile_range of a segment for a plan of (tx, ty, tz) tiles over the grid
extern "C" int hx_tile_range(const int32_t *r, int nx, int ny, int nz, int tx, int ty, int tz,
                             int32_t *lo, int32_t *hi)
{
    hd::TilePlan tp{};
    tp.nx = nx; tp.ny = ny; tp.nz = nz;
    tp.tx = tx; tp.ty = ty; tp.tz = tz;
    auto magic = [](int t) { return t == 1 ? 0u : static_cast<unsigned>((1ull << 32) / static_cast<unsigned>(t)) + 1u; };
    tp.mtx = magic(tx); tp.mty = magic(ty); tp.mtz = magic(tz);
    int l[3], h[3];
    const int c = hd::tile_range(tp, r, l, h);
    for (int a = 0; a < 3; ++a) { lo[a] = l[a]; hi[a] = h[a]; }
    return c;
}

// The chunk split shared by the ingest and the scatter (hd_internal.cuh).
extern "C" void hx_chunk_split(long long n, int sm_count, int *blocks, long long *per_block)
{
    const hd::ChunkSplit c = hd::chunk_split(n, sm_count);
    *blocks = c.blocks;
    *per_block = c.per_block;
}

// The loop-free floor division against the looping one (hd_geom.cuh), for
// operand pairs whose quotient is below 2^20 in magnitude.
extern "C" long long hx_fdiv_small(long long a, long long b) { return hd::fdiv_small(a, b); }

// The Euclidean thick rays' row search (hd_euclid.cuh) against a voxel-by-
// voxel exact search: for every history the capsule is set up as the kernel
// does it, and every row of the grid is searched both ways (rows outside the
// capsule's index box must hold no voxel).  The float filter's certificates
// are checked at every centre, with the empty-row certificate around every
// centre of every nonempty row, the filtered row-meets test on every row and
// the band of candidate rows (k_range) around every meeting row of the box.
// st: [rows with voxels, voxels, interval
// mismatches, filter errors, centres settled by the exact test, centres
// tested, histories set up]; returns 0, or -1 on bad arguments.
#include "../../paper_1402_1720_gb300/csrc/hd_euclid.cuh"
extern "C" int hx_euclid_rows(int nx, int ny, int nz, float sx, float sy, float sz, float T,
                              const long long *theta, long long K, float d0, const float *ang,
                              const float *ui, const float *vi, const float *uo, const float *vo,
                              int n, long long *st)
{
    if (n < 0 || !(d0 >= 0.0f)) return -1;
    hd::GeomQ g = hd::make_geomq(nx, ny, nz, sx, sy, sz, T);
    hd::Cordic cd;
    for (int i = 0; i < 32; ++i) cd.theta[i] = theta[i];
    cd.K = K;
    const long long R = 2 * hd::q16_of(d0);
    for (int q = 0; q < 7; ++q) st[q] = 0;
    for (int h = 0; h < n; ++h) {
        long long c, s;
        hd::cordic_cs(hd::q16_of(ang[h]), cd, c, s);
        int32_t G[6];
        if (!hd::endpoints_cs(g, c, s, ui[h], vi[h], uo[h], vo[h], G)) continue;
        long long W[6];
        hd::world_cs(g, c, s, ui[h], vi[h], uo[h], vo[h], W);
        long long A[3], B[3];
        int blo[3], bhi[3];
        bool ymaj;
        float S;
        const bool box = hd::capsule_frame(g, W, R, A, B, ymaj, blo, bhi, S);
        hd::CapX cx;
        hd::capx_of(g, A, B, ymaj, R, cx);
        const hd::CapF cf = hd::capf_of(cx, S, R);
        st[6] += 1;
        for (int k = 0; k < cx.n[2]; ++k)
            for (int a = 0; a < cx.n[1]; ++a) {
                const hd::RowF r = hd::rowf_of(cf, a, k);
                int blo_i = -1, bhi_i = -2, cnt = 0;
                for (int i = 0; i < cx.n[0]; ++i) {
                    const bool in = hd::F_exact(cx, a, k, i) <= cx.T;
                    float e0;
                    const float d2 = hd::d2_filter(cf, r, i, e0);
                    st[5] += 1;
                    if ((d2 <= cf.Tin && !in) || (d2 > cf.Tout && in)) st[3] += 1;
                    if (!(d2 <= cf.Tin) && !(d2 > cf.Tout)) st[4] += 1;
                    if (in) {
                        if (blo_i < 0) blo_i = i;
                        if (bhi_i != i - 1 && bhi_i >= 0) st[2] += 1;  // not one interval
                        bhi_i = i;
                        ++cnt;
                    }
                }
                const bool inbox = box && a >= blo[1] && a <= bhi[1] && k >= blo[2] && k <= bhi[2];
                const bool meets = hd::row_meets_at(cf, cx, a, k);
                if (meets != hd::meets_exact(cx, a, k)) st[3] += 1;
                // a meeting row of the box lies in its band of k
                if (meets && inbox) {
                    int klo, khi;
                    hd::k_range(cf, a, blo[2], bhi[2], klo, khi);
                    if (k < klo || k > khi) st[3] += 1;
                }
                // the empty-row certificate around every centre of the row
                for (int j = 0; j < cx.n[0]; ++j)
                    if (cnt > 0 && hd::row_empty(cf, r, j)) st[3] += 1;
                // the row search on every row of the box, meeting or not
                int lo = 0, hi = -1;
                const bool got = inbox && hd::row_interval(cf, cx, a, k, lo, hi);
                if (cnt == 0) {
                    if (got) st[2] += 1;
                } else {
                    st[0] += 1;
                    st[1] += cnt;
                    if (!meets || !got || lo != blo_i || hi != bhi_i) st[2] += 1;
                }
            }
    }
    return 0;
}

// The run walk expanded in path order (each run from its start in the
// direction the major axis moves), as linear voxel indices.
extern "C" int hx_runs_path_order(const int32_t *gi, const int32_t *go, int nx, int ny, int nz,
                                  int32_t *out, int cap)
{
    hd::RunWalk w;
    int n = 0;
    if (!hd::run_begin(w, gi, go, nx, ny, nz)) return 0;
    const bool ymaj = (w.flags >> 5) & 1, up = w.flags & 1;
    int row, lo, hi;
    while (hd::run_next(w, row, lo, hi)) {
        for (int j = 0; j <= hi - lo; ++j) {
            const int m = up ? lo + j : hi - j;
            const int v = !ymaj ? m + nx * row : (row % nx) + nx * (m + ny * (row / nx));
            if (n < cap) out[n] = v;
            ++n;
        }
    }
    return n;
}

// The whole-grid walk as one-slice walks, slice by slice in the direction
// the path moves along z: each slice's walk from the direct one-slice set-up
// (slab_lean) stepped as a lean cursor, or from the general set-up when
// slab_lean declines; runs expanded in path order, as linear voxel indices.
extern "C" int hx_slices_path_order(const int32_t *gi, const int32_t *go, int nx, int ny, int nz,
                                    int32_t *out, int cap)
{
    int n = 0;
    hd::TilePlan tp{};
    tp.nx = nx;
    tp.ny = ny;
    tp.nz = nz;
    const int32_t r[6] = {gi[0], gi[1], gi[2], go[0], go[1], go[2]};
    int zlo, zhi;
    if (!hd::grid_z_range(tp, r, zlo, zhi)) return 0;
    const bool zup = go[2] >= gi[2];
    for (int t = 0; t <= zhi - zlo; ++t) {
        const int z = zup ? zlo + t : zhi - t;
        const int32_t a[3] = {gi[0], gi[1], gi[2] - (z << 16)};
        const int32_t b[3] = {go[0], go[1], go[2] - (z << 16)};
        const int zoff = z * nx * ny;
        hd::LeanWalk L;
        const int rl = hd::slab_lean(a, b, nx, ny, L);
        if (rl == 0) continue;
        if (rl == 1) {
            uint32_t o[hd::kLeanWords];
            hd::lean_pack(L, o);
            const bool ymaj = (L.fl >> 2) & 1;
            hd::LeanCursor c;
            if (!hd::lean_start(o, ymaj ? ny : nx, c)) continue;
            bool more = true;
            while (more) {
                int rb, lo, hi;
                unsigned ends = 0;
                const int start = c.ms;
                more = hd::lean_run(c, rb, lo, hi, ends);
                const bool up = start == lo;  // a run goes from where it starts
                for (int j = 0; j <= hi - lo; ++j) {
                    const int m = up ? lo + j : hi - j;
                    const int row = rb / (ymaj ? ny : nx);
                    const int v = zoff + (!ymaj ? m + nx * row : row + nx * m);
                    if (n < cap) out[n] = v;
                    ++n;
                }
            }
        } else {
            hd::RunWalk w;
            if (!hd::run_begin(w, a, b, nx, ny, 1)) continue;
            const bool ymaj = (w.flags >> 5) & 1, up = w.flags & 1;
            int row, lo, hi;
            while (hd::run_next(w, row, lo, hi)) {
                for (int j = 0; j <= hi - lo; ++j) {
                    const int m = up ? lo + j : hi - j;
                    const int v = zoff + (!ymaj ? m + nx * row : row + nx * m);
                    if (n < cap) out[n] = v;
                    ++n;
                }
            }
        }
    }
    return n;
}
