"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(never against the CUDA path).  CPU only."""
import math
import os

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = 65536


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split("|")])
    return rows


def _ints(s):
    return [int(x) for x in s.split()] if s.strip() else []


# ------------------------------------------------------------------ CORDIC
def test_cordic_table_matches_definition(oracle_mod):
    theta, K = oracle_mod.cordic_table()
    assert theta[0] == 45 << 30                 # atan(1) = 45 degrees
    for i in range(32):
        exact = math.atan(2.0 ** -i) * 180.0 / math.pi * 2.0 ** 30
        assert abs(theta[i] - exact) <= 0.5 + 1e-4
    # small-angle closed form: atan(x) = x - x^3/3 + ..., so for i >= 20
    # theta_i = round(2^(30-i) * 180/pi) to within one unit
    for i in range(20, 32):
        assert abs(theta[i] - 2.0 ** (30 - i) * 180.0 / math.pi) <= 1.0
    k = 2.0 ** 30
    for i in range(32):
        k /= math.sqrt(1.0 + 2.0 ** (-2 * i))
    assert abs(K - k) <= 0.5 + 1e-3


def test_cordic_cos_sin_error_bound(oracle_mod):
    rng = np.random.default_rng(0)
    angles = np.concatenate([np.arange(-720, 721, 0.25),
                             rng.uniform(-1e4, 1e4, 4000),
                             np.arange(0, 360, 90) + 1e-4])
    worst = 0.0
    for a in angles:
        aq = int(round(a * Q))
        c, s = oracle_mod.cordic(aq)
        ang = math.radians(aq / Q)
        worst = max(worst, abs(c / 2 ** 30 - math.cos(ang)), abs(s / 2 ** 30 - math.sin(ang)))
        # unit length up to the same error
        assert abs((c * c + s * s) / 2 ** 60 - 1.0) < 2 ** -24
    assert worst < 2 ** -26, worst


def test_cordic_quadrant_symmetry(oracle_mod):
    # rotating by 90 degrees maps (c, s) -> (-s, c) exactly (the quadrant step)
    for a in [0.0, 13.7, 44.99, 77.25]:
        aq = int(round(a * Q))
        c0, s0 = oracle_mod.cordic(aq)
        c1, s1 = oracle_mod.cordic(aq + 90 * Q)
        c2, s2 = oracle_mod.cordic(aq + 180 * Q)
        c4, s4 = oracle_mod.cordic(aq - 360 * Q)
        assert (c1, s1) == (-s0, c0)
        assert (c2, s2) == (-c0, -s0)
        assert (c4, s4) == (c0, s0)


# ---------------------------------------------------------------- geometry
def _float_grid(g, angle, u_in, v_in, u_out, v_out):
    phi = math.radians(float(np.float32(angle)))
    c, s = math.cos(phi), math.sin(phi)
    T = float(np.float32(g.T))
    pin = (-T * c - float(u_in) * s, -T * s + float(u_in) * c, float(v_in))
    pout = (T * c - float(u_out) * s, T * s + float(u_out) * c, float(v_out))
    n = (g.nx, g.ny, g.nz)
    sz = (g.sx, g.sy, g.sz)
    f = lambda p: [(p[a] + n[a] * sz[a] / 2) / sz[a] * Q for a in range(3)]
    return f(pin), f(pout)


def test_grid_endpoints_match_float64_geometry(oracle_mod):
    rng = np.random.default_rng(1)
    for g in [synth.geometry_for(1), synth.geometry_for(2), synth.geometry_for(3)]:
        for _ in range(400):
            ang = np.float32(rng.uniform(-400, 400))
            u0, v0, u1, v1 = (np.float32(x) for x in rng.uniform(-150, 150, 4))
            rej, gin, gout = oracle_mod.grid_endpoints(g, ang, u0, v0, u1, v1)
            assert not rej
            fin, fout = _float_grid(g, ang, u0, v0, u1, v1)
            # error: CORDIC (T * 2^-26 mm) plus quantisation, well under 4 Q16 units
            for a in range(3):
                assert abs(gin[a] - fin[a]) < 4 * (1 + 0.5 / min(g.sx, g.sy, g.sz))
                assert abs(gout[a] - fout[a]) < 4 * (1 + 0.5 / min(g.sx, g.sy, g.sz))


def test_grid_endpoints_exact_cases(oracle_mod):
    g = synth.Geometry(4, 4, 4, 1.0, 1.0, 2.0, 10.0)
    # angle 0: beam along +x; entry x = -10 mm -> grid (-10 + 2)/1 = -8 voxels
    rej, gin, gout = oracle_mod.grid_endpoints(g, 0.0, 0.5, 1.0, 0.5, 1.0)
    assert not rej
    assert abs(gin[0] - (-8 * Q)) <= 1 and abs(gout[0] - 12 * Q) <= 1
    assert abs(gin[1] - int(2.5 * Q)) <= 1
    assert gin[2] == int((1.0 + 4.0) / 2.0 * Q)   # z is not rotated: exact
    # angle 90: beam along +y, lateral along -x
    rej, gin, gout = oracle_mod.grid_endpoints(g, 90.0, 0.5, 0.0, 0.5, 0.0)
    assert abs(gin[1] - (-8 * Q)) <= 1 and abs(gin[0] - int(1.5 * Q)) <= 1


def test_grid_endpoints_reject_rules(oracle_mod):
    g = synth.geometry_for(1)
    ok = dict(angle=10.0, u_in=1.0, v_in=1.0, u_out=1.0, v_out=1.0)
    assert not oracle_mod.grid_endpoints(g, *ok.values())[0]
    for k in ok:
        for bad in [float("nan"), float("inf"), -float("inf")]:
            args = dict(ok)
            args[k] = bad
            assert oracle_mod.grid_endpoints(g, *args.values())[0]
    for k in ["u_in", "v_in", "u_out", "v_out"]:
        args = dict(ok)
        args[k] = 4096.0
        assert oracle_mod.grid_endpoints(g, *args.values())[0]
        args[k] = -4095.5
        assert not oracle_mod.grid_endpoints(g, *args.values())[0]
    args = dict(ok)
    args["angle"] = 1048576.0
    assert oracle_mod.grid_endpoints(g, *args.values())[0]
    # grid coordinates beyond 2^30 / 2^16 = 16384 voxels: tiny voxels, far points
    gsmall = synth.Geometry(8, 8, 8, 0.125, 0.125, 0.125, 100.0)
    args = dict(ok)
    args["v_in"] = 2500.0      # 2500 mm / 0.125 mm = 20000 voxels
    assert oracle_mod.grid_endpoints(gsmall, *args.values())[0]


# ---------------------------------------------------------------- voxel set
@pytest.mark.parametrize("row", _golden("voxel_set_cases.txt"), ids=lambda r: r[0])
def test_voxel_set_golden(oracle_mod, row):
    name, dims, gi, go, expect = row
    nx, ny, nz = _ints(dims)
    gin = [int(round(float(x) * Q)) for x in gi.split()]
    gout = [int(round(float(x) * Q)) for x in go.split()]
    got = oracle_mod.voxel_set(gin, gout, nx, ny, nz)
    assert got.tolist() == _ints(expect)
    assert oracle_mod.voxel_set_bruteforce(gin, gout, nx, ny, nz).tolist() == _ints(expect)


def _random_segments(rng, n, dims):
    nx, ny, nz = dims
    hi = np.array([nx, ny, nz]) * Q
    out = []
    for k in range(n):
        mode = k % 6
        if mode == 0:    # lattice points: every tie there is
            a = rng.integers(-2, np.array(dims) + 3) * Q
            b = rng.integers(-2, np.array(dims) + 3) * Q
        elif mode == 1:  # half-lattice points
            a = rng.integers(-4, 2 * np.array(dims) + 5) * (Q // 2)
            b = rng.integers(-4, 2 * np.array(dims) + 5) * (Q // 2)
        elif mode == 2:  # axis-aligned
            a = rng.integers(-Q, hi + Q)
            b = a.copy()
            ax = rng.integers(0, 3)
            b[ax] = rng.integers(-2 * Q, hi[ax] + 2 * Q)
        elif mode == 3:  # on a plane in one axis
            a = rng.integers(-Q, hi + Q)
            b = rng.integers(-Q, hi + Q)
            ax = rng.integers(0, 3)
            a[ax] = b[ax] = rng.integers(0, dims[ax] + 1) * Q
        elif mode == 4:  # short segments, including degenerate ones
            a = rng.integers(-Q, hi + Q)
            b = a + rng.integers(-2, 3, 3) * rng.integers(0, Q, 3)
        else:            # generic
            a = rng.integers(-3 * Q, hi + 3 * Q)
            b = rng.integers(-3 * Q, hi + 3 * Q)
        out.append((a.astype(np.int64), b.astype(np.int64)))
    return out


@pytest.mark.parametrize("dims", [(5, 4, 3), (1, 1, 1), (7, 1, 2), (3, 3, 3), (6, 5, 1)])
def test_voxel_set_equals_slab_test(oracle_mod, dims):
    rng = np.random.default_rng(sum(dims))
    for a, b in _random_segments(rng, 3000, dims):
        got = oracle_mod.voxel_set(a, b, *dims)
        ref = oracle_mod.voxel_set_bruteforce(a, b, *dims)
        assert np.array_equal(got, ref), (a.tolist(), b.tolist(), got, ref)


def test_voxel_set_axis_aligned_row(oracle_mod):
    # a segment along x at interior (y, z) that spans the grid visits exactly nx voxels
    nx, ny, nz = 37, 5, 3
    for yq, zq in [(1.3, 0.2), (4.999, 2.5), (0.0, 0.0)]:
        a = [-5 * Q, int(yq * Q), int(zq * Q)]
        b = [(nx + 5) * Q, int(yq * Q), int(zq * Q)]
        got = oracle_mod.voxel_set(a, b, nx, ny, nz)
        y, z = int(yq), int(zq)
        assert got.tolist() == [x + nx * (y + ny * z) for x in range(nx)]


def test_voxel_set_count_identity(oracle_mod):
    # a segment inside the grid with no two plane crossings at the same
    # parameter visits 1 + sum_a |floor(out_a) - floor(in_a)| voxels; a
    # same-direction tie merges two steps (one fewer), a mixed one adds the
    # corner voxel (one more)
    rng = np.random.default_rng(5)
    dims = (40, 30, 20)
    exact = 0
    for _ in range(500):
        a = rng.integers(Q, np.array(dims) * Q - Q) + 7
        b = rng.integers(Q, np.array(dims) * Q - Q) + 11
        got = oracle_mod.voxel_set(a, b, *dims)
        expect = 1 + int(np.abs((b >> 16) - (a >> 16)).sum())
        assert abs(len(got) - expect) <= 1
        exact += len(got) == expect
    assert exact >= 495


# ----------------------------------------------------------- classification
def test_classify_hand_cases(oracle_mod):
    w = np.array([0.999, 1.0, 3.0, 5.0, 5.0001, float("nan"), -float("inf"), float("inf"),
                  -2.0, np.nextafter(np.float32(1.0), np.float32(0))], dtype=np.float32)
    assert oracle_mod.classify(w).tolist() == [1, 0, 0, 0, 2, 0, 1, 2, 1, 1]


# ------------------------------------------------------------- accumulation
def test_single_history_reproduces_slab_test(oracle_mod):
    g = synth.Geometry(9, 7, 5, 1.0, 1.5, 2.0, 20.0)
    rng = np.random.default_rng(7)
    h = synth.tiny_random_case(rng, 200, g, span=1.0)
    for i in range(len(h)):
        one = h.take([i])
        acc = oracle_mod.accumulate(g, one)
        cls = oracle_mod.classify(one.wepl)[0]
        rej, gin, gout = oracle_mod.grid_endpoints(g, one.angle_deg[0], one.u_in[0],
                                                   one.v_in[0], one.u_out[0], one.v_out[0])
        ref = np.zeros(g.n_voxels, np.uint32)
        if cls in (1, 2) and not rej:
            ref[oracle_mod.voxel_set_bruteforce(gin, gout, g.nx, g.ny, g.nz)] = 1
        if cls == 1:
            assert np.array_equal(acc["N"], ref) and not acc["M"].any()
            assert np.array_equal(acc["H1_carved"], 1 - ref)
        elif cls == 2:
            assert np.array_equal(acc["M"], ref) and not acc["N"].any()
        else:
            assert not acc["N"].any() and not acc["M"].any()


def test_accumulate_sum_identities_and_order_invariance(oracle_mod):
    g = synth.Geometry(12, 10, 6, 1.0, 1.0, 2.5, 30.0)
    rng = np.random.default_rng(11)
    h = synth.tiny_random_case(rng, 3000, g)
    acc = oracle_mod.accumulate(g, h)
    # sum_v N(v) = sum_{i in I_L} |A_i| with |A_i| from the slab test
    cls = oracle_mod.classify(h.wepl)
    tot = {1: 0, 2: 0}
    for i in range(len(h)):
        if cls[i] == 0:
            continue
        rej, gin, gout = oracle_mod.grid_endpoints(g, h.angle_deg[i], h.u_in[i], h.v_in[i],
                                                   h.u_out[i], h.v_out[i])
        if not rej:
            tot[int(cls[i])] += len(oracle_mod.voxel_set_bruteforce(gin, gout, g.nx, g.ny, g.nz))
    assert int(acc["N"].sum()) == tot[1] == acc["stats"]["steps_miss"]
    assert int(acc["M"].sum()) == tot[2] == acc["stats"]["steps_hit"]
    assert np.array_equal(acc["H1_carved"], (acc["N"] == 0).astype(np.uint8))
    perm = rng.permutation(len(h))
    acc2 = oracle_mod.accumulate(g, h.take(perm))
    assert np.array_equal(acc["N"], acc2["N"]) and np.array_equal(acc["M"], acc2["M"])
    par = oracle_mod.accumulate_parallel(g, h, threads=3)
    assert np.array_equal(acc["N"], par["N"]) and np.array_equal(acc["M"], par["M"])
    assert acc["stats"] == par["stats"]


def test_sampled_voxel_counts_match_definition(oracle_mod):
    w = synth.make_config(1, fraction=0.1)
    g = w.geometry
    acc = oracle_mod.accumulate(g, w.histories)
    rng = np.random.default_rng(3)
    for _ in range(6):
        x, y, z = int(rng.integers(g.nx)), int(rng.integers(g.ny)), int(rng.integers(g.nz))
        v = x + g.nx * (y + g.ny * z)
        assert oracle_mod.count_through_voxel(g, w.histories, 1, x, y, z) == acc["N"][v]
        assert oracle_mod.count_through_voxel(g, w.histories, 2, x, y, z) == acc["M"][v]


def test_methods_mask_selects_classes(oracle_mod):
    g = synth.Geometry(8, 8, 4, 1.0, 1.0, 2.0, 20.0)
    h = synth.tiny_random_case(np.random.default_rng(2), 500, g)
    full = oracle_mod.accumulate(g, h)
    only_sm = oracle_mod.accumulate(g, h, oracle_mod.Params(methods=oracle_mod.SM))
    only_msc = oracle_mod.accumulate(g, h, oracle_mod.Params(methods=oracle_mod.MSC))
    assert not only_sm["N"].any() and np.array_equal(only_sm["M"], full["M"])
    assert not only_msc["M"].any() and np.array_equal(only_msc["N"], full["N"])


# ----------------------------------------------------------------- decisions
@pytest.mark.parametrize("row", _golden("msc_decision_cases.txt"), ids=lambda r: r[0])
def test_msc_golden(oracle_mod, row):
    name, dims, nt, nbhd, N, H2 = row
    dims = tuple(_ints(dims))
    got = oracle_mod.msc_decide(np.array(_ints(N), np.uint32), dims, int(nt), int(nbhd))
    assert got.tolist() == _ints(H2)


@pytest.mark.parametrize("row", _golden("sm_decision_cases.txt"), ids=lambda r: r[0])
def test_sm_golden(oracle_mod, row):
    name, dims, per_slice, nbhd, ge, M, Mt, slope, index, H3 = row
    dims = tuple(_ints(dims))
    r = oracle_mod.sm_decide(np.array(_ints(M), np.uint32), dims, int(per_slice), int(nbhd),
                             int(ge))
    assert r["Mt"].tolist() == _ints(Mt)
    assert r["slope"].tolist() == _ints(slope)
    assert r["index"].tolist() == _ints(index)
    assert r["H3"].tolist() == _ints(H3)


def test_sm_single_step_edge_sets_upper_value(oracle_mod):
    # a disc of value 40 on a background of 10: the steepest drop is 30 and
    # M_t is the disc value; H_3 is the disc
    nx = ny = 16
    yy, xx = np.mgrid[0:ny, 0:nx]
    disc = (xx - 7.5) ** 2 + (yy - 7.5) ** 2 < 25
    M = np.where(disc, 40, 10).astype(np.uint32).reshape(-1)
    r = oracle_mod.sm_decide(M, (nx, ny, 1))
    assert r["Mt"][0] == 40 and r["slope"][0] == 30
    assert np.array_equal(r["H3"], disc.reshape(-1).astype(np.uint8))


def test_msc_contains_sc(oracle_mod):
    # N(v) = 0 gives N(v) - N(w) <= 0 < N_t for every w, so H_1 is inside H_2
    w = synth.make_config(1, fraction=0.2)
    r = oracle_mod.run(w.geometry, w.histories, threads=4)
    assert np.all(r["H2"] >= r["H1"])
    assert np.array_equal(r["H1"], r["H1_carved"])


def test_sc_hull_contains_deep_object_voxels(oracle_mod):
    # Noise-free WEPL = chord * RSP.  A line through a point at depth d inside
    # a convex object has a chord of at least 2 d, so if a voxel's whole cube
    # lies at depth >= tau_L / (2 RSP) (+ a margin for the fixed-point path),
    # no missed line passes through it and SC keeps it (Sec. 3.2, Sec. 3.1).
    w = synth.make_config(1, noise_free=True, fraction=0.5)
    g = w.geometry
    r = oracle_mod.run(g, w.histories, threads=4)
    e = w.phantom[0]
    a, b, c = e.semi
    depth = 1.0 / (2 * e.rsp) + 0.05
    # conservative: shrink the ellipsoid by `depth` along each semi-axis and
    # require all 8 cube corners inside the shrunk ellipsoid
    keep = np.zeros(g.n_voxels, bool)
    for z in range(g.nz):
        for y in range(g.ny):
            for x in range(g.nx):
                ok = True
                for dx in (0, 1):
                    for dy in (0, 1):
                        for dz in (0, 1):
                            px = (x + dx) * g.sx - g.nx * g.sx / 2
                            py = (y + dy) * g.sy - g.ny * g.sy / 2
                            pz = (z + dz) * g.sz - g.nz * g.sz / 2
                            if (px / (a - depth)) ** 2 + (py / (b - depth)) ** 2 + \
                                    (pz / (c - depth)) ** 2 >= 1:
                                ok = False
                keep[x + g.nx * (y + g.ny * z)] = ok
    assert keep.sum() > 1000
    assert np.all(r["H1"][keep] == 1)
    assert np.all(r["H2"][keep] == 1)


# ----------------------------------------- FP64 geometry (reported, not gated)
def test_fp64_voxel_set_equals_exact_set_on_generic_segments(oracle_mod):
    """The FP64 statement of the set equals the exact rational one when the
    endpoints are exactly representable and the segment hits no edge or
    corner: generic Q16 endpoints agree in all but rare cases, and the rare
    ones differ by a voxel or two (a crossing within rounding of another)."""
    rng = np.random.default_rng(71)
    for dims in [(40, 30, 20), (64, 64, 8), (7, 1, 3)]:
        hi = np.array(dims) * Q
        same = 0
        trials = 3000
        for _ in range(trials):
            a = rng.integers(-Q, hi + Q)
            b = rng.integers(-Q, hi + Q)
            exact = oracle_mod.voxel_set(a, b, *dims)
            fp = oracle_mod.voxel_set_fp64(a / Q, b / Q, *dims)
            if np.array_equal(exact, fp):
                same += 1
            else:
                assert len(np.setxor1d(exact, fp)) <= 2
        assert same >= 0.995 * trials


def test_fp64_endpoints_close_to_fixed_point(oracle_mod):
    """Unquantised FP64 endpoints and the fixed-point ones differ by the
    quantisation only (Q16 rounding of u, v, T and the CORDIC's 2^-27)."""
    rng = np.random.default_rng(72)
    g = synth.geometry_for(2)
    h = synth.tiny_random_case(rng, 2000, g, span=1.2)
    for i in range(len(h)):
        args = [float(x[i]) for x in h.arrays()[:5]]
        rq, gin, gout = oracle_mod.grid_endpoints(g, *args)
        rf, fin, fout = oracle_mod.grid_endpoints_fp64(g, *args)
        assert rq == rf
        if not rq:
            assert np.max(np.abs(np.asarray(gin) / Q - fin)) < 1e-3
            assert np.max(np.abs(np.asarray(gout) / Q - fout)) < 1e-3


def test_fp64_comparison_reports_small_differences(oracle_mod):
    w = synth.make_config(1, fraction=0.2)
    r = oracle_mod.compare_fp64(w.geometry, w.histories, threads=4)
    assert r["histories"] > 30000 and r["histories_one_geometry_only"] == 0
    assert r["membership_diff_frac"] < 1e-3
    assert r["H1_diff_frac_of_hull"] < 1e-2 and r["H3_diff_frac_of_hull"] < 1e-2


# ------------------------ hull-restricted system-matrix rows (next row f1)
def _entry_parameter(a, b, v, dims):
    """The smallest t in [0, 1] with P(t) in voxel v's half-open cube, in
    exact fractions (None when the segment misses it)."""
    from fractions import Fraction
    lo, hi = Fraction(0), Fraction(1)
    for ax in range(3):
        p0, d = Fraction(int(a[ax]), Q), Fraction(int(b[ax]) - int(a[ax]), Q)
        k = v[ax]
        if d == 0:
            if not (k <= p0 < k + 1):
                return None
            continue
        t1, t2 = (k - p0) / d, (k + 1 - p0) / d
        lo = max(lo, min(t1, t2))
        hi = min(hi, max(t1, t2))
    return lo if lo <= hi else None


def test_voxel_path_order_is_entry_order(oracle_mod):
    """On generic segments (no edge or corner crossing) the path order is the
    voxels sorted by the parameter at which the segment enters them."""
    rng = np.random.default_rng(81)
    for dims in [(7, 6, 5), (12, 3, 4)]:
        hi = np.array(dims) * Q
        for _ in range(300):
            a = rng.integers(-Q, hi + Q)
            b = rng.integers(-Q, hi + Q)
            path = oracle_mod.voxel_path(a, b, *dims)
            assert np.array_equal(np.sort(path), oracle_mod.voxel_set(a, b, *dims))
            nx, ny, _ = dims
            coords = [(v % nx, (v // nx) % ny, v // (nx * ny)) for v in path]
            t = [_entry_parameter(a, b, c, dims) for c in coords]
            assert all(x is not None for x in t)
            assert all(t[i] <= t[i + 1] for i in range(len(t) - 1))


def test_voxel_path_steps_and_monotone(oracle_mod):
    """Every segment (ties included): consecutive voxels differ by at most one
    in each index, and each index moves only in the segment's direction."""
    rng = np.random.default_rng(82)
    for dims in [(5, 4, 3), (9, 9, 2)]:
        nx, ny, _ = dims
        for a, b in _random_segments(rng, 3000, dims):
            path = oracle_mod.voxel_path(a, b, *dims)
            assert np.array_equal(np.sort(path), oracle_mod.voxel_set(a, b, *dims))
            c = np.stack([path % nx, (path // nx) % ny, path // (nx * ny)], 1)
            if len(c) > 1:
                step = np.diff(c, axis=0)
                assert np.all(np.abs(step) <= 1)
                for ax in range(3):
                    d = int(b[ax]) - int(a[ax])
                    if d > 0:
                        assert np.all(step[:, ax] >= 0)
                    elif d < 0:
                        assert np.all(step[:, ax] <= 0)
                    else:
                        assert np.all(step[:, ax] == 0)


def test_system_rows_are_hull_filtered_paths(oracle_mod):
    """Rows with an all-ones hull are the exact voxel sets in path order
    (empty for rejected histories); with a random hull, the hull's voxels of
    each path in the same order."""
    rng = np.random.default_rng(83)
    g = synth.geometry_for(1)
    h = synth.tiny_random_case(rng, 1500, g, span=1.3)
    arrs = h.arrays()
    V = g.n_voxels
    for hull in (np.ones(V, np.uint8), (rng.random(V) < 0.4).astype(np.uint8)):
        row_ptr, cols = oracle_mod.system_rows(g, h, hull, threads=3)
        assert row_ptr[0] == 0 and len(cols) == row_ptr[-1]
        for i in range(len(h)):
            rej, gin, gout = oracle_mod.grid_endpoints(g, *[float(x[i]) for x in arrs[:5]])
            row = cols[row_ptr[i]:row_ptr[i + 1]]
            if rej:
                assert len(row) == 0
                continue
            path = oracle_mod.voxel_path(gin, gout, g.nx, g.ny, g.nz)
            assert np.array_equal(row, path[hull[path] != 0])
