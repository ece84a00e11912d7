"""Pins for the oracle's binned SC (Sec. 2.2 data cuts, Sec. 3.2 as the paper
ran SC): bin assignment against numpy's histogram, the 3 sigma cuts against
float64 statistics and Chebyshev's bound, the missed-bin decision and the
carved lines against the slab test of every voxel, and the averaging filter
against scipy's correlation."""
import math

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth

G_TINY = synth.Geometry(16, 16, 4, 1.0, 1.0, 2.5, 30.0)


def _hist(angle, u_in, v_in, u_out, v_out, wepl):
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))  # noqa: E731
    return synth.Histories(f(angle), f(u_in), f(v_in), f(u_out), f(v_out), f(wepl))


def _random_hist(rng, n, bp, wepl_lo=0.0, wepl_hi=20.0):
    n_ang = int(round(360 / bp.angle_bin_deg))
    ang = rng.integers(0, n_ang, n) * bp.angle_bin_deg + rng.uniform(-1.9, 1.9, n)
    um = rng.uniform(bp.u_lo_mm + 0.01, bp.u_lo_mm + bp.n_u * bp.u_bin_mm - 0.01, n)
    vm = rng.uniform(bp.v_lo_mm + 0.01, bp.v_lo_mm + bp.v_bins * bp.v_bin_mm - 0.01, n)
    du, dv = rng.normal(0, 1.0, n), rng.normal(0, 1.0, n)
    return _hist(np.mod(ang, 360.0), um - du / 2, vm - dv / 2, um + du / 2, vm + dv / 2,
                 rng.uniform(wepl_lo, wepl_hi, n))


def _bin_index_float64(h, bp):
    """Bins from numpy's histogramdd on float64 values."""
    n_ang = int(round(360 / bp.angle_bin_deg))
    a = np.mod(h.angle_deg.astype(np.float64) + bp.angle_bin_deg / 2, 360.0)
    um = (h.u_in.astype(np.float64) + h.u_out.astype(np.float64)) / 2
    vm = (h.v_in.astype(np.float64) + h.v_out.astype(np.float64)) / 2
    ea = np.arange(n_ang + 1) * bp.angle_bin_deg
    eu = bp.u_lo_mm + np.arange(bp.n_u + 1) * bp.u_bin_mm
    ev = bp.v_lo_mm + np.arange(bp.v_bins + 1) * bp.v_bin_mm
    cnt, _ = np.histogramdd(np.stack([vm, um, a], 1), bins=[ev, eu, ea])
    return cnt.astype(np.int64).ravel()  # v slowest, angle fastest


def test_bin_counts_match_histogram(oracle_mod):
    bp = oracle_mod.binned_params_for(G_TINY)
    h = _random_hist(np.random.default_rng(1), 20000, bp)
    r = oracle_mod.sc_binned(G_TINY, h, bp)
    assert np.array_equal(r["bins"][:, 0], _bin_index_float64(h, bp))
    assert r["stats"]["binned"] == len(h)


def test_angle_bins_are_centred_and_wrap(oracle_mod):
    bp = oracle_mod.binned_params_for(G_TINY)
    angles = [0.0, 4.0, 8.0, 358.0, 1.999, 2.0, -2.0, 362.0, 180.0, 357.999]
    want = [0, 1, 2, 0, 0, 1, 0, 1, 45, 89]  # 362 = 2: the lower edge of bin 1
    h = _hist(angles, [0.2] * 10, [0.2] * 10, [0.2] * 10, [0.2] * 10, [9.0] * 10)
    r = oracle_mod.sc_binned(G_TINY, h, bp)
    iu = int(math.floor(0.2 - bp.u_lo_mm))
    iv = int(math.floor((0.2 - bp.v_lo_mm) / bp.v_bin_mm))
    base = 90 * (iu + bp.n_u * iv)
    got = np.zeros(90, np.int64)
    got[:] = r["bins"][base:base + 90, 0]
    exp = np.bincount(want, minlength=90)
    assert np.array_equal(got, exp)


def test_sums_match_float64_within_rounding(oracle_mod):
    bp = oracle_mod.binned_params_for(G_TINY)
    h = _random_hist(np.random.default_rng(2), 20000, bp)
    r = oracle_mod.sc_binned(G_TINY, h, bp)
    bins = r["bins"]
    idx = _bin_of_each(h, bp)
    nb = bp.n_bins
    for q, x in enumerate([h.wepl, h.u_out.astype(np.float64) - h.u_in,
                           h.v_out.astype(np.float64) - h.v_in]):
        s = np.bincount(idx, weights=x.astype(np.float64), minlength=nb)
        # each value is rounded to 1/256 mm (a slope from two roundings)
        tol = bins[:, 0] * (1.0 / 256 if q else 0.5 / 256) + 1e-9
        assert np.all(np.abs(bins[:, 1 + q] / 256.0 - s) <= tol)


def _bin_of_each(h, bp):
    """Each history's bin from float64 arithmetic (ties avoided by the inputs)."""
    n_ang = int(round(360 / bp.angle_bin_deg))
    a = np.floor(np.mod(h.angle_deg.astype(np.float64) + bp.angle_bin_deg / 2, 360.0)
                 / bp.angle_bin_deg).astype(np.int64) % n_ang
    um = (h.u_in.astype(np.float64) + h.u_out.astype(np.float64)) / 2
    vm = (h.v_in.astype(np.float64) + h.v_out.astype(np.float64)) / 2
    iu = np.floor((um - bp.u_lo_mm) / bp.u_bin_mm).astype(np.int64)
    iv = np.floor((vm - bp.v_lo_mm) / bp.v_bin_mm).astype(np.int64)
    return a + n_ang * (iu + bp.n_u * iv)


def test_cuts_match_float64_sigma(oracle_mod):
    """Kept histories per bin equal those within 3 population standard
    deviations by numpy's mean and std of the 1/256 mm values, in every bin
    where no value lies within 1e-9 of the boundary."""
    bp = oracle_mod.binned_params_for(G_TINY, angle_bin_deg=90.0)
    rng = np.random.default_rng(3)
    h = _random_hist(rng, 30000, bp)
    h.wepl[rng.random(len(h)) < 0.02] = 400.0  # outliers the cut should remove
    r = oracle_mod.sc_binned(G_TINY, h, bp)
    idx = _bin_of_each(h, bp)
    xs = [np.rint(h.wepl.astype(np.float64) * 256) / 256,
          (np.rint(h.u_out.astype(np.float64) * 256) - np.rint(h.u_in.astype(np.float64) * 256))
          / 256,
          (np.rint(h.v_out.astype(np.float64) * 256) - np.rint(h.v_in.astype(np.float64) * 256))
          / 256]
    order = np.argsort(idx, kind="stable")
    bounds = np.flatnonzero(np.diff(np.r_[-1, idx[order], -2]))
    checked = 0
    cut_total = 0
    for s, e in zip(bounds[:-1], bounds[1:]):
        sel = order[s:e]
        keep = np.ones(len(sel), bool)
        near = False
        for x in xs:
            v = x[sel]
            d = np.abs(v - v.mean())
            lim = 3 * v.std()
            near |= bool(np.any(np.abs(d - lim) < 1e-9 * max(1.0, lim)))
            keep &= d <= lim
        if near:
            continue
        b = idx[sel[0]]
        assert r["bins"][b, 7] == keep.sum()
        assert r["bins"][b, 8] == int(np.rint(xs[0][sel][keep] * 256).sum())
        checked += 1
        cut_total += int((~keep).sum())
    assert checked > 100 and cut_total > 0
    assert r["stats"]["cut"] >= cut_total


def test_cut_keeps_a_value_at_exactly_three_sigma(oracle_mod):
    """Nine zeros and one a: |a - a/10| = 0.9 a = 3 sigma exactly, so it stays
    (only values beyond 3 sigma are cut); nineteen zeros and one a put a at
    sqrt(19) sigma, beyond, so it is cut."""
    bp = oracle_mod.binned_params_for(G_TINY)
    for n0, kept in ((9, 10), (19, 19)):
        w = [0.0] * n0 + [10.0]
        n = len(w)
        h = _hist([0.0] * n, [0.3] * n, [0.3] * n, [0.3] * n, [0.3] * n, w)
        r = oracle_mod.sc_binned(G_TINY, h, bp)
        b = np.flatnonzero(r["bins"][:, 0])
        assert len(b) == 1 and r["bins"][b[0], 7] == kept


def test_cuts_obey_chebyshev(oracle_mod):
    """At most 1/9 of a bin lies beyond 3 sigma in any one variable, so at
    most a third of it is cut."""
    w = synth.make_config(1, fraction=0.5)
    bp = oracle_mod.binned_params_for(w.geometry)
    r = oracle_mod.sc_binned(w.geometry, w.histories, bp)
    n, kept = r["bins"][:, 0], r["bins"][:, 7]
    assert np.all(3 * (n - kept) <= n)
    assert r["stats"]["cut"] == int((n - kept).sum()) > 0


def _expected_carve(oracle_mod, g, bp, missed):
    """Carved image of the missed bins from the bin centres written out here
    and the slab test of every voxel."""
    carved = np.ones(g.nx * g.ny * g.nz, np.uint8)
    n_ang = int(round(360 / bp.angle_bin_deg))
    for b in missed:
        ia, iu, iv = b % n_ang, (b // n_ang) % bp.n_u, b // (n_ang * bp.n_u)
        la = ia * bp.angle_bin_deg
        lu = bp.u_lo_mm + (iu + 0.5) * bp.u_bin_mm
        vlo = bp.v_lo_mm + iv * bp.v_bin_mm
        for z in range(g.nz):
            zc = (z + 0.5) * g.sz - g.nz * g.sz / 2
            if not (vlo <= zc < vlo + bp.v_bin_mm):
                continue
            rej, gi, go = oracle_mod.grid_endpoints(g, la, lu, zc, lu, zc)
            if rej:
                continue
            vox = oracle_mod.voxel_set_bruteforce(gi, go, g.nx, g.ny, g.nz)
            carved[vox] = 0
    return carved


def test_missed_bins_carve_their_lines(oracle_mod):
    """Bins of mean kept WEPL 0.9 mm are carved, 1.1 mm are not; the carved
    voxels are exactly those the slab test puts on the missed bins' lines,
    one line per slice whose centre lies in the bin."""
    g = G_TINY
    bp = oracle_mod.binned_params_for(g)
    rng = np.random.default_rng(5)
    n_ang = 90
    picks = rng.choice(bp.n_bins, 60, replace=False)
    rows = []
    missed = []
    for j, b in enumerate(picks):
        ia, iu, iv = b % n_ang, (b // n_ang) % bp.n_u, b // (n_ang * bp.n_u)
        mean = 0.9 if j % 2 == 0 else 1.1
        if mean < 1.0:
            missed.append(int(b))
        for w in (mean - 0.25, mean + 0.25):
            a = 4.0 * ia + 0.5
            u = bp.u_lo_mm + iu + 0.5
            v = bp.v_lo_mm + bp.v_bin_mm * iv + 2.0
            rows.append((a, u, v, u, v, w))
    h = _hist(*np.asarray(rows).T)
    r = oracle_mod.sc_binned(g, h, bp)
    assert r["stats"]["bins_missed"] == len(missed)
    assert np.array_equal(r["carved"], _expected_carve(oracle_mod, g, bp, missed))


def test_filter_is_zero_padded_window_count(oracle_mod):
    ndimage = pytest.importorskip("scipy.ndimage")
    w = synth.make_config(1, fraction=0.2)
    g = w.geometry
    bp = oracle_mod.binned_params_for(g)
    r = oracle_mod.sc_binned(g, w.histories, bp)
    c = r["carved"].reshape(g.nz, g.ny, g.nx).astype(np.int64)
    cnt = ndimage.correlate(c, np.ones((1, 5, 5), np.int64), mode="constant", cval=0)
    assert np.array_equal(r["mask"], (cnt >= 11).astype(np.uint8).ravel())
    assert 0 < r["mask"].sum() < g.nx * g.ny * g.nz


def test_nothing_missed_keeps_all_but_corners(oracle_mod):
    """With no missed bin the filtered image is the window count of an
    all-ones slice: a corner window holds 9 voxels (out), the voxels next to
    a corner 12 (in)."""
    g = G_TINY
    bp = oracle_mod.binned_params_for(g)
    h = _random_hist(np.random.default_rng(6), 2000, bp, wepl_lo=5.0, wepl_hi=9.0)
    r = oracle_mod.sc_binned(g, h, bp)
    assert r["stats"]["bins_missed"] == 0 and r["carved"].all()
    m = r["mask"].reshape(g.nz, g.ny, g.nx)
    corner = np.zeros((g.ny, g.nx), bool)
    for y in (0, g.ny - 1):
        for x in (0, g.nx - 1):
            corner[y, x] = True
    for z in range(g.nz):
        assert np.array_equal(m[z].astype(bool), ~corner)


def test_unbinnable_histories_are_skipped(oracle_mod):
    g = G_TINY
    bp = oracle_mod.binned_params_for(g)
    h = _hist([0, np.nan, 0, 0, 0, 0], [0, 0, 500.0, 0, 0, 0], [0, 0, 0, 0, 0, 0],
              [0, 0, 0, 2000.0, 0, 0], [0, 0, 0, 0, 0, 0], [1, 1, 1, 1, 1500.0, np.inf])
    r = oracle_mod.sc_binned(g, h, bp)
    # NaN angle; mid-point outside the bins; slope >= 1024 mm; WEPL >= 1024 mm; inf
    assert r["stats"]["binned"] == 1
