"""Pins for the oracle's thick rays (next row f4): k = 0 reduces to the thin
counts, single-history sets equal an exact slab test on the dilated box
written here with rationals, sums equal the set sizes, and counts grow with
k."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth
from tests.test_oracle_pins import _random_segments


def _meets_box(a, b, lo, hi):
    """Does the closed segment a -> b meet the half-open box [lo, hi)?"""
    t_lo, lo_open = Fraction(0), False
    t_hi, hi_open = Fraction(1), False
    for ax in range(3):
        d = b[ax] - a[ax]
        if d == 0:
            if not (lo[ax] <= a[ax] < hi[ax]):
                return False
            continue
        if d > 0:
            l, lop = (lo[ax] - a[ax]) / d, False  # p >= lo: t >= l (closed)
            h, hop = (hi[ax] - a[ax]) / d, True   # p < hi: t < h (open)
        else:
            l, lop = (hi[ax] - a[ax]) / d, True   # p < hi: t > l (open)
            h, hop = (lo[ax] - a[ax]) / d, False  # p >= lo: t <= h (closed)
        if l > t_lo or (l == t_lo and lop):
            t_lo, lo_open = l, lop
        if h < t_hi or (h == t_hi and hop):
            t_hi, hi_open = h, hop
    return t_lo < t_hi or (t_lo == t_hi and not lo_open and not hi_open)


def test_k0_equals_thin_counts(oracle_mod):
    w = synth.make_config(1, fraction=0.2)
    thick = oracle_mod.accumulate_thick(w.geometry, w.histories, 0)
    thin = oracle_mod.accumulate(w.geometry, w.histories)
    assert np.array_equal(thick["N"], thin["N"]) and np.array_equal(thick["M"], thin["M"])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_single_histories_equal_dilated_slab_test(oracle_mod, k):
    g = synth.Geometry(12, 10, 4, 1.0, 1.0, 2.5, 20.0)
    rng = np.random.default_rng(10 + k)
    done = 0
    while done < 25:
        ang = float(rng.choice([0.0, 90.0, 45.0, 4.0 * rng.integers(0, 90),
                                rng.uniform(0, 360)]))
        u0, u1 = rng.uniform(-7, 7, 2)
        v0, v1 = rng.uniform(-5, 5, 2)
        if rng.random() < 0.3:
            v1 = v0
        rej, gi, go = oracle_mod.grid_endpoints(g, ang, u0, v0, u1, v1)
        if rej:
            continue
        h = synth.Histories(*[np.array([x], np.float32) for x in (ang, u0, v0, u1, v1, 0.5)])
        r = oracle_mod.accumulate_thick(g, h, k)
        a = [Fraction(int(c), 65536) for c in gi]
        b = [Fraction(int(c), 65536) for c in go]
        want = np.zeros(g.nx * g.ny * g.nz, np.uint32)
        for z in range(g.nz):
            for y in range(g.ny):
                for x in range(g.nx):
                    lo = [max(x - k, 0), max(y - k, 0), z]
                    hi = [min(x + k + 1, g.nx), min(y + k + 1, g.ny), z + 1]
                    want[x + g.nx * (y + g.ny * z)] = _meets_box(a, b, lo, hi)
        assert np.array_equal(r["N"], want), (ang, u0, v0, u1, v1)
        done += 1


def test_sums_and_growth(oracle_mod):
    w = synth.make_config(1, fraction=0.1)
    prev = None
    for k in range(4):
        r = oracle_mod.accumulate_thick(w.geometry, w.histories, k)
        assert int(r["N"].sum()) == int(r["stats"][5]) and int(r["M"].sum()) == int(r["stats"][6])
        if prev is not None:
            assert np.all(r["N"] >= prev["N"]) and np.all(r["M"] >= prev["M"])
        prev = r


def test_box_test_equals_rational_slab_test(oracle_mod):
    """The oracle's box slab test against the rational one written here, on
    random segments and boxes (ties on box faces included)."""
    rng = np.random.default_rng(31)
    for _ in range(3000):
        a = rng.integers(-3 * 65536, 12 * 65536, 3)
        b = rng.integers(-3 * 65536, 12 * 65536, 3)
        if rng.random() < 0.3:
            a = (a // 65536) * 65536  # on lattice planes
        if rng.random() < 0.2:
            b[2] = a[2]
        lo = rng.integers(0, 8, 3)
        hi = lo + rng.integers(1, 5, 3)
        want = _meets_box([Fraction(int(c), 65536) for c in a],
                          [Fraction(int(c), 65536) for c in b], list(lo), list(hi))
        assert oracle_mod.segment_meets_box(a, b, lo, hi) == want


def test_count_thick_voxels_equals_accumulation(oracle_mod):
    w = synth.make_config(1, fraction=0.05)
    g = w.geometry
    r = oracle_mod.accumulate_thick(g, w.histories, 2)
    vox = np.random.default_rng(32).choice(g.nx * g.ny * g.nz, 40, replace=False)
    assert np.array_equal(oracle_mod.count_thick_voxels(g, w.histories, 2, 1, vox), r["N"][vox])
    assert np.array_equal(oracle_mod.count_thick_voxels(g, w.histories, 2, 2, vox), r["M"][vox])


def test_run_thick_k0_is_run(oracle_mod):
    """At k = 0 the thick-ray run is the thin run: counts, hulls, thresholds."""
    w = synth.make_config(1, fraction=0.1)
    a = oracle_mod.run_thick(w.geometry, w.histories, 0)
    b = oracle_mod.run(w.geometry, w.histories)
    for key in ("N", "M", "H1", "H2", "H3", "Mt"):
        assert np.array_equal(a[key], b[key]), key


def test_unit_box_is_the_voxel_test(oracle_mod):
    """A box of one voxel is the voxel slab test of the thin sets."""
    rng = np.random.default_rng(34)
    dims = (6, 5, 4)
    for a, b in _random_segments(rng, 1500, dims):
        x, y, z = (int(rng.integers(0, d)) for d in dims)
        assert oracle_mod.segment_meets_box(a, b, [x, y, z], [x + 1, y + 1, z + 1]) == \
            oracle_mod.segment_meets_voxel(a, b, x, y, z)
