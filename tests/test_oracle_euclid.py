"""Pins of the oracle's Euclidean thick rays (Eq. 3.2 with d_0 > 0, d the
Euclidean distance from the voxel centre to the closed segment L_i).

The membership test is checked against the textbook point-to-segment
distance computed with exact rationals (projection parameter clamped to
[0, 1]), a different formulation from the oracle's case split with a cross
product; the accumulation is checked against a test of every voxel of small
grids (so its bounding box loses nothing), a closed form for a segment along
a row of voxel centres, the containment of the thin set A_i (d_0 = 0 read
against voxel cubes) once d_0 reaches the voxel's half diagonal, and
monotonicity in d_0."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth


def _dist2_exact(A, B, C):
    u = [Fraction(int(b) - int(a)) for a, b in zip(A, B)]
    w = [Fraction(int(c) - int(a)) for a, c in zip(A, C)]
    uu = sum(x * x for x in u)
    t = Fraction(0) if uu == 0 else min(Fraction(1), max(Fraction(0), sum(
        x * y for x, y in zip(w, u)) / uu))
    return sum((wi - t * ui) ** 2 for wi, ui in zip(w, u))


def test_in_capsule_equals_exact_rational_distance(oracle_mod):
    rng = np.random.default_rng(41)
    cases = 0
    for scale in (2**8, 2**20, 2**29 - 1):
        for _ in range(1500):
            A = rng.integers(-scale, scale, 3)
            B = A.copy() if rng.random() < 0.05 else rng.integers(-scale, scale, 3)
            C = rng.integers(-scale, scale, 3)
            if rng.random() < 0.3:  # near the segment
                t = rng.random()
                C = (A + t * (B - A)).astype(np.int64) + rng.integers(-scale // 64 - 2,
                                                                      scale // 64 + 2, 3)
            d2 = _dist2_exact(A, B, C)
            R = int(rng.integers(0, 2**23))
            if rng.random() < 0.3:  # a radius at the exact distance, or one unit around it
                r = int(np.floor(float(d2) ** 0.5))
                R = min(2**23, max(0, r + int(rng.integers(-1, 2))))
            assert oracle_mod.in_capsule(A, B, C, R) == (d2 <= R * R), (A, B, C, R)
            cases += 1
    assert cases == 4500


def test_in_capsule_boundaries_and_degenerate_segment(oracle_mod):
    A, B = np.array([0, 0, 0]), np.array([1000, 0, 0])
    # perpendicular offset exactly R from the segment's interior: inside
    assert oracle_mod.in_capsule(A, B, np.array([500, 30, 40]), 50)
    assert not oracle_mod.in_capsule(A, B, np.array([500, 30, 40]), 49)
    # beyond the ends: the distance is to the end point
    assert oracle_mod.in_capsule(A, B, np.array([1030, 40, 0]), 50)
    assert not oracle_mod.in_capsule(A, B, np.array([1030, 41, 0]), 50)
    assert oracle_mod.in_capsule(A, B, np.array([-30, 0, 40]), 50)
    # a point segment is a ball
    P = np.array([7, -3, 2])
    assert oracle_mod.in_capsule(P, P, np.array([10, 1, 2]), 5)
    assert not oracle_mod.in_capsule(P, P, np.array([10, 1, 3]), 5)


def _all_voxels(oracle_mod, g, A, B, R):
    out = []
    for z in range(g.nz):
        for y in range(g.ny):
            for x in range(g.nx):
                if oracle_mod.in_capsule(A, B, oracle_mod.voxel_centre2(g, x, y, z), R):
                    out.append(x + g.nx * (y + g.ny * z))
    return np.array(out, np.int64)


@pytest.mark.parametrize("d0", [0.5, 1.0, 2.5])
def test_accumulation_equals_every_voxel_test(oracle_mod, d0):
    """Single histories on a small grid: the counted voxels are exactly the
    voxels of the whole grid whose centre passes the test."""
    g = synth.Geometry(12, 10, 5, 1.0, 1.5, 2.5, 20.0)
    rng = np.random.default_rng(int(d0 * 10))
    h = synth.tiny_random_case(rng, 40, g, span=1.2)
    h.wepl[:] = 0.5  # all missed
    for i in range(len(h)):
        one = h.take([i])
        rej, A, B, R = oracle_mod.capsule_of(g, d0, *[a[0] for a in one.arrays()[:5]])
        acc = oracle_mod.accumulate_euclid(g, one, d0)
        got = np.flatnonzero(acc["N"])
        if rej:
            assert got.size == 0 and acc["stats"][4] == 1
            continue
        assert np.array_equal(got, _all_voxels(oracle_mod, g, A, B, R))
        assert acc["stats"][5] == got.size and acc["N"].max(initial=0) <= 1


def test_row_closed_form(oracle_mod):
    """A segment along x through the centres of row (j, k): with d_0 below
    the in-plane and slice spacings only that row is reached, at the voxels
    whose centre lies within d_0 of the segment's x range."""
    g = synth.Geometry(20, 9, 4, 1.0, 1.0, 2.5, 50.0)
    j, k = 4, 2
    c = oracle_mod.voxel_centre2(g, 0, j, k)
    for d0, (x0, x1) in [(0.4, (-3.0, 4.2)), (0.75, (-7.5, 7.5)), (0.5, (-2.25, 3.5))]:
        A = np.array([int(x0 * 2**17), c[1], c[2]])
        B = np.array([int(x1 * 2**17), c[1], c[2]])
        R = 2 * int(round(d0 * 65536))
        got = _all_voxels(oracle_mod, g, A, B, R)
        xs = [(2 * x + 1 - g.nx) / 2 for x in range(g.nx)]
        want = [x + g.nx * (j + g.ny * k) for x in range(g.nx)
                if x0 - d0 <= xs[x] <= x1 + d0]
        assert np.array_equal(got, np.array(want, np.int64)), d0


def test_contains_thin_set_and_grows_with_d0(oracle_mod):
    """Every voxel whose cube the segment meets has its centre within half
    a voxel diagonal of the segment, so from that d_0 on the thick counts
    dominate the thin ones voxel by voxel; and counts grow with d_0."""
    w = synth.make_config(1, fraction=0.01)
    g, h = w.geometry, w.histories
    thin = oracle_mod.accumulate(g, h)
    half_diag = 0.5 * float(np.sqrt(g.sx ** 2 + g.sy ** 2 + g.sz ** 2))
    prev = None
    for d0 in sorted((0.5, 1.0, 1.5, half_diag + 0.01, 2.5)):
        acc = oracle_mod.accumulate_euclid(g, h, d0, threads=8)
        if d0 > half_diag:
            assert np.all(acc["N"] >= thin["N"]) and np.all(acc["M"] >= thin["M"])
        if prev is not None:
            assert np.all(acc["N"] >= prev["N"]) and np.all(acc["M"] >= prev["M"])
        assert acc["stats"][5] == int(acc["N"].sum()) and acc["stats"][6] == int(acc["M"].sum())
        prev = acc
    for k in range(5):
        assert prev["stats"][k] == list(thin["stats"].values())[k]
