"""Pins for the oracle's hull diagnostics (next row f3): the enclosed-region
fill against scipy's hole filling and hand-built slices, the extra/missing
counts against their set identities and a hand case, and the filled MSC hull
on the tiny workload."""
import numpy as np
import pytest

from paper_1402_1720_gb300 import synth


def _ring(n, gap=None):
    """An n x n slice of ones with a one-voxel square ring of zeros (the
    shell) from (1, 1) to (n - 2, n - 2); `gap` opens one ring voxel."""
    m = np.ones((n, n), np.uint8)
    m[1, 1:n - 1] = 0
    m[n - 2, 1:n - 1] = 0
    m[1:n - 1, 1] = 0
    m[1:n - 1, n - 2] = 0
    if gap is not None:
        m[gap] = 1
    return m


def test_fill_hand_cases(oracle_mod):
    n = 7
    m = _ring(n)
    out = oracle_mod.fill_enclosed(m, (n, n, 1)).reshape(n, n)
    want = np.zeros((n, n), np.uint8)
    want[2:n - 2, 2:n - 2] = 1
    assert np.array_equal(out, want)
    # an opening in the side of the ring joins the inside to the border
    side = _ring(n, gap=(1, 3))
    assert oracle_mod.fill_enclosed(side, (n, n, 1)).sum() == 0
    # a diagonal step is not a 4-connected path: the inside stays enclosed
    d = _ring(n)
    d[1, 1] = 1  # the corner voxel joins the border only diagonally to the inside
    assert np.array_equal(oracle_mod.fill_enclosed(d, (n, n, 1)).reshape(n, n), want)
    # no shell: everything reaches the border
    assert oracle_mod.fill_enclosed(np.ones((5, 4, 2), np.uint8), (4, 5, 2)).sum() == 0


def test_fill_equals_scipy_hole_filling(oracle_mod):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    cross = ndimage.generate_binary_structure(2, 1)
    for nx, ny, nz, p in [(17, 13, 3, 0.35), (31, 29, 2, 0.45), (8, 40, 4, 0.25), (1, 6, 2, 0.5)]:
        shell = rng.random((nz, ny, nx)) < p
        mask = (~shell).astype(np.uint8)
        out = oracle_mod.fill_enclosed(mask, (nx, ny, nz)).reshape(nz, ny, nx)
        for z in range(nz):
            filled = ndimage.binary_fill_holes(shell[z], structure=cross)
            assert np.array_equal(out[z].astype(bool), filled & ~shell[z]), (nx, ny, z)


def test_compare_identities_and_hand_case(oracle_mod):
    rng = np.random.default_rng(4)
    dims = (9, 7, 5)
    h = (rng.random(315) < 0.4).astype(np.uint8)
    o = (rng.random(315) < 0.3).astype(np.uint8)
    r = oracle_mod.hull_compare(h, o, dims)
    assert r["extra"] - r["missing"] == int(h.sum()) - int(o.sum())
    assert r["extra"] == r["extra_per_slice"].sum() and r["missing"] == r["missing_per_slice"].sum()
    assert oracle_mod.hull_compare(o, o, dims)["extra"] == 0
    hh = np.zeros(8, np.uint8)
    oo = np.zeros(8, np.uint8)
    hh[[0, 1, 5]] = 1
    oo[[1, 2, 6, 7]] = 1
    r = oracle_mod.hull_compare(hh, oo, (2, 2, 2))
    assert list(r["extra_per_slice"]) == [1, 1] and list(r["missing_per_slice"]) == [1, 2]


def test_filled_msc_of_a_clean_shell_is_the_object(oracle_mod):
    """N = 0 inside a disk and 120 outside: Eq. 3.6 excludes exactly the
    outside voxels 4-adjacent to the disk (a closed ring), and the enclosed
    part of H_2 is the disk itself."""
    nx = ny = 24
    nz = 2
    yy, xx = np.mgrid[0:ny, 0:nx]
    disk = ((xx - 11.3) ** 2 + (yy - 12.6) ** 2 <= 49.0)
    N = np.where(disk, 0, 120).astype(np.uint32)
    N = np.ascontiguousarray(np.broadcast_to(N, (nz, ny, nx))).ravel()
    for nbhd in (4, 6):
        h2 = oracle_mod.msc_decide(N, (nx, ny, nz), nt=50, nbhd=nbhd)
        f = oracle_mod.fill_enclosed(h2, (nx, ny, nz)).reshape(nz, ny, nx)
        for z in range(nz):
            assert np.array_equal(f[z].astype(bool), disk)


def test_filled_msc_is_within_h2(oracle_mod):
    """On the tiny workload the enclosed part is a subset of H_2 (here the
    literal shell is open in the middle slices, where exterior voxels next
    to the object see few missed protons, so those slices fill to nothing:
    a diagnostic, not a better hull)."""
    w = synth.make_config(1, noise_free=True)
    g = w.geometry
    dims = (g.nx, g.ny, g.nz)
    r = oracle_mod.run(g, w.histories, threads=8)
    f = oracle_mod.fill_enclosed(r["H2"], dims)
    assert np.all(f <= r["H2"]) and 0 < f.sum() < r["H2"].sum()
