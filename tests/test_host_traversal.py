"""The CUDA library's geometry and traversal code (hd_geom.cuh), compiled for
the host, against the CPU oracle: exact voxel sets for adversarial segments,
the same sets when the walk is clipped to shared-memory tiles, and identical
fixed-point endpoints, and the Euclidean thick rays' row search against a
voxel-by-voxel exact search.  Runs without a GPU (nvcc compiles host code)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth
from tests.test_oracle_pins import _random_segments

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host_harness", "host_walk.cu")
I32P = ctypes.POINTER(ctypes.c_int32)


@pytest.fixture(scope="module")
def hx(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hx") / "libhostwalk.so")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-gencode", "arch=compute_103a,code=sm_103a",
                           "-diag-suppress", "20014", "-o", out, SRC,
                           "-I", os.path.join(HERE, "..", "include")])
    L = ctypes.CDLL(out)
    L.hx_walk.restype = ctypes.c_int
    L.hx_walk_tiled.restype = ctypes.c_int
    L.hx_endpoints.restype = ctypes.c_int
    L.hx_runs.restype = ctypes.c_int
    return L


def _walk(L, a, b, dims):
    a = np.asarray(a, np.int32)
    b = np.asarray(b, np.int32)
    out = np.zeros(sum(dims) + 16, np.int32)
    n = L.hx_walk(a.ctypes.data_as(I32P), b.ctypes.data_as(I32P), *dims,
                  out.ctypes.data_as(I32P), out.size)
    assert n <= out.size
    v = out[:n]
    assert len(np.unique(v)) == n  # each voxel once (C(v) is a set)
    return np.sort(v)


@pytest.mark.parametrize("dims", [(5, 4, 3), (1, 1, 1), (7, 1, 2), (3, 3, 3), (40, 30, 20)])
def test_walk_equals_oracle(oracle_mod, hx, dims):
    rng = np.random.default_rng(sum(dims) + 7)
    for a, b in _random_segments(rng, 4000, dims):
        assert np.array_equal(_walk(hx, a, b, dims), oracle_mod.voxel_set(a, b, *dims)), \
            (a.tolist(), b.tolist())


@pytest.mark.parametrize("dims,tiles", [((6, 5, 4), (6, 5, 1)), ((17, 13, 11), (17, 4, 1)),
                                        ((9, 9, 9), (2, 2, 2)), ((40, 30, 6), (40, 30, 2))])
def test_tiled_walks_partition_the_set(oracle_mod, hx, dims, tiles):
    rng = np.random.default_rng(sum(dims) + sum(tiles))
    for a, b in _random_segments(rng, 2000, dims):
        out = np.zeros(4 * sum(dims) + 64, np.int32)
        n = hx.hx_walk_tiled(np.asarray(a, np.int32).ctypes.data_as(I32P),
                             np.asarray(b, np.int32).ctypes.data_as(I32P), *dims, *tiles,
                             out.ctypes.data_as(I32P), out.size)
        assert n >= 0
        assert np.array_equal(np.sort(out[:n]), oracle_mod.voxel_set(a, b, *dims))


def test_endpoints_equal_oracle(oracle_mod, hx):
    theta, K = oracle_mod.cordic_table()
    th = (ctypes.c_longlong * 32)(*theta)
    rng = np.random.default_rng(3)
    for g in [synth.geometry_for(1), synth.geometry_for(2), synth.geometry_for(3),
              synth.Geometry(8, 8, 8, 0.125, 0.125, 0.125, 100.0)]:
        h = synth.tiny_random_case(rng, 4000, g, span=3.0)
        for i in range(len(h)):
            args = [float(x[i]) for x in h.arrays()[:5]]
            if i % 97 == 0:
                args[1] = float("nan")
            if i % 89 == 0:
                args[2] = 4096.0
            rej, gin, gout = oracle_mod.grid_endpoints(g, *args)
            out = np.zeros(6, np.int32)
            ok = hx.hx_endpoints(g.nx, g.ny, g.nz, ctypes.c_float(g.sx), ctypes.c_float(g.sy),
                                 ctypes.c_float(g.sz), ctypes.c_float(g.T), th, K,
                                 *[ctypes.c_float(x) for x in args], out.ctypes.data_as(I32P))
            assert bool(ok) != rej
            if ok:
                assert out[:3].tolist() == gin.tolist() and out[3:].tolist() == gout.tolist()


@pytest.mark.parametrize("dims", [(5, 4, 3), (1, 1, 1), (7, 1, 2), (40, 30, 20), (1, 7, 3),
                                  (9, 1, 1)])
def test_run_walk_equals_oracle(oracle_mod, hx, dims):
    """The run-length form (major-axis runs between minor crossings) gives the
    same voxel set, each voxel once."""
    rng = np.random.default_rng(sum(dims) + 11)
    for a, b in _random_segments(rng, 4000, dims):
        out = np.zeros(2 * sum(dims) + 64, np.int32)
        nr = ctypes.c_int(0)
        n = hx.hx_runs(np.asarray(a, np.int32).ctypes.data_as(I32P),
                       np.asarray(b, np.int32).ctypes.data_as(I32P), *dims,
                       out.ctypes.data_as(I32P), out.size, ctypes.byref(nr))
        assert n >= 0
        got = np.sort(out[:n])
        assert len(np.unique(got)) == n
        assert np.array_equal(got, oracle_mod.voxel_set(a, b, *dims)), (a.tolist(), b.tolist())


def test_run_walk_nearly_axis_aligned(oracle_mod, hx):
    """Minor axes that move by a few 2^-16 voxel units: quotients far beyond
    the box (the sentinel in the run walk) and minors starting on planes."""
    Q = 65536
    rng = np.random.default_rng(5)
    for dims in [(40, 30, 20), (64, 64, 8), (7, 200, 3)]:
        hi = np.array(dims) * Q
        for k in range(3000):
            a = rng.integers(-2 * Q, hi + 2 * Q)
            b = a.copy()
            maj = rng.integers(0, 3)
            b[maj] = rng.integers(-2 * Q, hi[maj] + 2 * Q)
            for ax in range(3):
                if ax != maj:
                    b[ax] = a[ax] + rng.integers(-3, 4) * (rng.integers(1, 3) if k % 2 else 1)
            if k % 5 == 0:
                for ax in range(3):
                    if ax != maj:
                        a[ax] = (a[ax] >> 16) << 16
            out = np.zeros(2 * sum(dims) + 64, np.int32)
            nr = ctypes.c_int(0)
            n = hx.hx_runs(np.asarray(a, np.int32).ctypes.data_as(I32P),
                           np.asarray(b, np.int32).ctypes.data_as(I32P), *dims,
                           out.ctypes.data_as(I32P), out.size, ctypes.byref(nr))
            assert n >= 0
            assert np.array_equal(np.sort(out[:n]), oracle_mod.voxel_set(a, b, *dims))


@pytest.mark.parametrize("dims", [(5, 4, 3), (40, 30, 20), (1, 7, 3), (200, 200, 1)])
def test_packed_run_walk_equals_oracle(oracle_mod, hx, dims):
    """A walk prepared in one kernel and resumed in another (packed state)."""
    hx.hx_runs_packed.restype = ctypes.c_int
    rng = np.random.default_rng(sum(dims) + 13)
    for a, b in _random_segments(rng, 3000, dims):
        out = np.zeros(2 * sum(dims) + 64, np.int32)
        n = hx.hx_runs_packed(np.asarray(a, np.int32).ctypes.data_as(I32P),
                              np.asarray(b, np.int32).ctypes.data_as(I32P), *dims,
                              out.ctypes.data_as(I32P), out.size)
        assert n >= 0
        assert np.array_equal(np.sort(out[:n]), oracle_mod.voxel_set(a, b, *dims))


def test_tile_index_division_exhaustive(hx):
    """Tile indices by multiply-high equal integer division for every voxel
    index and tile size the library supports (including tiles of one voxel)."""
    hx.hx_check_tile_division.restype = ctypes.c_longlong
    assert hx.hx_check_tile_division() == 0


def _runs_lean(L, a, b, dims):
    L.hx_runs_lean.restype = ctypes.c_int
    out = np.zeros(2 * sum(dims) + 64, np.int32)
    lean = ctypes.c_int(0)
    steps = ctypes.c_uint(0)
    n = L.hx_runs_lean(np.asarray(a, np.int32).ctypes.data_as(I32P),
                       np.asarray(b, np.int32).ctypes.data_as(I32P), *dims,
                       out.ctypes.data_as(I32P), out.size, ctypes.byref(lean), ctypes.byref(steps))
    assert n >= 0
    return np.sort(out[:n]), bool(lean.value), steps.value


@pytest.mark.parametrize("dims", [(200, 200, 1), (40, 30, 1), (7, 1, 1), (1, 7, 1), (5, 4, 3),
                                  (40, 30, 20), (64, 3, 2)])
def test_lean_run_walk_equals_oracle(oracle_mod, hx, dims):
    """Walks in their lean form (closed-form runs) give the oracle's voxel set
    and report its size; adversarial segments (lattice points, shared
    planes) keep the general form and still agree."""
    rng = np.random.default_rng(sum(dims) + 17)
    n_lean = 0
    for a, b in _random_segments(rng, 4000, dims):
        got, lean, steps = _runs_lean(hx, a, b, dims)
        assert len(np.unique(got)) == len(got)
        assert np.array_equal(got, oracle_mod.voxel_set(a, b, *dims)), (a.tolist(), b.tolist())
        if lean:
            n_lean += 1
            assert steps == len(got)
    assert n_lean > 0


@pytest.mark.parametrize("dims", [(200, 200, 1), (64, 64, 1), (9, 200, 1), (40, 30, 6)])
def test_lean_run_walk_generic_inputs(oracle_mod, hx, dims):
    """Segments with arbitrary Q16 endpoints (as from float detector
    coordinates) and a small z slope: almost every walk is lean."""
    rng = np.random.default_rng(sum(dims) + 19)
    Q = 65536
    hi = np.array(dims, np.int64) * Q
    n_lean = n_walks = 0
    for k in range(3000):
        a = rng.integers(-Q, hi + Q)
        b = rng.integers(-Q, hi + Q)
        a[2] = rng.integers(0, hi[2])
        b[2] = a[2] + rng.integers(-Q // 2, Q // 2 + 1)
        if k % 7 == 0:
            b[2] = a[2]  # z does not move
        got, lean, steps = _runs_lean(hx, a, b, dims)
        assert np.array_equal(got, oracle_mod.voxel_set(a, b, *dims)), (a.tolist(), b.tolist())
        n_walks += len(got) > 0
        if lean:
            n_lean += 1
            assert steps == len(got)
    if dims[2] == 1:
        assert n_lean > 0.99 * n_walks


def test_lean_run_walk_nearly_axis_aligned(oracle_mod, hx):
    """Lean walks whose minor axes move by a few 2^-16 voxel units (saturated
    quotients, capped steps) or start on a plane."""
    Q = 65536
    rng = np.random.default_rng(23)
    n_lean = 0
    for dims in [(200, 200, 1), (64, 7, 1), (40, 30, 3)]:
        hi = np.array(dims) * Q
        for k in range(3000):
            a = rng.integers(-2 * Q, hi + 2 * Q)
            b = a.copy()
            maj = rng.integers(0, 2)
            b[maj] = rng.integers(-2 * Q, hi[maj] + 2 * Q)
            for ax in range(3):
                if ax != maj:
                    b[ax] = a[ax] + rng.integers(-3, 4) * (rng.integers(1, 3) if k % 2 else 1)
            if k % 5 == 0:
                a[1 - maj] = (a[1 - maj] >> 16) << 16
            got, lean, steps = _runs_lean(hx, a, b, dims)
            assert np.array_equal(got, oracle_mod.voxel_set(a, b, *dims)), (a.tolist(), b.tolist())
            if lean:
                n_lean += 1
                assert steps == len(got)
    assert n_lean > 1000


def _tile_cursor(L, a, b, dims):
    L.hx_tile_cursor.restype = ctypes.c_int
    out = np.zeros(int(np.prod(dims)) + 8, np.int32)
    nr = ctypes.c_int(0)
    n = L.hx_tile_cursor(np.asarray(a, np.int32).ctypes.data_as(I32P),
                         np.asarray(b, np.int32).ctypes.data_as(I32P), *dims,
                         out.ctypes.data_as(I32P), out.size, ctypes.byref(nr))
    return n, np.sort(out[:max(n, 0)]), nr.value


@pytest.mark.parametrize("dims", [(200, 200, 1), (41, 30, 1), (7, 1, 1), (1, 7, 1), (40, 30, 3),
                                  (64, 3, 2)])
def test_tile_cursor_equals_oracle(oracle_mod, hx, dims):
    """The traversal's byte-offset form of a lean walk: its +1/-1 updates in
    the padded one-word-per-voxel tile (x runs in the low halves, y runs in
    the high halves) stay inside the box's words, and the prefix sums along
    x and y give every voxel of the oracle's set exactly once and no other
    voxel; its run count is what the kernel reports."""
    rng = np.random.default_rng(sum(dims) + 29)
    Q = 65536
    hi = np.array(dims, np.int64) * Q
    n_lean = 0
    for k in range(1500):
        a = rng.integers(-Q, hi + Q)
        b = rng.integers(-Q, hi + Q)
        if k % 2:
            a[2] = rng.integers(0, hi[2])
            b[2] = a[2] + rng.integers(-Q // 2, Q // 2 + 1)
        n, got, runs = _tile_cursor(hx, a, b, dims)
        assert n >= -1, (n, a.tolist(), b.tolist())
        if n == -1:
            continue
        n_lean += 1
        assert np.array_equal(got, oracle_mod.voxel_set(a, b, *dims)), (a.tolist(), b.tolist())
        if n > 0:
            assert 1 <= runs <= n
    assert n_lean > 300


def _slab_segments(rng, count, dims):
    """Segments for one-slice boxes: generic ones, ones with lattice-aligned
    end points (shared planes, corners, entry through edges), nearly
    axis-parallel ones and ones starting on faces of the box."""
    Q = 65536
    nx, ny = dims
    hi = np.array([nx, ny, 1], np.int64) * Q
    for k in range(count):
        kind = k % 5
        a = rng.integers(-2 * Q, hi + 2 * Q)
        b = rng.integers(-2 * Q, hi + 2 * Q)
        if kind == 0:
            a[2] = rng.integers(-Q, 2 * Q)
            b[2] = a[2] + rng.integers(-Q, Q + 1)
        elif kind == 1:  # lattice points and planes
            a = (rng.integers(-2, np.array([nx, ny, 1]) + 3) * Q).astype(np.int64)
            b = (rng.integers(-2, np.array([nx, ny, 1]) + 3) * Q).astype(np.int64)
            if k % 2:
                b[rng.integers(0, 3)] += rng.integers(-3, 4)
        elif kind == 2:  # nearly axis-parallel in the plane
            ax = rng.integers(0, 2)
            b[1 - ax] = a[1 - ax] + rng.integers(-2, 3)
            b[2] = a[2] + rng.integers(-2, 3)
        elif kind == 3:  # start or end exactly on a face of the slab or grid
            a[rng.integers(0, 3)] = rng.choice([0, hi[0], hi[1], Q])
            b[2] = rng.choice([0, Q, a[2]])
        else:  # through the slab from above or below, steep in z
            a[2] = rng.integers(-3 * Q, 0) if k % 2 else rng.integers(Q, 4 * Q)
            b[2] = rng.integers(Q, 4 * Q) if k % 2 else rng.integers(-3 * Q, 0)
        yield a, b


@pytest.mark.parametrize("dims", [(200, 200), (41, 30), (7, 1), (1, 7), (400, 126), (3, 3)])
def test_slab_lean_equals_general_setup(hx, dims):
    """The direct set-up for one-slice boxes gives, bit for bit, the packed
    lean walk of the general set-up (walk_begin, run_begin, lean_of), finds
    the same empty walks, and never claims a lean form the general set-up
    lacks; it declines (to the general set-up) only rarely on generic
    segments."""
    hx.hx_slab_lean.restype = ctypes.c_int
    rng = np.random.default_rng(sum(dims) + 31)
    counts = {}
    for a, b in _slab_segments(rng, 20000, dims):
        r = hx.hx_slab_lean(np.asarray(a, np.int32).ctypes.data_as(I32P),
                            np.asarray(b, np.int32).ctypes.data_as(I32P), *dims)
        assert r > 0, (r, a.tolist(), b.tolist())
        counts[r] = counts.get(r, 0) + 1
    assert counts.get(1, 0) > 2000
    # generic segments (kind 0): the direct set-up covers nearly every lean one
    gen = {}
    rng = np.random.default_rng(sum(dims) + 37)
    for k, (a, b) in enumerate(_slab_segments(rng, 5000, dims)):
        if k % 5:
            continue
        r = hx.hx_slab_lean(np.asarray(a, np.int32).ctypes.data_as(I32P),
                            np.asarray(b, np.int32).ctypes.data_as(I32P), *dims)
        gen[r] = gen.get(r, 0) + 1
    assert gen.get(3, 0) <= 0.02 * (gen.get(1, 0) + gen.get(3, 0)) + 2, gen


@pytest.mark.parametrize("dims,tiles", [((200, 200, 32), (200, 200, 1)), ((40, 30, 20), (40, 30, 3)),
                                        ((64, 48, 9), (64, 13, 1)), ((9, 9, 40), (9, 9, 7))])
def test_tile_range_covers_the_voxel_set(oracle_mod, hx, dims, tiles):
    """The tiles a record is bucketed into (x-y bounding box, slices of the
    part inside the grid's x-y extent) hold every voxel of its set, and a
    record gets no tile only when its set is empty."""
    hx.hx_tile_range.restype = ctypes.c_int
    rng = np.random.default_rng(sum(dims) + 43)
    Q = 65536
    hi = np.array(dims, np.int64) * Q
    tight = 0
    for k in range(3000):
        a = rng.integers(-hi // 2, hi + hi // 2)
        b = rng.integers(-hi // 2, hi + hi // 2)
        if k % 3 == 0:  # lattice-aligned end points
            a = (a >> 16) << 16
            b = (b >> 16) << 16
        r = np.concatenate([a, b]).astype(np.int32)
        lo = np.zeros(3, np.int32)
        up = np.zeros(3, np.int32)
        c = hx.hx_tile_range(r.ctypes.data_as(I32P), *dims, *tiles, lo.ctypes.data_as(I32P),
                             up.ctypes.data_as(I32P))
        vs = oracle_mod.voxel_set(a, b, *dims)
        if c == 0:
            assert vs.size == 0, (a.tolist(), b.tolist())
            continue
        assert c == int(np.prod(up - lo + 1))
        x = vs % dims[0]
        y = (vs // dims[0]) % dims[1]
        z = vs // (dims[0] * dims[1])
        for v, t, l, u in ((x, tiles[0], lo[0], up[0]), (y, tiles[1], lo[1], up[1]),
                           (z, tiles[2], lo[2], up[2])):
            assert np.all(v // t >= l) and np.all(v // t <= u), (a.tolist(), b.tolist())
        zb = np.clip(np.array([a[2], b[2]]) >> 16, 0, dims[2] - 1) // tiles[2]
        tight += (up[2] - lo[2]) < (zb.max() - zb.min())
    assert tight > 0  # the x-y clip removes slices the bounding box would add


def test_chunk_split_covers_every_history_once(hx):
    """The split that ingest and scatter share: blocks of per_block
    consecutive histories (a multiple of 4), at most 8 per SM, covering
    [0, n) with no empty block."""
    hx.hx_chunk_split.restype = None
    blocks, per = ctypes.c_int(), ctypes.c_longlong()
    rng = np.random.default_rng(5)
    ns = [1, 2, 3, 4, 5, 255, 256, 257, 1023, 1024, 4096, 4097, 180000, 550000, 9000000,
          1 << 25] + [int(x) for x in rng.integers(1, 1 << 25, 200)]
    for sm in (1, 7, 152):
        for n in ns:
            hx.hx_chunk_split(ctypes.c_longlong(n), sm, ctypes.byref(blocks), ctypes.byref(per))
            b, p = blocks.value, per.value
            assert p % 4 == 0 and p > 0, (n, sm, p)
            assert 1 <= b <= 8 * sm, (n, sm, b)
            assert b * p >= n and (b - 1) * p < n, (n, sm, b, p)


def test_loop_free_floor_division(hx):
    """fdiv_small, the set-up's loop-free floor division, equals floor
    division wherever the quotient stays below 2^20: random operands at
    every scale, exact multiples and their neighbours, negative numerators."""
    hx.hx_fdiv_small.restype = ctypes.c_longlong
    hx.hx_fdiv_small.argtypes = [ctypes.c_longlong, ctypes.c_longlong]
    rng = np.random.default_rng(8)
    for _ in range(20000):
        b = int(rng.integers(1, 1 << int(rng.integers(1, 47))))
        q = int(rng.integers(-(1 << 20) + 1, 1 << 20))
        r = int(rng.integers(-2, 3))
        a = q * b + r
        if abs(a) >= 1 << 62:
            continue
        assert hx.hx_fdiv_small(a, b) == a // b, (a, b)


def _euclid_rows(L, oracle_mod, g, h, d0):
    theta, K = oracle_mod.cordic_table()
    th = (ctypes.c_longlong * 32)(*theta)
    FP = ctypes.POINTER(ctypes.c_float)
    arrs = [np.ascontiguousarray(a, np.float32)
            for a in (h.angle_deg, h.u_in, h.v_in, h.u_out, h.v_out)]
    st = (ctypes.c_longlong * 7)()
    r = L.hx_euclid_rows(g.nx, g.ny, g.nz, ctypes.c_float(g.sx), ctypes.c_float(g.sy),
                         ctypes.c_float(g.sz), ctypes.c_float(g.T), th, ctypes.c_longlong(K),
                         ctypes.c_float(d0), *[a.ctypes.data_as(FP) for a in arrs], len(h), st)
    assert r == 0
    return dict(zip(["rows", "voxels", "mismatch", "filter_errors", "exact", "tested",
                     "histories"], list(st)))


@pytest.mark.parametrize("dims,sizes,T,radii", [
    ((23, 17, 9), (1.0, 1.0, 2.5), 40.0, (0.3, 1.7, 4.0)),
    ((16, 40, 12), (0.5, 1.25, 0.75), 40.0, (0.3, 1.7, 4.0)),
    ((50, 6, 3), (2.0, 0.8, 3.0), 40.0, (0.3, 1.7, 4.0)),
    ((7, 1, 1), (1.0, 1.0, 1.0), 40.0, (0.3, 1.7, 4.0)),
    # the extremes of the geometry the library takes: 1/64 mm voxels (the
    # filter's band widest against a voxel), 64 mm voxels and radii with a
    # 4 m tracker distance (its coordinates largest)
    ((40, 30, 8), (1 / 64, 1 / 64, 1 / 64), 12.0, (0.0005, 0.01, 0.3)),
    ((12, 10, 6), (64.0, 64.0, 64.0), 4000.0, (10.0, 63.9, 64.0))])
def test_euclid_row_search_equals_voxel_search(oracle_mod, hx, dims, sizes, T, radii):
    """The Euclidean thick rays' row search (float filter, empty-row
    certificate, filtered row-meets test, band of candidate rows, exact
    tests in the band) gives, row by row, the interval a voxel-by-voxel
    exact search finds, and no filter certificate contradicts the exact test
    (Eq. 3.2 with d_0 > 0)."""
    g = synth.Geometry(*dims, *sizes, T)
    rng = np.random.default_rng(sum(dims) + 5)
    h = synth.tiny_random_case(rng, 600, g, span=1.3)
    h.u_out[:60] = h.u_in[:60] + rng.normal(0, 1e-3, 60).astype(np.float32)
    h.v_out[60:120] = h.v_in[60:120]
    for d0 in radii:
        st = _euclid_rows(hx, oracle_mod, g, h, d0)
        assert st["mismatch"] == 0 and st["filter_errors"] == 0, (d0, st)
        assert st["histories"] > 0 and st["rows"] > 0
        # the band is narrow: nearly every test settled in float
        assert st["exact"] < 1e-3 * st["tested"], st


def test_euclid_row_search_centres_on_the_boundary(oracle_mod, hx):
    """Paths along rows of voxel centres, radii at and next to multiples of
    the spacing: centres lie on the capsule's surface up to the fixed-point
    rounding, inside the filter's band, and the exact test decides."""
    g = synth.Geometry(32, 32, 8, 1.0, 1.0, 2.5, 40.0)
    n = 64
    ang = np.repeat(np.array([0.0, 90.0], np.float32), n // 2)
    u = (np.arange(n) % 16 - 8 + 0.5).astype(np.float32)
    v = ((np.arange(n) % 8) * 2.5 - 10.0 + 1.25).astype(np.float32)
    h = synth.Histories(ang, u, v, u.copy(), v.copy(), np.full(n, 0.5, np.float32))
    exact = 0
    for d0 in (0.0, 2.0**-15, 0.5, 1.0, 1.0 - 2**-16, 2.5, 2.5 + 2**-16):
        st = _euclid_rows(hx, oracle_mod, g, h, d0)
        assert st["mismatch"] == 0 and st["filter_errors"] == 0, (d0, st)
        exact += st["exact"]
    assert exact > 0


@pytest.mark.parametrize("dims", [(5, 4, 3), (1, 1, 1), (7, 1, 2), (40, 30, 20), (1, 7, 3),
                                  (9, 1, 1), (3, 3, 3)])
def test_runs_in_path_order(hx, dims):
    """The run walk, each run expanded from its start in the direction the
    major axis moves, visits the voxels in the voxel walk's order (the rows
    of the system matrix list them in that order)."""
    rng = np.random.default_rng(sum(dims) + 99)
    for a, b in _random_segments(rng, 2000, dims):
        a = np.asarray(a, np.int32)
        b = np.asarray(b, np.int32)
        o1 = np.zeros(4 * sum(dims) + 64, np.int32)
        o2 = np.zeros_like(o1)
        n1 = hx.hx_walk(a.ctypes.data_as(I32P), b.ctypes.data_as(I32P), *dims,
                        o1.ctypes.data_as(I32P), o1.size)
        n2 = hx.hx_runs_path_order(a.ctypes.data_as(I32P), b.ctypes.data_as(I32P), *dims,
                                   o2.ctypes.data_as(I32P), o2.size)
        assert n1 == n2 and np.array_equal(o1[:n1], o2[:n2]), (a.tolist(), b.tolist())


@pytest.mark.parametrize("dims", [(5, 4, 3), (1, 1, 1), (7, 1, 2), (40, 30, 20), (1, 7, 3),
                                  (9, 1, 1), (3, 3, 3), (200, 200, 32)])
def test_slice_walks_in_path_order(hx, dims):
    """The path cut at its z planes, each slice's walk from the direct
    one-slice set-up (or the general one where it declines), slices taken in
    the direction the path moves along z: the voxel walk's voxels in the
    voxel walk's order (the one-slice tiles of the traversal split every
    walk this way; this pins the split voxel for voxel and in order)."""
    rng = np.random.default_rng(sum(dims) + 99)
    for a, b in _random_segments(rng, 2000, dims):
        a = np.asarray(a, np.int32)
        b = np.asarray(b, np.int32)
        o1 = np.zeros(4 * sum(dims) + 64, np.int32)
        o2 = np.zeros_like(o1)
        n1 = hx.hx_walk(a.ctypes.data_as(I32P), b.ctypes.data_as(I32P), *dims,
                        o1.ctypes.data_as(I32P), o1.size)
        n2 = hx.hx_slices_path_order(a.ctypes.data_as(I32P), b.ctypes.data_as(I32P), *dims,
                                     o2.ctypes.data_as(I32P), o2.size)
        assert n1 == n2 and np.array_equal(o1[:n1], o2[:n2]), (a.tolist(), b.tolist())
