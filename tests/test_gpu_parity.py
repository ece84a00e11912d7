"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is integer work, so the bar is bit-exactness: counts N and M,
masks H1/H2/H3, SM thresholds and the statistics must equal the oracle's.
"""

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1402_1720_gb300 import hulld
    hulld.load()
    return hulld


def _params(hd, oracle_params):
    return hd._params(oracle_params)


def _run_gpu(hd, g, hist, params=None, chunks=1, device_inputs=True, order=None):
    arrs = hist.arrays()
    if order is not None:
        arrs = [a[order] for a in arrs]
    with hd.Scan(g, params) as s:
        bounds = np.linspace(0, len(hist), chunks + 1).astype(np.int64)
        for c in range(chunks):
            part = [np.ascontiguousarray(a[bounds[c]:bounds[c + 1]]) for a in arrs]
            if device_inputs:
                part = [torch.from_numpy(a).cuda() for a in part]
            s.add(part)
        s.finalize()
        torch.cuda.synchronize()
        m = s.params.methods
        out = {"stats": s.stats()}
        if m & (hd.HD_MSC):
            out["N"] = s.counts(hd.HD_MSC)
        if m & hd.HD_SM:
            out["M"] = s.counts(hd.HD_SM)
            out["Mt"], out["slope"], out["index"] = s.thresholds()
            out["H3"] = s.mask(hd.HD_SM)
        if m & hd.HD_SC:
            out["H1"] = s.mask(hd.HD_SC)
        if m & hd.HD_MSC:
            out["H2"] = s.mask(hd.HD_MSC)
    return out


def _assert_same(got, ref, keys):
    for k in keys:
        assert np.array_equal(got[k], ref[k]), f"{k}: {int((np.asarray(got[k]) != np.asarray(ref[k])).sum())} differ"


def _assert_stats(got, ref):
    g, r = got["stats"], ref["stats"]
    for k in ["n_in", "n_miss", "n_hit", "n_none", "n_reject", "steps_miss", "steps_hit"]:
        assert g[k] == r[k], (k, g[k], r[k])


ALL = ["N", "M", "H1", "H2", "H3", "Mt", "slope", "index"]


def test_config1_full_parity(hd, oracle_mod):
    w = synth.make_config(1)
    ref = oracle_mod.run(w.geometry, w.histories, threads=8)
    got = _run_gpu(hd, w.geometry, w.histories)
    _assert_same(got, ref, ALL)
    _assert_stats(got, ref)
    # generic float inputs: almost every walk has the closed-form lean runs
    st = got["stats"]
    assert st["pairs_general"] < 1e-3 * (st["n_miss"] + st["n_hit"])
    # SC: H1 from the carve (Alg. 1) equals {N = 0}
    assert np.array_equal(got["H1"], ref["H1_carved"])


def test_config1_host_inputs_and_chunks(hd, oracle_mod):
    w = synth.make_config(1, fraction=0.5)
    ref = oracle_mod.run(w.geometry, w.histories, threads=8)
    got = _run_gpu(hd, w.geometry, w.histories, chunks=7, device_inputs=False)
    _assert_same(got, ref, ALL)
    _assert_stats(got, ref)
    perm = np.random.default_rng(0).permutation(len(w.histories))
    got2 = _run_gpu(hd, w.geometry, w.histories, chunks=3, order=perm)
    _assert_same(got2, ref, ALL)


FUZZ_GEOMS = [
    synth.Geometry(1, 1, 1, 1.0, 1.0, 1.0, 5.0),
    synth.Geometry(7, 1, 2, 0.5, 3.0, 1.25, 12.0),
    synth.Geometry(5, 4, 3, 1.0, 1.0, 2.5, 9.0),
    synth.Geometry(33, 17, 9, 1.0, 0.75, 2.0, 40.0),
    synth.Geometry(64, 64, 8, 1.0, 1.0, 2.5, 100.0),
    synth.Geometry(13, 40, 21, 2.0, 0.5, 0.25, 35.0),
]


@pytest.mark.parametrize("gi", range(len(FUZZ_GEOMS)))
def test_fuzz_random_histories(hd, oracle_mod, gi):
    g = FUZZ_GEOMS[gi]
    for seed in range(4):
        rng = np.random.default_rng(1000 * gi + seed)
        h = synth.tiny_random_case(rng, 3000, g, span=1.2 + 0.3 * seed)
        ref = oracle_mod.run(g, h)
        got = _run_gpu(hd, g, h)
        _assert_same(got, ref, ALL)
        _assert_stats(got, ref)


# grids whose shared-memory tiles are z-slabs of one or more slices, or x-y
# strips of one slice, so records are split over several tiles
TILED_GEOMS = [
    synth.Geometry(200, 200, 6, 1.0, 1.0, 2.5, 155.0),    # slabs of one slice
    synth.Geometry(256, 256, 4, 1.0, 1.0, 2.5, 190.0),    # x-y strips, one slice
    synth.Geometry(64, 64, 40, 1.0, 1.0, 0.5, 100.0),     # slabs of 10 slices
    synth.Geometry(400, 130, 3, 0.5, 0.5, 1.25, 155.0),   # x-y strips
    # 20 x-y strips per slice: steep diagonal paths touch more than 32 tiles
    # of their box and take the global path's list
    synth.Geometry(1000, 1000, 4, 0.2, 0.2, 2.5, 155.0),
]


@pytest.mark.parametrize("gi", range(len(TILED_GEOMS)))
def test_multi_tile_grids(hd, oracle_mod, gi):
    g = TILED_GEOMS[gi]
    for seed in range(2):
        rng = np.random.default_rng(77 + 10 * gi + seed)
        h = synth.tiny_random_case(rng, 6000, g, span=1.1)
        # mostly shallow paths, as in a scan, plus the steep ones of the case
        h.v_out[: len(h) // 2] = h.v_in[: len(h) // 2] + rng.normal(0, 2.0, len(h) // 2).astype(np.float32)
        ref = oracle_mod.run(g, h, threads=8)
        got = _run_gpu(hd, g, h)
        _assert_same(got, ref, ALL)
        _assert_stats(got, ref)
    # SC alone counts N over the same tiles and keeps {N = 0}
    p = oracle_mod.Params(methods=oracle_mod.SC)
    ref = oracle_mod.run(g, h, p, threads=8)
    got = _run_gpu(hd, g, h, p)
    _assert_same(got, ref, ["H1"])


def _lattice_histories(rng, g, n):
    """Histories whose entry/exit points sit on voxel planes, edges and
    corners (angles on multiples of 45 degrees, u/v on voxel boundaries), to
    exercise every tie of the traversal."""
    angle = rng.choice(np.arange(-360, 720, 45), n).astype(np.float32)
    step = min(g.sx, g.sy, g.sz)
    ext = max(g.nx * g.sx, g.ny * g.sy, g.nz * g.sz)
    k = int(ext / step)
    u_in = (rng.integers(-k, k + 1, n) * step / 2).astype(np.float32)
    u_out = (u_in + rng.integers(-3, 4, n) * step).astype(np.float32)
    v_in = (rng.integers(-g.nz, g.nz + 1, n) * g.sz / 2).astype(np.float32)
    v_out = (v_in + rng.integers(-2, 3, n) * g.sz).astype(np.float32)
    wepl = rng.choice(np.array([0.0, 9.0], np.float32), n)
    return synth.Histories(angle, u_in, v_in, u_out, v_out, wepl)


@pytest.mark.parametrize("g", [synth.Geometry(8, 8, 4, 1.0, 1.0, 1.0, 8.0),
                               synth.Geometry(6, 10, 3, 0.5, 0.5, 2.0, 6.0),
                               synth.Geometry(16, 16, 2, 1.0, 1.0, 2.5, 16.0)])
def test_lattice_aligned_ties(hd, oracle_mod, g):
    rng = np.random.default_rng(g.nx * 100 + g.ny)
    h = _lattice_histories(rng, g, 4000)
    ref = oracle_mod.run(g, h)
    got = _run_gpu(hd, g, h)
    _assert_same(got, ref, ALL)
    _assert_stats(got, ref)
    # ties send walks to the general run walk (the fallback list)
    assert got["stats"]["pairs_general"] > 0


@pytest.mark.parametrize("variant", ["sc_only", "msc_only", "sm_only", "sm_gt", "sm_global",
                                     "nbhd4", "sc_sm", "cutoffs"])
def test_parameter_variants(hd, oracle_mod, variant):
    P = oracle_mod.Params
    params = {
        "sc_only": P(methods=oracle_mod.SC),
        "msc_only": P(methods=oracle_mod.MSC),
        "sm_only": P(methods=oracle_mod.SM),
        "sm_gt": P(sm_ge=0),
        "sm_global": P(sm_per_slice=0),
        "nbhd4": P(nbhd=4, sm_per_slice=0),
        "sc_sm": P(methods=oracle_mod.SC | oracle_mod.SM),
        "cutoffs": P(tau_l=2.0, tau_h=2.0, nt=7),
    }[variant]
    w = synth.make_config(1, fraction=0.25)
    ref = oracle_mod.run(w.geometry, w.histories, params, threads=8)
    got = _run_gpu(hd, w.geometry, w.histories, params)
    keys = []
    if params.methods & oracle_mod.SC:
        keys.append("H1")
    if params.methods & oracle_mod.MSC:
        keys += ["N", "H2"]
    if params.methods & oracle_mod.SM:
        keys += ["M", "H3", "Mt", "slope", "index"]
    _assert_same(got, ref, keys)
    # the oracle counts steps for both classes only when the class is traversed
    assert got["stats"]["n_miss"] == ref["stats"]["n_miss"]
    assert got["stats"]["n_hit"] == ref["stats"]["n_hit"]
    assert got["stats"]["n_reject"] == ref["stats"]["n_reject"]


def test_edge_cases(hd, oracle_mod):
    g = synth.Geometry(10, 9, 4, 1.0, 1.0, 2.0, 20.0)
    nan, inf = float("nan"), float("inf")
    rows = [
        # angle, u_in, v_in, u_out, v_out, wepl
        (0.0, 0.5, 0.5, 0.5, 0.5, 0.0),          # plain miss
        (90.0, 0.0, 0.0, 0.0, 0.0, 9.0),         # hit through the centre lines
        (nan, 0.0, 0.0, 0.0, 0.0, 0.0),          # rejected angle
        (10.0, inf, 0.0, 0.0, 0.0, 0.0),         # rejected u
        (10.0, 0.0, 4096.0, 0.0, 0.0, 9.0),      # rejected v
        (10.0, 0.0, 0.0, 0.0, -4095.0, 9.0),     # huge but valid, mostly outside
        (33.0, 200.0, 0.0, 200.0, 0.0, 0.0),     # entirely outside the grid
        (45.0, 0.0, 4.0, 0.0, 4.0, 0.0),         # on the top face z = +4 mm (outside)
        (45.0, 0.0, -4.0, 0.0, -4.0, 0.0),       # on the bottom face (inside)
        (0.0, 0.0, 0.0, 0.0, 0.0, nan),          # NaN WEPL: unused
        (0.0, 0.0, 0.0, 0.0, 0.0, 1.0),          # exactly the miss cutoff: unused
        (0.0, 0.0, 0.0, 0.0, 0.0, 5.0),          # exactly the hit cutoff: unused
        (720.0, 1.0, 1.0, -1.0, -1.0, -5.0),     # angle beyond one turn
        (-1e5, 3.0, 2.0, -3.0, -2.0, 1e30),      # large negative angle, huge WEPL
    ]
    h = synth.Histories(*[np.array(c, np.float32) for c in zip(*rows)])
    ref = oracle_mod.run(g, h)
    got = _run_gpu(hd, g, h)
    _assert_same(got, ref, ALL)
    _assert_stats(got, ref)
    assert got["stats"]["n_reject"] == 3
    # an empty add is a no-op; all-unused histories give empty counts
    with hd.Scan(g) as s:
        s.add([np.zeros(0, np.float32)] * 6)
        s.add([np.zeros(5, np.float32)] * 5 + [np.full(5, 3.0, np.float32)])
        s.finalize()
        st = s.stats()
        assert st["n_in"] == 5 and st["n_none"] == 5 and st["steps_miss"] == 0
        assert not s.counts(hd.HD_MSC).any() and not s.counts(hd.HD_SM).any()
        assert s.mask(hd.HD_SC).all() and s.mask(hd.HD_MSC).all()
        assert not s.mask(hd.HD_SM).any()   # no edge anywhere


def test_reset_and_refinalize(hd, oracle_mod):
    w = synth.make_config(1, fraction=0.1)
    ref = oracle_mod.run(w.geometry, w.histories)
    with hd.Scan(w.geometry) as s:
        junk = synth.tiny_random_case(np.random.default_rng(9), 500, w.geometry)
        s.add(junk.arrays())
        s.finalize()
        s.reset()
        half = len(w.histories) // 2
        s.add([a[:half].copy() for a in w.histories.arrays()])
        s.finalize()
        s.add([a[half:].copy() for a in w.histories.arrays()])
        s.finalize()
        assert np.array_equal(s.counts(hd.HD_MSC), ref["N"])
        assert np.array_equal(s.mask(hd.HD_SM), ref["H3"])
        assert np.array_equal(s.mask(hd.HD_MSC), ref["H2"])


def test_mask_layouts_and_hull_indices(hd, oracle_mod):
    w = synth.make_config(1, fraction=0.2)
    ref = oracle_mod.run(w.geometry, w.histories)
    V = w.geometry.n_voxels
    with hd.Scan(w.geometry) as s:
        s.add(w.histories.arrays())
        s.finalize()
        for meth, key in [(hd.HD_SC, "H1"), (hd.HD_MSC, "H2"), (hd.HD_SM, "H3")]:
            bits = s.mask(meth, hd.HD_MASK_BITS)
            unpacked = np.unpackbits(bits.view(np.uint8), bitorder="little")[:V]
            assert np.array_equal(unpacked, ref[key])
            # device destination, bits layout
            dbits = torch.zeros(bits.size, dtype=torch.int32, device="cuda")
            s.mask(meth, hd.HD_MASK_BITS, out=dbits)
            torch.cuda.synchronize()
            assert np.array_equal(dbits.cpu().numpy().view(np.uint32), bits)
            count, idx = s.hull_indices(meth)
            expect = np.flatnonzero(ref[key]).astype(np.int32)
            assert count == expect.size
            assert np.array_equal(idx[:count], expect)
            didx = torch.zeros(max(1, expect.size), dtype=torch.int32, device="cuda")
            c2, _ = s.hull_indices(meth, didx)
            torch.cuda.synchronize()
            assert c2 == expect.size
            assert np.array_equal(didx.cpu().numpy()[:c2], expect)


def test_classify_entry_point(hd, oracle_mod):
    w = np.array([0.999, 1.0, 3.0, 5.0, 5.0001, float("nan"), -float("inf"), float("inf"),
                  -2.0], dtype=np.float32)
    w = np.concatenate([w, np.random.default_rng(4).normal(3, 4, 100000).astype(np.float32)])
    ref = oracle_mod.classify(w)
    assert np.array_equal(hd.hd_classify(w), ref)
    dw = torch.from_numpy(w).cuda()
    got = hd.hd_classify(dw)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref)


def test_api_errors(hd):
    g = synth.geometry_for(1)
    bad_geoms = [synth.Geometry(0, 4, 4, 1, 1, 1, 10), synth.Geometry(4, 4, 5000, 1, 1, 1, 10),
                 synth.Geometry(4, 4, 4, 0.001, 1, 1, 10), synth.Geometry(4, 4, 4, 1, 1, 1, 0.0),
                 synth.Geometry(4, 4, 4, 1, 1, float("nan"), 10)]
    for bg in bad_geoms:
        with pytest.raises(hd.HDError) as e:
            hd.Scan(bg)
        assert e.value.status == hd.HD_ERR_RANGE
    p = hd.hd_params_default()
    p.wepl_miss_lt = 6.0
    with pytest.raises(hd.HDError) as e:
        hd.Scan(g, p)
    assert e.value.status == hd.HD_ERR_ARG
    p = hd.hd_params_default()
    p.methods = 0
    with pytest.raises(hd.HDError):
        hd.Scan(g, p)
    p = hd.hd_params_default()
    p.methods = hd.HD_SM
    with hd.Scan(g, p) as s:
        s.finalize()
        with pytest.raises(hd.HDError) as e:
            s.mask(hd.HD_MSC)
        assert e.value.status == hd.HD_ERR_STATE
        with pytest.raises(hd.HDError):
            s.counts(hd.HD_MSC)
        with pytest.raises(hd.HDError) as e:
            hd.hd_scan_get_mask(s.handle, hd.HD_SM, hd.HD_MASK_U8, np.zeros(10, np.uint8))
        assert e.value.status == hd.HD_ERR_ARG


@pytest.mark.parametrize("setting", [
    {"threads": 256, "refill": 4, "job_size": 4096, "slab_depth": 1},
    {"threads": 768, "refill": 24, "job_size": 32767, "slab_depth": 2},
    {"threads": 512, "refill": 1, "job_size": 256, "slab_depth": 0},
    {"threads": 1024, "refill": 8, "job_size": 16384, "slab_depth": 4},
])
def test_tuning_settings_do_not_change_results(hd, oracle_mod, setting):
    """Launch parameters change speed only: every setting gives the oracle's
    results, on a one-tile grid and on slabbed grids."""
    t = hd.hd_tuning(setting["threads"], setting["refill"], setting["job_size"],
                     setting["slab_depth"])
    w = synth.make_config(1, fraction=0.2)
    cases = [(w.geometry, w.histories)]
    g2 = synth.Geometry(64, 64, 40, 1.0, 1.0, 0.5, 100.0)
    cases.append((g2, synth.tiny_random_case(np.random.default_rng(8), 8000, g2, span=1.1)))
    for g, h in cases:
        ref = oracle_mod.run(g, h, threads=8)
        with hd.Scan(g) as s:
            hd.hd_scan_set_tuning(s.handle, t)
            assert hd.hd_scan_get_tuning(s.handle) == setting
            s.add([torch.from_numpy(a).cuda() for a in h.arrays()])
            s.finalize()
            torch.cuda.synchronize()
            assert np.array_equal(s.counts(hd.HD_MSC), ref["N"])
            assert np.array_equal(s.counts(hd.HD_SM), ref["M"])
            assert np.array_equal(s.mask(hd.HD_MSC), ref["H2"])
            assert np.array_equal(s.mask(hd.HD_SM), ref["H3"])
            # tuning is refused while the scan holds histories
            with pytest.raises(hd.HDError) as e:
                hd.hd_scan_set_tuning(s.handle, t)
            assert e.value.status == hd.HD_ERR_STATE


def test_autotuner_picks_a_valid_setting(hd, tmp_path):
    from paper_1402_1720_gb300 import autotune
    w = synth.make_config(1, fraction=0.3)
    dev = [torch.from_numpy(a).cuda() for a in w.histories.arrays()]
    space = {"slab_depth": [0, 2], "threads": [256, 512], "refill": [8, 16],
             "job_size": [8192, 16384]}
    res = autotune.autotune(w.geometry, dev, space=space, repeats=1)
    s = res["setting"]
    # the search starts from the defaults and tries the space's values
    for k, vals in space.items():
        assert s[k] in list(vals) + [autotune.DEFAULT[k]], k
    assert res["ms"] == min(ms for _, ms in res["trials"])
    path = str(tmp_path / "cache.json")
    got = autotune.tuned_setting(w.geometry, dev, path=path, repeats=1)
    assert autotune.tuned_setting(w.geometry, None, path=path) == got  # from the cache


def test_host_inputs_equal_device_inputs(hd):
    """Host inputs at scale: pageable numpy (copied to the staging buffer),
    page-locked tensors (read in place by the ingest kernel) and two calls in
    a row give the device-input counts exactly."""
    w = synth.make_config(2, fraction=0.5)
    g, h = w.geometry, w.histories
    arrs = h.arrays()
    with hd.Scan(g) as s:
        s.add([torch.from_numpy(a).cuda() for a in arrs])
        s.finalize()
        torch.cuda.synchronize()
        ref_n, ref_m = s.counts(hd.HD_MSC), s.counts(hd.HD_SM)
        ref_st = s.stats()
    pinned = [torch.from_numpy(a).pin_memory() for a in arrs]
    half = len(h) // 2
    for inputs in (arrs, pinned, "split"):
        with hd.Scan(g) as s:
            if inputs == "split":
                s.add([a[:half] for a in arrs])
                s.add([a[half:] for a in arrs])
            else:
                s.add(inputs)
            s.finalize()
            torch.cuda.synchronize()
            assert np.array_equal(s.counts(hd.HD_MSC), ref_n)
            assert np.array_equal(s.counts(hd.HD_SM), ref_m)
            st = s.stats()
            for k in ("n_in", "n_miss", "n_hit", "steps_miss", "steps_hit"):
                assert st[k] == ref_st[k], k


def test_atomic_probe_and_run_count(hd):
    """The atomic-throughput probe returns a rate for every kind, and the run
    count of a scan is consistent with its voxel count (each run covers at
    least one voxel, and a walk of L voxels has at most L runs)."""
    rates = [hd.hd_probe_atomics(k) for k in (hd.HD_PROBE_SMEM_RANDOM, hd.HD_PROBE_SMEM_COHERENT,
                                              hd.HD_PROBE_L2_RANDOM, hd.HD_PROBE_HBM_RANDOM)]
    assert all(r > 1e8 for r in rates)
    with pytest.raises(hd.HDError):
        hd.hd_probe_atomics(7)
    w = synth.make_config(1, fraction=0.2)
    got = _run_gpu(hd, w.geometry, w.histories)
    st = got["stats"]
    steps = st["steps_miss"] + st["steps_hit"]
    assert 0 < st["runs"] <= steps
