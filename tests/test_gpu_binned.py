"""Binned SC (SC as the paper ran it) on the GPU against the oracle: the bin
table, the carved image and the hull, element by element, with the counters;
over chunks in any order, on bin-edge ties, with unbinnable histories, with
no histories, on a slice too wide for shared memory, and at the head-sized
workload's full size."""
import ctypes

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


def _dev(h):
    return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in h.arrays()]


def _hist(*cols):
    return synth.Histories(*[np.ascontiguousarray(np.asarray(c, np.float32)) for c in cols])


def _compare(hd, g, bp, b, ref):
    assert np.array_equal(b.bins(), ref["bins"])
    assert np.array_equal(b.image(hd.HD_BINNED_CARVED), ref["carved"])
    assert np.array_equal(b.image(hd.HD_BINNED_HULL), ref["mask"])
    st = b.stats()
    rs = ref["stats"]
    assert st["histories_binned"] == rs["binned"]
    assert st["histories_cut"] == rs["cut"]
    assert st["bins"] == bp.n_bins
    assert st["bins_used"] == rs["bins_used"]
    assert st["bins_missed"] == rs["bins_missed"]
    assert st["lines"] == rs["lines"]
    assert st["lines_outside"] == rs["lines_outside"]


def _run(hd, g, bp, h):
    b = hd.Binned(g, bp)
    b.run(_dev(h))
    return b


def test_params_default_matches_oracle(hd, oracle_mod):
    for g in [synth.geometry_for(1), synth.geometry_for(2), synth.geometry_for(3),
              synth.Geometry(128, 128, 32, 1.0, 1.0, 2.5, 110.0)]:
        p = hd.hd_binned_params_default(g)
        bp = oracle_mod.binned_params_for(g)
        assert (p.angle_bin_deg, p.u_bin_mm, p.v_bin_mm) == (4.0, 1.0, 5.0)
        assert (p.u_lo_mm, p.v_lo_mm, p.n_u, p.n_v) == (bp.u_lo_mm, bp.v_lo_mm, bp.n_u,
                                                        bp.v_bins)
        assert (p.k_sigma, p.miss_wepl_mm, p.window, p.min_count) == (3, 1.0, 5, 11)


def test_config1_matches_oracle(hd, oracle_mod):
    w = synth.make_config(1)
    g = w.geometry
    bp = oracle_mod.binned_params_for(g)
    ref = oracle_mod.sc_binned(g, w.histories, bp)
    assert ref["stats"]["cut"] > 0 and ref["stats"]["bins_missed"] > 0
    b = _run(hd, g, bp, w.histories)
    _compare(hd, g, bp, b, ref)
    b.close()


def test_chunks_in_any_order(hd, oracle_mod):
    """Statistics over chunks in one order and cuts over them in another give
    the single-array result (integer sums do not depend on order)."""
    w = synth.make_config(1, fraction=0.5)
    g = w.geometry
    bp = oracle_mod.binned_params_for(g)
    ref = oracle_mod.sc_binned(g, w.histories, bp)
    n = len(w.histories)
    perm = np.random.default_rng(7).permutation(n)
    parts = [w.histories.take(np.sort(perm[k::3])) for k in range(3)]
    dev = [_dev(p) for p in parts]
    with hd.Binned(g, bp) as b:
        for d in dev:
            b.add(d)
        for d in reversed(dev):
            b.cut(d)
        b.finalize()
        _compare(hd, g, bp, b, ref)


def test_bin_edge_ties_and_unbinnable(hd, oracle_mod):
    """Mid-points exactly on displacement bin edges, angles exactly on angle
    bin edges, values exactly at 3 sigma, and histories that must be skipped
    (NaN, infinity, out of range)."""
    g = synth.Geometry(16, 16, 4, 1.0, 1.0, 2.5, 30.0)
    bp = oracle_mod.binned_params_for(g)
    rng = np.random.default_rng(8)
    n = 6000
    ang = rng.integers(-2, 92, n) * 4.0 + rng.choice([-2.0, 2.0, 0.0, 1.75], n)
    um = bp.u_lo_mm + rng.integers(0, bp.n_u + 1, n) * bp.u_bin_mm
    vm = bp.v_lo_mm + rng.integers(0, bp.v_bins + 1, n) * bp.v_bin_mm
    du = rng.choice([0.0, 0.5, -0.25, 2.0], n)
    dv = rng.choice([0.0, 1.0, -0.5], n)
    wepl = rng.choice([0.0, 0.5, 1.0, 10.0, 0.25], n)
    cols = [ang, um - du / 2, vm - dv / 2, um + du / 2, vm + dv / 2, wepl]
    bad = rng.random(n) < 0.05
    cols[0] = np.where(bad & (rng.random(n) < 0.3), np.nan, cols[0])
    cols[5] = np.where(bad & (rng.random(n) < 0.3), np.inf, cols[5])
    cols[1] = np.where(bad & (rng.random(n) < 0.3), 5000.0, cols[1])
    cols[3] = np.where(bad & (rng.random(n) < 0.3), 1100.0, cols[3])
    h = _hist(*cols)
    # the exact 3 sigma tie of the oracle's pins, in a bin of its own
    tie = _hist([100.0] * 10, [0.3] * 10, [0.3] * 10, [0.3] * 10, [0.3] * 10, [0.0] * 9 + [10.0])
    h = synth.Histories.concat([h, tie])
    ref = oracle_mod.sc_binned(g, h, bp)
    b = _run(hd, g, bp, h)
    _compare(hd, g, bp, b, ref)
    b.close()


def test_no_histories(hd, oracle_mod):
    g = synth.Geometry(16, 16, 4, 1.0, 1.0, 2.5, 30.0)
    bp = oracle_mod.binned_params_for(g)
    h = _hist([], [], [], [], [], [])
    ref = oracle_mod.sc_binned(g, h, bp)
    b = _run(hd, g, bp, h)
    _compare(hd, g, bp, b, ref)
    b.close()


def test_wide_slice_uses_global_bitmap(hd, oracle_mod):
    """A 1280 x 1280 slice (51200 bitmap words) is carved in global memory."""
    g = synth.Geometry(1280, 1280, 2, 0.25, 0.25, 2.5, 240.0)
    bp = oracle_mod.binned_params_for(g)
    rng = np.random.default_rng(9)
    n = 20000
    ang = rng.integers(0, 90, n) * 4.0
    u = rng.uniform(bp.u_lo_mm * 0.9, -bp.u_lo_mm * 0.9, n)
    v = rng.uniform(-2.4, 2.4, n)
    wepl = np.where(np.abs(u) > 60, rng.uniform(0, 1.2, n), rng.uniform(3, 50, n))
    h = _hist(ang, u, v, u, v, wepl)
    ref = oracle_mod.sc_binned(g, h, bp)
    assert ref["stats"]["lines"] > 0
    b = _run(hd, g, bp, h)
    _compare(hd, g, bp, b, ref)
    b.close()


def test_page_locked_host_inputs(hd, oracle_mod):
    w = synth.make_config(1, fraction=0.1)
    g = w.geometry
    bp = oracle_mod.binned_params_for(g)
    ref = oracle_mod.sc_binned(g, w.histories, bp)
    pinned = [torch.from_numpy(a).pin_memory() for a in w.histories.arrays()]
    with hd.Binned(g, bp) as b:
        b.run(pinned)
        torch.cuda.synchronize()
        _compare(hd, g, bp, b, ref)
        with pytest.raises(hd.HDError) as e:  # pageable host memory is refused
            b.run([np.ascontiguousarray(a) for a in w.histories.arrays()])
        assert e.value.status == hd.HD_ERR_ARG


def test_states_and_ranges(hd, oracle_mod):
    g = synth.Geometry(16, 16, 4, 1.0, 1.0, 2.5, 30.0)
    bp = oracle_mod.binned_params_for(g)
    h = _dev(_hist([0.0] * 4, [0.1] * 4, [0.1] * 4, [0.1] * 4, [0.1] * 4, [0.5] * 4))
    with hd.Binned(g, bp) as b:
        out = np.zeros(g.nx * g.ny * g.nz, np.uint8)
        with pytest.raises(hd.HDError) as e:
            hd.hd_binned_get_image(b.handle, hd.HD_BINNED_HULL, out)
        assert e.value.status == hd.HD_ERR_STATE
        with pytest.raises(hd.HDError) as e:
            b.finalize()
        assert e.value.status == hd.HD_ERR_STATE
        b.add(h)
        b.cut(h)
        with pytest.raises(hd.HDError) as e:
            b.add(h)
        assert e.value.status == hd.HD_ERR_STATE
        b.finalize()
        with pytest.raises(hd.HDError) as e:
            b.cut(h)
        assert e.value.status == hd.HD_ERR_STATE
        assert b.stats()["bins_missed"] == 1
        hd.hd_binned_reset(b.handle)
        b.add(h)
    for bad in (dict(angle_bin_deg=7.0), dict(window=4), dict(min_count=26),
                dict(k_sigma=0), dict(u_bin_mm=0.0), dict(n_u=0)):
        p = hd.hd_binned_params_default(g)
        for k, v in bad.items():
            setattr(p, k, v)
        with pytest.raises(hd.HDError) as e:
            hd.hd_binned_create(g, p)
        assert e.value.status == hd.HD_ERR_RANGE, bad


def test_config2_full_size(hd, oracle_mod):
    """The head-sized workload, all 9e6 histories, in the launch
    configuration the bench times."""
    w = synth.make_config(2)
    g = w.geometry
    bp = oracle_mod.binned_params_for(g)
    ref = oracle_mod.sc_binned(g, w.histories, bp)
    assert ref["stats"]["cut"] > 0
    b = _run(hd, g, bp, w.histories)
    _compare(hd, g, bp, b, ref)
    b.close()


def test_extreme_values_exact(hd, oracle_mod):
    """WEPL and slopes near the 1024 mm limit, thousands of histories per
    bin (sums of squares near 2^48), with rare extreme values that the cuts
    remove: the integer square root of the cut bounds must be exact."""
    g = synth.Geometry(16, 16, 4, 1.0, 1.0, 2.5, 30.0)
    bp = oracle_mod.binned_params_for(g)
    rng = np.random.default_rng(11)
    n = 40000
    ang = rng.integers(0, 3, n) * 4.0
    um = rng.choice([-3.5, 0.5, 4.5], n)
    vm = np.full(n, 1.0)
    du = rng.choice([-1023.9, 1023.9, 0.0, -1000.0, 511.7], n, p=[0.003, 0.003, 0.5, 0.25, 0.244])
    dv = rng.choice([1023.9, -1023.9, 3.0], n, p=[0.004, 0.002, 0.994])
    wepl = rng.choice([1023.99, -1023.99, 0.0, 700.5, -0.004], n, p=[0.003, 0.002, 0.3, 0.6, 0.095])
    h = _hist(ang, um - du / 2, vm - dv / 2, um + du / 2, vm + dv / 2, wepl)
    ref = oracle_mod.sc_binned(g, h, bp)
    assert ref["bins"][:, 0].max() > 1000 and ref["stats"]["cut"] > 0
    b = _run(hd, g, bp, h)
    _compare(hd, g, bp, b, ref)
    b.close()
