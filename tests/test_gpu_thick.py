"""Thick rays on the GPU against the oracle, bit for bit: N and M for k =
0, 1, 2 and 5 on the tiny workload, lattice ties on two small grids, a sample
of the head-sized workload, accumulation over calls, and the range check."""
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


def _gpu(hd, g, h, k, times=1):
    V = g.nx * g.ny * g.nz
    N = torch.zeros(V, dtype=torch.int32, device="cuda")
    M = torch.zeros(V, dtype=torch.int32, device="cuda")
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in h.arrays()]
    for _ in range(times):
        hd.hd_accumulate_thick(g, None, k, dev, N, M)
    torch.cuda.synchronize()
    return N.cpu().numpy().view(np.uint32), M.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("k", [0, 1, 2, 5])
def test_tiny_workload(hd, oracle_mod, k):
    w = synth.make_config(1, fraction=0.3)
    N, M = _gpu(hd, w.geometry, w.histories, k)
    ref = oracle_mod.accumulate_thick(w.geometry, w.histories, k)
    assert np.array_equal(N, ref["N"]) and np.array_equal(M, ref["M"])


@pytest.mark.parametrize("g", [synth.Geometry(8, 8, 4, 1.0, 1.0, 1.0, 8.0),
                               synth.Geometry(16, 16, 2, 1.0, 1.0, 2.5, 16.0)])
def test_lattice_ties(hd, oracle_mod, g):
    from tests.test_gpu_parity import _lattice_histories
    h = _lattice_histories(np.random.default_rng(g.nx + 5), g, 3000)
    for k in (1, 2):
        N, M = _gpu(hd, g, h, k)
        ref = oracle_mod.accumulate_thick(g, h, k)
        assert np.array_equal(N, ref["N"]) and np.array_equal(M, ref["M"])


def test_head_sample_and_accumulation(hd, oracle_mod):
    w = synth.make_config(2, fraction=0.03)
    N, M = _gpu(hd, w.geometry, w.histories, 2, times=2)
    ref = oracle_mod.accumulate_thick(w.geometry, w.histories, 2)
    assert np.array_equal(N, 2 * ref["N"]) and np.array_equal(M, 2 * ref["M"])


def test_k_range(hd):
    g = synth.Geometry(8, 8, 4, 1.0, 1.0, 1.0, 8.0)
    h = synth.make_config(1, fraction=0.01).histories
    with pytest.raises(hd.HDError) as e:
        _gpu(hd, g, h, 17)
    assert e.value.status == hd.HD_ERR_RANGE


def _scan_thick(hd, g, h, k, params=None):
    s = hd.Scan(g, params)
    s.set_thick(k)
    s.add([torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in h.arrays()])
    s.finalize()
    torch.cuda.synchronize()
    return s


@pytest.mark.parametrize("k", [1, 3])
def test_scan_with_thick_rays(hd, oracle_mod, k):
    """All three methods on thick sets: counts, hulls, thresholds and
    statistics equal the oracle's run on A_i(k)."""
    w = synth.make_config(1, fraction=0.5)
    g, h = w.geometry, w.histories
    s = _scan_thick(hd, g, h, k)
    ref = oracle_mod.run_thick(g, h, k)
    assert np.array_equal(s.counts(hd.HD_MSC), ref["N"])
    assert np.array_equal(s.counts(hd.HD_SM), ref["M"])
    for m, key in ((hd.HD_SC, "H1"), (hd.HD_MSC, "H2"), (hd.HD_SM, "H3")):
        assert np.array_equal(s.mask(m), ref[key]), key
    mt, slope, index = s.thresholds()
    assert np.array_equal(np.asarray(mt), ref["Mt"])
    st = s.stats()
    r = ref["stats"]
    assert (st["n_in"], st["n_miss"], st["n_hit"], st["n_none"], st["n_reject"]) == \
        tuple(int(x) for x in r[:5])
    assert (st["steps_miss"], st["steps_hit"]) == (int(r[5]), int(r[6]))
    s.close()


def test_scan_thick_sc_only_chunks_and_states(hd, oracle_mod):
    """SC alone counts N for its thick sets; chunks add up; k is fixed once
    histories have arrived; thick scans stay out of batches."""
    w = synth.make_config(1, fraction=0.3)
    g, h = w.geometry, w.histories
    params = oracle_mod.Params(methods=oracle_mod.SC)
    s = hd.Scan(g, params)
    s.set_thick(2)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in h.arrays()]
    n = len(h)
    s.add([a[: n // 3] for a in dev])
    with pytest.raises(hd.HDError) as e:
        s.set_thick(1)
    assert e.value.status == hd.HD_ERR_STATE
    s.add([a[n // 3:] for a in dev])
    s.finalize()
    torch.cuda.synchronize()
    ref = oracle_mod.run_thick(g, h, 2, params)
    assert np.array_equal(s.mask(hd.HD_SC), ref["H1"])
    b = hd.hd_batch_create(4)
    with pytest.raises(hd.HDError) as e:
        hd.hd_batch_add(b, s.handle, *dev)
    assert e.value.status == hd.HD_ERR_STATE
    hd.hd_batch_destroy(b)
    s.close()
    with pytest.raises(hd.HDError) as e:
        hd.Scan(g).set_thick(17)
    assert e.value.status == hd.HD_ERR_RANGE


@pytest.mark.parametrize("case", ["strips", "deep_slabs", "head_sample"])
def test_scan_thick_plans(hd, oracle_mod, case):
    """Whole-plane one-slice tiles take the tiled thick traversal; other
    plans (x-y strips, slabs two slices deep) the lane walk over the grid;
    both equal the oracle."""
    if case == "strips":
        g = synth.Geometry(256, 256, 4, 1.0, 1.0, 2.5, 200.0)
        h = synth.make_histories(np.random.default_rng(21), g, synth.head_phantom(0.9),
                                 np.arange(0, 360, 30), 400, 150.0, 5.0, 2.0, 0.01, 0.3)
    elif case == "deep_slabs":
        w = synth.make_config(1, fraction=0.2)
        g, h = w.geometry, w.histories
    else:
        w = synth.make_config(2, fraction=0.02)
        g, h = w.geometry, w.histories
    s = hd.Scan(g)
    if case == "deep_slabs":
        t = hd.hd_scan_get_tuning(s.handle)
        tun = hd.hd_tuning(t["threads"], t["refill"], t["job_size"], 2)
        hd.hd_scan_set_tuning(s.handle, tun)
    s.set_thick(2)
    s.add([torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in h.arrays()])
    s.finalize()
    torch.cuda.synchronize()
    ref = oracle_mod.run_thick(g, h, 2)
    assert np.array_equal(s.counts(hd.HD_MSC), ref["N"])
    assert np.array_equal(s.counts(hd.HD_SM), ref["M"])
    for m, key in ((hd.HD_SC, "H1"), (hd.HD_MSC, "H2"), (hd.HD_SM, "H3")):
        assert np.array_equal(s.mask(m), ref[key]), key
    st = s.stats()
    assert (st["steps_miss"], st["steps_hit"]) == (int(ref["stats"][5]), int(ref["stats"][6]))
    s.close()


def test_scan_thick_config2_full_size(hd, oracle_mod):
    """The head-sized workload, all 9e6 histories, k = 2, in the launch
    configuration the bench times: sampled voxels (random and on the object's
    boundary) counted by the oracle's slab test of the dilated box over every
    history; the decisions re-derived by the oracle from the GPU's counts; the
    count identities."""
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    dims = (g.nx, g.ny, g.nz)
    s = _scan_thick(hd, g, h, 2)
    N = s.counts(hd.HD_MSC)
    M = s.counts(hd.HD_SM)
    rng = np.random.default_rng(33)
    obj = synth.object_mask(g, w.phantom).reshape(g.nz, g.ny, g.nx)
    edge = np.flatnonzero((obj ^ np.roll(obj, 1, axis=2)).ravel())
    vox = np.concatenate([rng.choice(g.nx * g.ny * g.nz, 10, replace=False),
                          rng.choice(edge, 10, replace=False)])
    assert np.array_equal(N[vox], oracle_mod.count_thick_voxels(g, h, 2, 1, vox))
    assert np.array_equal(M[vox], oracle_mod.count_thick_voxels(g, h, 2, 2, vox))
    assert np.array_equal(s.mask(hd.HD_SC), (N == 0).astype(np.uint8))
    assert np.array_equal(s.mask(hd.HD_MSC), oracle_mod.msc_decide(N, dims))
    assert np.array_equal(s.mask(hd.HD_SM), oracle_mod.sm_decide(M, dims)["H3"])
    st = s.stats()
    assert st["steps_miss"] == int(N.sum()) and st["steps_hit"] == int(M.sum())
    assert st["n_in"] == len(h)
    s.close()
