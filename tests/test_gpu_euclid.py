"""Thick rays by the Euclidean distance of Eq. 3.2 on the GPU (through the C
ABI) against the oracle: the counts N and M of the standalone accumulation,
and scans set to a thick distance (counts, the three hulls, thresholds and
statistics), bit for bit; at d_0 of 0.5, 1 and 2.5 mm (the last reaching
across 2.5 mm slices), on random segments over anisotropic grids, on
segments along rows of voxel centres (boundary cases of the distance test),
and with d_0 = 0."""
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


def _gpu_counts(hd, g, h, d0, params=None):
    params = params or hd.hd_params_default()
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    N = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    M = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    rows = torch.zeros(1, dtype=torch.int64, device="cuda")
    hd.hd_accumulate_euclid(g, params, d0, dev, N, M, rows=rows)
    torch.cuda.synchronize()
    return N.cpu().numpy().view(np.uint32), M.cpu().numpy().view(np.uint32), int(rows.item())


@pytest.mark.parametrize("d0", [0.5, 1.0, 2.5])
def test_config1_sample_counts(hd, oracle_mod, d0):
    w = synth.make_config(1, fraction=0.2)
    g, h = w.geometry, w.histories
    ref = oracle_mod.accumulate_euclid(g, h, d0, threads=16)
    N, M, rows = _gpu_counts(hd, g, h, d0)
    assert np.array_equal(N, ref["N"]) and np.array_equal(M, ref["M"])
    assert 0 < rows <= int(ref["N"].sum() + ref["M"].sum())


@pytest.mark.parametrize("dims,sizes", [((23, 17, 9), (1.0, 1.0, 2.5)),
                                        ((16, 40, 12), (0.5, 1.25, 0.75)),
                                        ((50, 6, 3), (2.0, 0.8, 3.0))])
def test_random_segments_anisotropic(hd, oracle_mod, dims, sizes):
    """Segments in every direction (also nearly parallel to an axis, and
    some rejected), several radii."""
    g = synth.Geometry(*dims, *sizes, 40.0)
    rng = np.random.default_rng(sum(dims))
    h = synth.tiny_random_case(rng, 3000, g, span=1.3)
    # a few nearly axis-parallel paths and rejected histories
    h.u_out[:200] = h.u_in[:200] + rng.normal(0, 1e-3, 200).astype(np.float32)
    h.v_out[200:400] = h.v_in[200:400]
    h.u_in[400:410] = np.float32(5000.0)
    h.angle_deg[410:420] = np.float32(np.nan)
    for d0 in (0.3, 1.7, 4.0):
        ref = oracle_mod.accumulate_euclid(g, h, d0, threads=16)
        N, M, _ = _gpu_counts(hd, g, h, d0)
        assert np.array_equal(N, ref["N"]), d0
        assert np.array_equal(M, ref["M"]), d0


@pytest.mark.parametrize("dims,sizes,T,radii", [
    ((40, 30, 8), (1 / 64, 1 / 64, 1 / 64), 12.0, (0.0005, 0.01, 0.3)),
    ((12, 10, 6), (64.0, 64.0, 64.0), 4000.0, (10.0, 63.9, 64.0)),
    ((20, 7, 9), (2.0, 0.125, 0.0625), 100.0, (0.05, 0.3, 5.0))])
def test_extreme_geometries(hd, oracle_mod, dims, sizes, T, radii):
    """The geometry's extremes (1/64 mm and 64 mm voxels, a 4 m tracker
    distance, strongly anisotropic voxels), where the kernel's float filter
    works with its widest band against a voxel or its largest coordinates:
    counts equal the oracle's."""
    g = synth.Geometry(*dims, *sizes, T)
    rng = np.random.default_rng(sum(dims) + 17)
    h = synth.tiny_random_case(rng, 2000, g, span=1.3)
    h.u_out[:200] = h.u_in[:200] + rng.normal(0, 1e-4, 200).astype(np.float32)
    h.v_out[200:400] = h.v_in[200:400]
    for d0 in radii:
        ref = oracle_mod.accumulate_euclid(g, h, d0, threads=16)
        N, M, _ = _gpu_counts(hd, g, h, d0)
        assert ref["N"].sum() + ref["M"].sum() > 0, d0
        assert np.array_equal(N, ref["N"]), d0
        assert np.array_equal(M, ref["M"]), d0


def test_rows_of_centres_and_zero_radius(hd, oracle_mod):
    """Paths along rows of voxel centres at angle 0 (x) and 90 degrees (y)
    (the fixed-point rotation leaves them within a unit of 2^-16 mm of the
    centres): radii at and around one spacing decide membership at the
    boundary, 2^-15 mm keeps about the centres on the path, and d_0 = 0
    only what lies exactly on it."""
    g = synth.Geometry(32, 32, 8, 1.0, 1.0, 2.5, 40.0)
    n = 64
    ang = np.repeat(np.array([0.0, 90.0], np.float32), n // 2)
    # u = 0.5 + j puts the path through the centres of one row (grid centred)
    u = (np.arange(n) % 16 - 8 + 0.5).astype(np.float32)
    v = ((np.arange(n) % 8) * 2.5 - 10.0 + 1.25).astype(np.float32)
    h = synth.Histories(ang, u, v, u.copy(), v.copy(), np.full(n, 0.5, np.float32))
    for d0 in (0.0, 2.0**-15, 0.5, 1.0, 1.0 - 2**-16, 2.5, 2.5 + 2**-16):
        ref = oracle_mod.accumulate_euclid(g, h, d0)
        N, _, _ = _gpu_counts(hd, g, h, d0)
        assert np.array_equal(N, ref["N"]), d0
        if d0 == 2.0**-15:
            assert ref["N"].sum() > 0


@pytest.mark.parametrize("d0", [0.5, 2.5])
def test_scan_set_to_euclidean_distance(hd, oracle_mod, d0):
    """A scan counting Euclidean thick sets, in two chunks: counts, hulls,
    thresholds and statistics equal the oracle's run on the same sets."""
    w = synth.make_config(1, fraction=0.1)
    g, h = w.geometry, w.histories
    ref = oracle_mod.run_euclid(g, h, d0, threads=16)
    half = len(h) // 2
    with hd.Scan(g) as s:
        s.set_thick_distance(d0)
        s.add([torch.from_numpy(a[:half]).cuda() for a in h.arrays()])
        s.add([torch.from_numpy(a[half:]).cuda() for a in h.arrays()])
        s.finalize()
        torch.cuda.synchronize()
        mt, slope, index = s.thresholds()
        got = {"N": s.counts(hd.HD_MSC), "M": s.counts(hd.HD_SM), "H1": s.mask(hd.HD_SC),
               "H2": s.mask(hd.HD_MSC), "H3": s.mask(hd.HD_SM), "Mt": mt, "slope": slope,
               "index": index}
        st = s.stats()
    for k, v in got.items():
        assert np.array_equal(v, ref[k]), k
    names = ["n_in", "n_miss", "n_hit", "n_none", "n_reject", "steps_miss", "steps_hit"]
    for i, k in enumerate(names):
        assert st[k] == int(ref["stats"][i]), k


def test_config2_sample_across_slices(hd, oracle_mod):
    """The head-sized geometry (2.5 mm slices) at d_0 = 2.5 mm: the sets reach
    the neighbouring slices; 50 histories of every angle."""
    w = synth.make_config(2, fraction=0.0005)
    g, h = w.geometry, w.histories
    ref = oracle_mod.accumulate_euclid(g, h, 2.5, threads=16)
    N, M, _ = _gpu_counts(hd, g, h, 2.5)
    assert np.array_equal(N, ref["N"]) and np.array_equal(M, ref["M"])
    # thickness across slices: some set reaches more slices than its thin path
    thin = oracle_mod.accumulate(g, h)
    per_slice = lambda a: (a.reshape(g.nz, -1).sum(1) > 0).sum()
    assert per_slice(ref["N"]) >= per_slice(thin["N"])


def test_euclid_api_errors(hd):
    g = synth.geometry_for(1)
    p = hd.hd_params_default()
    dev = [torch.zeros(4, dtype=torch.float32, device="cuda") for _ in range(6)]
    N = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    M = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    for bad in (-0.5, 64.5, float("nan")):
        with pytest.raises(hd.HDError) as e:
            hd.hd_accumulate_euclid(g, p, bad, dev, N, M)
        assert e.value.status == hd.HD_ERR_RANGE
    with hd.Scan(g) as s:
        with pytest.raises(hd.HDError) as e:
            s.set_thick_distance(-1.0)
        assert e.value.status == hd.HD_ERR_RANGE
        s.add(dev)
        with pytest.raises(hd.HDError) as e:
            s.set_thick_distance(1.0)
        assert e.value.status == hd.HD_ERR_STATE
    with hd.Scan(g) as s, hd.Batch(2) as b:
        s.set_thick_distance(1.0)
        with pytest.raises(hd.HDError) as e:
            b.add(s, dev)
        assert e.value.status == hd.HD_ERR_STATE
