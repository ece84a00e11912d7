"""Rows of the hull-restricted system matrix on the GPU against the oracle:
every row, element by element and in path order, for each hull (the GPU's
own hull masks, themselves pinned elsewhere, are the oracle's input so that
the rows are compared alone)."""
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


def _scan(hd, g, h):
    s = hd.Scan(g)
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    s.add(dev)
    s.finalize()
    torch.cuda.synchronize()
    return s, dev


def _check_rows(hd, oracle_mod, s, g, h, dev, methods=None):
    methods = methods or [hd.HD_SC, hd.HD_MSC, hd.HD_SM]
    for m in methods:
        row_ptr, cols = s.system_rows(m, dev)
        torch.cuda.synchronize()
        hull = s.mask(m)
        ref_ptr, ref_cols = oracle_mod.system_rows(g, h, hull, threads=8)
        assert np.array_equal(row_ptr.cpu().numpy(), ref_ptr), m
        assert np.array_equal(cols.cpu().numpy(), ref_cols), m


def test_rows_config1(hd, oracle_mod):
    w = synth.make_config(1, fraction=0.3)
    s, dev = _scan(hd, w.geometry, w.histories)
    _check_rows(hd, oracle_mod, s, w.geometry, w.histories, dev)
    s.close()


@pytest.mark.parametrize("g", [synth.Geometry(8, 8, 4, 1.0, 1.0, 1.0, 8.0),
                               synth.Geometry(16, 16, 2, 1.0, 1.0, 2.5, 16.0)])
def test_rows_lattice_ties(hd, oracle_mod, g):
    """Segments through voxel edges and corners: the path order of the tie
    rule (an axis moving + enters at the crossing, one moving - just after)."""
    from tests.test_gpu_parity import _lattice_histories
    h = _lattice_histories(np.random.default_rng(g.nx + 3), g, 3000)
    s, dev = _scan(hd, g, h)
    _check_rows(hd, oracle_mod, s, g, h, dev)
    s.close()


def test_rows_hull_beyond_shared_memory(hd, oracle_mod):
    """A grid whose hull bitmap (51 200 words) exceeds what a block keeps in
    shared memory: the kernels test the hull as bytes from global memory,
    voxel by voxel along either axis; every row of every hull equals the
    oracle's."""
    g = synth.Geometry(160, 160, 64, 1.0, 1.0, 1.0, 120.0)
    h = synth.tiny_random_case(np.random.default_rng(21), 4000, g, span=1.3)
    s, dev = _scan(hd, g, h)
    _check_rows(hd, oracle_mod, s, g, h, dev)
    s.close()


def test_rows_rejected_histories_are_empty(hd, oracle_mod):
    w = synth.make_config(1, fraction=0.05)
    h = w.histories
    arrs = [a.copy() for a in h.arrays()]
    arrs[1][::7] = np.nan
    arrs[2][3::11] = 5000.0
    h2 = synth.Histories(*arrs)
    s, dev = _scan(hd, w.geometry, h2)
    row_ptr, cols = s.system_rows(hd.HD_SC, dev)
    lens = np.diff(row_ptr.cpu().numpy())
    assert np.all(lens[::7] == 0) and np.all(lens[3::11] == 0)
    _check_rows(hd, oracle_mod, s, w.geometry, h2, dev, [hd.HD_SC])
    s.close()


def test_rows_capacity_and_errors(hd):
    w = synth.make_config(1, fraction=0.05)
    s, dev = _scan(hd, w.geometry, w.histories)
    n = len(w.histories)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    small = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.hd_scan_system_rows(s.handle, hd.HD_MSC, *dev[:5], row_ptr, small)
    assert e.value.status == hd.HD_ERR_RANGE
    total = int(row_ptr[-1].item())
    assert total > 10
    full_ptr, cols = s.system_rows(hd.HD_MSC, dev)
    assert torch.equal(full_ptr, row_ptr) and len(cols) == total
    # a scan that is not finalised has no hull
    with hd.Scan(w.geometry) as s2:
        s2.add(dev)
        with pytest.raises(hd.HDError) as e:
            hd.hd_scan_system_rows(s2.handle, hd.HD_MSC, *dev[:5], row_ptr, cols)
        assert e.value.status == hd.HD_ERR_STATE
    s.close()


def test_rows_config2_sample(hd, oracle_mod):
    """The head-sized scan's MSC hull; rows of a sample of 150k histories."""
    w = synth.make_config(2)
    s, dev = _scan(hd, w.geometry, w.histories)
    idx = np.random.default_rng(4).choice(len(w.histories), 150_000, replace=False)
    idx.sort()
    sub = w.histories.take(idx)
    sub_dev = [torch.from_numpy(a).cuda() for a in sub.arrays()]
    _check_rows(hd, oracle_mod, s, w.geometry, sub, sub_dev, [hd.HD_MSC, hd.HD_SM])
    s.close()
