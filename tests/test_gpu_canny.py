"""The edge-detection SM threshold on the GPU against the oracle, bit for
bit: random count volumes of awkward sizes at three quantiles, the M volumes
of scans, a disk and a flat slice."""
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


def _check(hd, oracle_mod, M, dims, q):
    mt, he, H3 = hd.hd_sm_canny(torch.from_numpy(np.ascontiguousarray(M, np.uint32).ravel()
                                                 .view(np.int32)).cuda(), dims, q_pct=q)
    torch.cuda.synchronize()
    ref = oracle_mod.sm_canny(M, dims, q_pct=q)
    assert np.array_equal(mt.cpu().numpy().view(np.uint32), ref["Mt"])
    assert np.array_equal(he.cpu().numpy(), ref["has_edge"])
    assert np.array_equal(H3.cpu().numpy(), ref["H3"])
    return ref


@pytest.mark.parametrize("dims", [(23, 17, 2), (1, 7, 2), (7, 1, 3), (40, 40, 1), (95, 130, 3),
                                  (200, 200, 4), (600, 500, 1)])
def test_random_volumes(hd, oracle_mod, dims):
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 7 + ny)
    yy, xx = np.mgrid[0:ny, 0:nx]
    blob = ((xx - nx / 2.1) ** 2 / (0.3 * nx + 1) ** 2 + (yy - ny / 1.9) ** 2 / (0.35 * ny + 1) ** 2) < 1
    M = (rng.integers(0, 300, (nz, ny, nx)) + 900 * blob[None]).astype(np.uint32)
    for q in (0, 50, 100):
        _check(hd, oracle_mod, M, dims, q)


def test_large_counts(hd, oracle_mod):
    """Counts near 2^32: the smoothed and derivative values need 64 bits."""
    rng = np.random.default_rng(5)
    M = rng.integers(2 ** 32 - 2 ** 20, 2 ** 32, (2, 33, 31), dtype=np.uint64).astype(np.uint32)
    M[:, 10:20, 8:25] //= 3
    _check(hd, oracle_mod, M, (31, 33, 2), 50)


def test_scan_volumes(hd, oracle_mod):
    for cid, frac in ((1, 1.0), (2, 0.2)):
        w = synth.make_config(cid, fraction=frac)
        g = w.geometry
        with hd.Scan(g) as s:
            s.add([torch.from_numpy(a).cuda() for a in w.histories.arrays()])
            s.finalize()
            M = s.counts(hd.HD_SM)
        _check(hd, oracle_mod, np.asarray(M), (g.nx, g.ny, g.nz), 50)


def test_disk_and_flat(hd, oracle_mod):
    nx = ny = 40
    yy, xx = np.mgrid[0:ny, 0:nx]
    disk = (xx - 19.3) ** 2 + (yy - 20.6) ** 2 <= 12.5 ** 2
    M = np.stack([np.where(disk, 1000, 0), np.full((ny, nx), 77)]).astype(np.uint32)
    ref = _check(hd, oracle_mod, M, (nx, ny, 2), 50)
    assert ref["Mt"][0] == 1000 and ref["has_edge"][1] == 0


def test_range(hd):
    M = torch.zeros(800 * 1000, dtype=torch.int32, device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.hd_sm_canny(M, (800, 1000, 1))
    assert e.value.status == hd.HD_ERR_RANGE


def test_many_edge_voxels(hd, oracle_mod):
    """Stripes give more edge voxels than the shared-memory list holds, so
    the select runs over the edge bitmap."""
    nx, ny = 300, 200
    yy, xx = np.mgrid[0:ny, 0:nx]
    M = np.where((xx // 4) % 2 == 0, 1000 + 7 * yy, 10 + xx % 13).astype(np.uint32)[None]
    ref = oracle_mod.sm_canny(M, (nx, ny, 1), debug=True)
    assert ref["edge"].sum() > 4096
    for q in (0, 50, 100):
        _check(hd, oracle_mod, M, (nx, ny, 1), q)
