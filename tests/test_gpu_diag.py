"""Hull diagnostics on the GPU against the oracle: the enclosed part of a mask
per slice and the extra/missing counts against the true object, bit for bit,
on random masks of awkward sizes and on the hulls of scans."""
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


def _fill_gpu(hd, mask, dims):
    out = hd.hd_fill_enclosed(torch.from_numpy(np.ascontiguousarray(mask).ravel()).cuda(), dims)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dims,p", [((17, 13, 3), 0.35), ((1, 9, 2), 0.3), ((9, 1, 2), 0.3),
                                    ((33, 31, 4), 0.45), ((64, 64, 8), 0.4),
                                    ((200, 200, 4), 0.42), ((784, 700, 2), 0.41),
                                    ((95, 257, 3), 0.38)])
def test_fill_random_masks(hd, oracle_mod, dims, p):
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 1000 + ny)
    mask = (rng.random(nx * ny * nz) >= p).astype(np.uint8)
    assert np.array_equal(_fill_gpu(hd, mask, dims), oracle_mod.fill_enclosed(mask, dims))


def test_fill_rings_and_spiral(hd, oracle_mod):
    """Nested rings and a spiral corridor (the exterior must travel far)."""
    n = 101
    m = np.ones((n, n), np.uint8)
    for r in range(2, n // 2, 4):
        m[r, r:n - r] = 0
        m[n - 1 - r, r:n - r] = 0
        m[r:n - r, r] = 0
        m[r:n - r, n - 1 - r] = 0
        m[r, r + 1] = 1  # an opening in every ring: a spiral-like corridor
    for vol in (m, 1 - m):
        v = np.ascontiguousarray(np.stack([vol, vol.T]))
        assert np.array_equal(_fill_gpu(hd, v, (n, n, 2)), oracle_mod.fill_enclosed(v, (n, n, 2)))


def test_fill_of_msc_hulls(hd, oracle_mod):
    for cid, frac in ((1, 1.0), (2, 0.2)):
        w = synth.make_config(cid, fraction=frac)
        g = w.geometry
        dims = (g.nx, g.ny, g.nz)
        with hd.Scan(g) as s:
            s.add([torch.from_numpy(a).cuda() for a in w.histories.arrays()])
            s.finalize()
            h2 = s.mask(hd.HD_MSC)
        assert np.array_equal(_fill_gpu(hd, h2, dims), oracle_mod.fill_enclosed(h2, dims))


def test_compare_random_and_scan(hd, oracle_mod):
    rng = np.random.default_rng(9)
    for dims in [(7, 5, 3), (200, 200, 32), (1, 1, 1)]:
        V = int(np.prod(dims))
        h = (rng.random(V) < 0.4).astype(np.uint8)
        o = (rng.random(V) < 0.3).astype(np.uint8)
        c = hd.hd_hull_compare(torch.from_numpy(h).cuda(), torch.from_numpy(o).cuda(), dims)
        ref = oracle_mod.hull_compare(h, o, dims)
        got = c.cpu().numpy()
        nz = dims[2]
        assert np.array_equal(got[:nz], ref["extra_per_slice"])
        assert np.array_equal(got[nz:2 * nz], ref["missing_per_slice"])
        assert (got[2 * nz], got[2 * nz + 1]) == (ref["extra"], ref["missing"])


def test_fill_range_and_args(hd):
    big = torch.zeros(800 * 1000, dtype=torch.uint8, device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.hd_fill_enclosed(big, (800, 1000, 1))
    assert e.value.status == hd.HD_ERR_RANGE
    with pytest.raises(ValueError):
        hd.hd_fill_enclosed(np.zeros(8, np.uint8), (2, 2, 2))
