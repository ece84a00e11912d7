"""Pins for the oracle's edge-detection SM threshold picker (next row f3):
smoothing and Sobel derivatives against scipy's integer correlation,
non-maximum suppression on step edges, hysteresis against scipy's connected
components, the quantile against numpy's sort, and a disk whose hull is the
disk itself."""
import numpy as np
import pytest

from paper_1402_1720_gb300 import synth


def _rand_M(rng, dims):
    nx, ny, nz = dims
    base = rng.integers(0, 60, (nz, ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx]
    blob = ((xx - nx / 2.1) ** 2 / (0.3 * nx) ** 2 + (yy - ny / 1.9) ** 2 / (0.35 * ny) ** 2) < 1
    return (base + 400 * blob[None]).astype(np.uint32)


def test_smoothing_and_sobel_equal_scipy(oracle_mod):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    for dims in [(23, 17, 2), (5, 31, 1), (1, 7, 2), (40, 40, 1)]:
        nx, ny, nz = dims
        M = _rand_M(rng, dims)
        r = oracle_mod.sm_canny(M, dims, debug=True)
        b = np.outer([1, 2, 1], [1, 2, 1]).astype(np.int64)
        kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], np.int64)
        for z in range(nz):
            S = ndimage.correlate(M[z].astype(np.int64), b, mode="nearest")
            assert np.array_equal(r["S"].reshape(nz, ny, nx)[z], S)
            assert np.array_equal(r["gx"].reshape(nz, ny, nx)[z],
                                  ndimage.correlate(S, kx, mode="nearest"))
            assert np.array_equal(r["gy"].reshape(nz, ny, nx)[z],
                                  ndimage.correlate(S, kx.T, mode="nearest"))


def test_nms_on_step_edges(oracle_mod):
    """A step keeps one line of voxels: the first on the high side."""
    nx, ny = 24, 10
    yy, xx = np.mgrid[0:ny, 0:nx]
    M = np.where(xx >= 10, 1000, 0).astype(np.uint32)
    r = oracle_mod.sm_canny(M, (nx, ny, 1), debug=True)
    nms = r["nms"].reshape(ny, nx)
    assert np.array_equal(nms, (xx == 10).astype(np.uint8))
    M = np.where(yy >= 4, 1000, 0).astype(np.uint32)
    r = oracle_mod.sm_canny(M, (nx, ny, 1), debug=True)
    assert np.array_equal(r["nms"].reshape(ny, nx), (yy == 4).astype(np.uint8))
    assert r["Mt"][0] == 1000 and np.array_equal(r["H3"].reshape(ny, nx), (yy >= 4).astype(np.uint8))


def test_hysteresis_equals_components(oracle_mod):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    eight = np.ones((3, 3), bool)
    for dims in [(40, 36, 3), (64, 64, 2)]:
        nx, ny, nz = dims
        M = _rand_M(rng, dims) + rng.integers(0, 300, (nz, ny, nx)).astype(np.uint32)
        r = oracle_mod.sm_canny(M, dims, debug=True)
        mag = r["mag"].reshape(nz, ny, nx)
        nms = r["nms"].reshape(nz, ny, nx).astype(bool)
        edge = r["edge"].reshape(nz, ny, nx).astype(bool)
        for z in range(nz):
            mmax = mag[z][nms[z]].max()
            weak = nms[z] & (5 * mag[z] >= mmax)
            strong = nms[z] & (2 * mag[z] >= mmax)
            lab, _ = ndimage.label(weak, structure=eight)
            keep = np.unique(lab[strong])
            want = np.isin(lab, keep[keep > 0])
            assert np.array_equal(edge[z], want)
            k = int(edge[z].sum())
            for q in (0, 50, 100):
                rq = oracle_mod.sm_canny(M[z], (nx, ny, 1), q_pct=q)
                vals = np.sort(M[z][edge[z]])
                assert rq["Mt"][0] == vals[(q * (k - 1)) // 100]
                assert np.array_equal(rq["H3"], (M[z].ravel() >= rq["Mt"][0]).astype(np.uint8))


def test_disk_and_flat_slices(oracle_mod):
    nx = ny = 40
    yy, xx = np.mgrid[0:ny, 0:nx]
    disk = (xx - 19.3) ** 2 + (yy - 20.6) ** 2 <= 12.5 ** 2
    M = np.stack([np.where(disk, 1000, 0), np.full((ny, nx), 77)]).astype(np.uint32)
    r = oracle_mod.sm_canny(M, (nx, ny, 2))
    H3 = r["H3"].reshape(2, ny, nx)
    assert r["Mt"][0] == 1000 and np.array_equal(H3[0].astype(bool), disk)
    assert r["has_edge"][1] == 0 and H3[1].sum() == 0  # a flat slice has no edge
