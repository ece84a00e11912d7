"""Serving (continuous batching of streamed scans): every scan's result is
identical alone and in the mix, admission by device footprint, and bounded
waits that give up on a scan whose last chunk never arrives."""
import threading

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


def _chunks(h, rng, lo=3000, hi=20000):
    """Per-angle pieces split into chunks of lo..hi histories, in angle order."""
    out = []
    angles = np.unique(h.angle_deg)
    for a in angles:
        idx = np.flatnonzero(h.angle_deg == a)
        s = 0
        while s < len(idx):
            e = min(len(idx), s + int(rng.integers(lo, hi)))
            out.append(h.take(idx[s:e]))
            s = e
    return out


def _alone(hd, g, h):
    with hd.Scan(g) as s:
        s.add([torch.from_numpy(a).cuda() for a in h.arrays()])
        s.finalize()
        torch.cuda.synchronize()
        mt, _, idx = s.thresholds()
        return {"N": s.counts(hd.HD_MSC), "M": s.counts(hd.HD_SM), "H1": s.mask(hd.HD_SC),
                "H2": s.mask(hd.HD_MSC), "H3": s.mask(hd.HD_SM), "Mt": mt, "index": idx}


def _served(hd, view):
    mt, _, idx = view.thresholds()
    return {"N": view.counts(hd.HD_MSC), "M": view.counts(hd.HD_SM), "H1": view.mask(hd.HD_SC),
            "H2": view.mask(hd.HD_MSC), "H3": view.mask(hd.HD_SM), "Mt": mt, "index": idx}


@pytest.fixture(scope="module")
def scans_case():
    specs = synth.batch_scan_specs(10, hist_lo=2e4, hist_hi=2e5, seed=99)
    rng = np.random.default_rng(5)
    return [(sp, h, _chunks(h, rng)) for sp in specs for h in [synth.scan_histories(sp)]]


def test_served_equals_alone(hd, scans_case):
    refs = [_alone(hd, sp.geometry, h) for sp, h, _ in scans_case]
    with hd.Server() as srv:
        ids = [srv.open_scan(sp.geometry, None, len(ch)) for sp, _, ch in scans_case]
        # a client thread interleaves the chunks of all scans
        def client():
            pos = [0] * len(ids)
            while any(p < len(ch) for p, (_, _, ch) in zip(pos, scans_case)):
                for k, (sid, (_, _, ch)) in enumerate(zip(ids, scans_case)):
                    if pos[k] < len(ch):
                        srv.submit(sid, ch[pos[k]].arrays())
                        pos[k] += 1
        t = threading.Thread(target=client)
        t.start()
        t.join()
        for sid, (sp, _, _), ref in zip(ids, scans_case, refs):
            assert srv.wait(sid, 60000) == hd.HD_OK
            got = _served(hd, srv.scan(sid, sp.geometry))
            for k in ref:
                assert np.array_equal(got[k], ref[k]), k
            info = srv.info(sid)
            assert info["state"] == 2 and info["t_ready"] >= info["t_last_chunk"] >= 0
            srv.close_scan(sid)
        st = srv.stats()
        assert st["scans_done"] == len(ids) and st["bytes_in_use"] == 0
        assert st["chunks_launched"] == sum(len(ch) for _, _, ch in scans_case)
        assert st["launches"] < st["chunks_launched"]  # chunks of several scans per launch


def test_admission_by_footprint(hd, scans_case):
    cfg = hd.hd_server_config_default()
    cfg.max_chunk = 20000
    fp = max(sp.geometry.n_voxels * 11 + sp.geometry.n_voxels // 4 + 20000 * (28 + 512) + (4 << 20)
             for sp, _, _ in scans_case)
    cfg.hbm_budget_bytes = int(2.2 * fp)  # about two scans at a time
    with hd.Server(cfg) as srv:
        ids = [srv.open_scan(sp.geometry, None, len(ch)) for sp, _, ch in scans_case]
        for sid, (_, _, ch) in zip(ids, scans_case):
            for c in ch:
                srv.submit(sid, c.arrays())
        refs = {}
        remaining = list(zip(ids, scans_case))
        while remaining:
            sid, (sp, h, _) = remaining.pop(0)
            assert srv.stats()["bytes_in_use"] <= cfg.hbm_budget_bytes
            assert srv.wait(sid, 60000) == hd.HD_OK
            got = _served(hd, srv.scan(sid, sp.geometry))
            ref = _alone(hd, sp.geometry, h)
            for k in ref:
                assert np.array_equal(got[k], ref[k]), k
            srv.close_scan(sid)
        assert srv.stats()["scans_done"] == len(ids)
        # a scan that can never fit
        big = synth.Geometry(1024, 1024, 512, 0.25, 0.25, 0.25, 300.0)
        with pytest.raises(hd.HDError) as e:
            srv.open_scan(big, None, 1)
        assert e.value.status == hd.HD_ERR_ADMISSION


def test_withheld_last_chunk_times_out(hd, scans_case):
    sp, h, ch = scans_case[0]
    with hd.Server() as srv:
        sid = srv.open_scan(sp.geometry, None, len(ch) + 1)
        for c in ch:
            srv.submit(sid, c.arrays())
        # the scan waits for a chunk that has not come: a bounded wait gives up
        assert srv.wait(sid, 200) == hd.HD_ERR_TIMEOUT
        assert srv.poll(sid)[0] is False
        empty = synth.Histories(*[np.zeros(1, np.float32) for _ in range(5)],
                                np.full(1, 3.0, np.float32))  # unused history
        srv.submit(sid, empty.arrays())
        assert srv.wait(sid, 60000) == hd.HD_OK
        got = _served(hd, srv.scan(sid, sp.geometry))
        ref = _alone(hd, sp.geometry, h)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), k
        with pytest.raises(hd.HDError) as e:
            srv.submit(sid, empty.arrays())
        assert e.value.status == hd.HD_ERR_STATE
        srv.close_scan(sid)
