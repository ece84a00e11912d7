"""Serving (continuous batching of streamed scans): every scan's result is
identical alone and in the mix, admission by device footprint, bounded
staging memory with bounded submit waits, and bounded waits that give up on
a scan whose last chunk never arrives."""
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


def test_served_equals_alone(hd, oracle_mod, scans_case):
    """Every served scan equals the same scan run alone and the oracle."""
    refs = [_alone(hd, sp.geometry, h) for sp, h, _ in scans_case]
    for (sp, h, _), ref in zip(scans_case, refs):
        orc = oracle_mod.run(sp.geometry, h, threads=8)
        for k in ref:
            assert np.array_equal(ref[k], orc[k]), k
    with hd.Server() as srv:
        ids = [srv.open_scan(sp.geometry, None, len(ch)) for sp, _, ch in scans_case]
        # chunks alternate between pageable numpy arrays, page-locked host
        # tensors, device tensors, and the rows of one page-locked or device
        # 6 x n array (equally spaced columns: one strided copy per submit)
        payload = []
        for k, (_, _, ch) in enumerate(scans_case):
            row = []
            for j, c in enumerate(ch):
                kind = (k + j) % 5
                if kind == 0:
                    row.append(c.arrays())
                elif kind == 1:
                    row.append([torch.from_numpy(a).pin_memory() for a in c.arrays()])
                elif kind == 2:
                    row.append([torch.from_numpy(a).cuda() for a in c.arrays()])
                else:
                    block = torch.from_numpy(np.stack(c.arrays()))
                    row.append(block.pin_memory() if kind == 3 else block.cuda())
            payload.append(row)
        torch.cuda.synchronize()

        # a client thread interleaves the chunks of all scans
        def client():
            pos = [0] * len(ids)
            while any(p < len(ch) for p, (_, _, ch) in zip(pos, scans_case)):
                for k, (sid, (_, _, ch)) in enumerate(zip(ids, scans_case)):
                    if pos[k] < len(ch):
                        item = payload[k][pos[k]]
                        if isinstance(item, list):
                            srv.submit(sid, item)
                        else:  # a 6 x n array: one strided copy
                            srv.submit_rows(sid, item, 0, item.shape[1])
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
        assert st["launches"] <= st["items_launched"] <= st["chunks_launched"]


def test_admission_by_footprint(hd, scans_case):
    cfg = hd.hd_server_config_default()
    cfg.max_chunk = 20000
    cfg.segment_histories = 20000
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


def test_staging_backpressure(hd, scans_case):
    """Two staging segments only, and room for one scan: the waiting scan's
    chunks fill the staging and a further submit gives up after its timeout;
    once the first scan is closed the second one is admitted, its segments
    run, and submits go through again.  Both results equal the lone scans."""
    (sp_a, h_a, ch_a), (sp_b, h_b, ch_b) = scans_case[0], scans_case[1]
    cfg = hd.hd_server_config_default()
    cfg.max_chunk = 20000
    cfg.segment_histories = 40000
    cfg.staging_bytes = 2 * 24 * 40000
    cfg.submit_timeout_ms = 300
    fp = lambda g: g.n_voxels * 11 + g.n_voxels // 4 + 40000 * (28 + 512) + (4 << 20)
    cfg.hbm_budget_bytes = max(fp(sp_a.geometry), fp(sp_b.geometry)) + 1  # one scan at a time
    with hd.Server(cfg) as srv:
        a = srv.open_scan(sp_a.geometry, None, len(ch_a))
        b = srv.open_scan(sp_b.geometry, None, len(ch_b))
        for c in ch_a:
            srv.submit(a, c.arrays())
        assert srv.wait(a, 60000) == hd.HD_OK
        assert srv.info(b)["state"] == 0  # not admitted while a is open
        # b's chunks fill both segments (at least 2 x 20000 histories each)
        k = 0
        timed_out = False
        while k < len(ch_b):
            try:
                srv.submit(b, ch_b[k].arrays())
            except hd.HDError as e:
                assert e.status == hd.HD_ERR_TIMEOUT
                timed_out = True
                break
            k += 1
        assert timed_out and 2 <= k < len(ch_b)
        got_a = _served(hd, srv.scan(a, sp_a.geometry))
        ref_a = _alone(hd, sp_a.geometry, h_a)
        for key in ref_a:
            assert np.array_equal(got_a[key], ref_a[key]), key
        srv.close_scan(a)
        for c in ch_b[k:]:  # the refused chunk again, then the rest
            srv.submit(b, c.arrays())
        assert srv.wait(b, 60000) == hd.HD_OK
        got_b = _served(hd, srv.scan(b, sp_b.geometry))
        ref_b = _alone(hd, sp_b.geometry, h_b)
        for key in ref_b:
            assert np.array_equal(got_b[key], ref_b[key]), key
        st = srv.stats()
        assert st["chunks_launched"] == len(ch_a) + len(ch_b)
        srv.close_scan(b)


def test_closed_scans_are_reused(hd, scans_case):
    """A closed scan is kept and reset for the next scan of the same geometry
    and parameters: the second scan gets the same results as a lone scan."""
    sp, h, ch = scans_case[0]
    ref = _alone(hd, sp.geometry, h)
    with hd.Server() as srv:
        for _ in range(2):
            sid = srv.open_scan(sp.geometry, None, len(ch))
            for c in ch:
                srv.submit(sid, c.arrays())
            assert srv.wait(sid, 60000) == hd.HD_OK
            got = _served(hd, srv.scan(sid, sp.geometry))
            for k in ref:
                assert np.array_equal(got[k], ref[k]), k
            srv.close_scan(sid)
        st = srv.stats()
        assert st["scans_reused"] == 1
        assert st["bytes_pooled"] > 0 and st["bytes_in_use"] == 0
