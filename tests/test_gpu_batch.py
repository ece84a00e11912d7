"""Batched execution (many scans, one persistent traversal launch, CUDA
graph replay) against one-scan-at-a-time runs and the oracle: results must
be identical (integer counts and masks)."""
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


def _outputs(hd, s):
    mt, slope, index = s.thresholds()
    return {"N": s.counts(hd.HD_MSC), "M": s.counts(hd.HD_SM), "H1": s.mask(hd.HD_SC),
            "H2": s.mask(hd.HD_MSC), "H3": s.mask(hd.HD_SM), "Mt": mt, "index": index,
            "stats": s.stats()}


def _same(a, b):
    for k in a:
        if k == "stats":
            assert a[k] == b[k]
        else:
            assert np.array_equal(a[k], b[k]), k


@pytest.fixture(scope="module")
def batch_case():
    specs = synth.batch_scan_specs(12, hist_lo=2e4, hist_hi=3e5)
    data = []
    for sp in specs:
        h = synth.scan_histories(sp)
        data.append((sp, h, [torch.from_numpy(a).cuda() for a in h.arrays()]))
    return data


def test_batch_equals_single_scans(hd, batch_case):
    refs = []
    for sp, h, dev in batch_case:
        with hd.Scan(sp.geometry) as s:
            s.add(dev)
            s.finalize()
            torch.cuda.synchronize()
            refs.append(_outputs(hd, s))
    scans = [hd.Scan(sp.geometry) for sp, _, _ in batch_case]
    stream = torch.cuda.Stream()
    with hd.Batch(len(scans)) as b:
        for rep in range(3):  # capture, then two replays of the graph
            for s, (_, _, dev) in zip(scans, batch_case):
                b.add(s, dev)
            b.run(hd.HD_BATCH_RESET | hd.HD_BATCH_FINALIZE, stream=stream)
            stream.synchronize()
            for s, ref in zip(scans, refs):
                _same(_outputs(hd, s), ref)
        st = b.stats()
        assert st["runs"] == 3 and st["graph_captures"] == 1 and st["graph_replays"] == 2
    for s in scans:
        s.close()


def test_batch_rounds_and_default_stream(hd, batch_case):
    """A scan with several chunks in one batch (successive rounds) and the
    legacy default stream (no graph)."""
    (spa, ha, deva), (spb, hb, devb) = batch_case[0], batch_case[1]
    with hd.Scan(spa.geometry) as ra, hd.Scan(spb.geometry) as rb:
        ra.add(deva)
        ra.finalize()
        rb.add(devb)
        rb.finalize()
        torch.cuda.synchronize()
        ref_a, ref_b = _outputs(hd, ra), _outputs(hd, rb)
    with hd.Scan(spa.geometry) as sa, hd.Scan(spb.geometry) as sb, hd.Batch(8) as b:
        n = len(ha)
        cuts = [0, n // 3, 2 * n // 3, n]
        for i in range(3):
            b.add(sa, [a[cuts[i]:cuts[i + 1]] for a in deva])
        b.add(sb, devb)
        b.run(hd.HD_BATCH_FINALIZE, stream=None)
        torch.cuda.synchronize()
        _same(_outputs(hd, sa), ref_a)
        _same(_outputs(hd, sb), ref_b)
        assert b.stats()["graph_captures"] == 0


def test_batch_small_scans_match_oracle(hd, oracle_mod, batch_case):
    picks = sorted(batch_case, key=lambda t: len(t[1]))[:3]
    scans = [hd.Scan(sp.geometry) for sp, _, _ in picks]
    stream = torch.cuda.Stream()
    with hd.Batch(4) as b:
        for s, (_, _, dev) in zip(scans, picks):
            b.add(s, dev)
        b.run(hd.HD_BATCH_RESET | hd.HD_BATCH_FINALIZE, stream=stream)
        stream.synchronize()
    for s, (sp, h, _) in zip(scans, picks):
        ref = oracle_mod.run(sp.geometry, h, threads=8)
        got = _outputs(hd, s)
        for k in ["N", "M", "H1", "H2", "H3", "Mt", "index"]:
            assert np.array_equal(got[k], ref[k]), k
        s.close()
