"""Full-size parity: the CUDA path at the stated sizes of every workload,
element by element against the CPU oracle.

The oracle's results were written once by oracle/make_golden.py (which calls
only the oracle and the seeded input generator) as SHA-256 hashes of every
output array, per-slice hashes and sums of N and M, and the oracle's
statistics.  Each test first checks that it generated the same inputs (their
hashes), runs the GPU in the configuration the benchmark uses, and then
compares every output hash and every statistic; a mismatch names the first
slice of N or M that differs and both sums there.

Workloads: the head-sized scan (200x200x32 voxels, 9e6 histories, one add
call), also set to Euclidean thick rays at d_0 = 2.5 and 0.5 mm and to in-plane thick
rays at k = 2, and its system-matrix rows inside the MSC hull; the large
streamed scan (400x400x128 voxels, 180 per-angle chunks of
550 000 histories, Sec. 4 online mode); the 48-scan mix in one batched run
(CUDA graph, one persistent traversal); the same 48 scans served as
per-angle chunks of 1e4-1e5 histories from page-locked host memory through
the continuous-batching server.
"""
import hashlib
import json
import multiprocessing as mp
import os
import threading

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STATS = ("n_in", "n_miss", "n_hit", "n_none", "n_reject", "steps_miss", "steps_hit")


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1402_1720_gb300 import hulld
    hulld.load()
    return hulld


def _golden(name):
    with open(os.path.join(GOLDEN, f"fullsize_{name}.json")) as f:
        return json.load(f)


def _sha(arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _pool():
    # spawn: the GPU context of this process must not be forked
    return mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))


def _outputs(hd, s):
    mt, slope, index = s.thresholds()
    return {"N": np.asarray(s.counts(hd.HD_MSC), np.uint32),
            "M": np.asarray(s.counts(hd.HD_SM), np.uint32),
            "H1": np.asarray(s.mask(hd.HD_SC), np.uint8),
            "H2": np.asarray(s.mask(hd.HD_MSC), np.uint8),
            "H3": np.asarray(s.mask(hd.HD_SM), np.uint8),
            "Mt": np.asarray(mt, np.uint32), "slope": np.asarray(slope, np.uint32),
            "index": np.asarray(index, np.int64), "stats": s.stats()}


def _check(rec, got, where):
    """Every output array and statistic against the oracle's record."""
    g = rec["geometry"]
    plane = g["nx"] * g["ny"]
    for k in STATS:
        assert got["stats"][k] == rec["stats"][k], f"{where}: {k} {got['stats'][k]} != oracle {rec['stats'][k]}"
    for k in ("N", "M"):
        if _sha([got[k]]) != rec["sha256"][k]:
            a = got[k].reshape(g["nz"], plane)
            for z in range(g["nz"]):
                if _sha([a[z]])[:16] != rec["slices"][k]["sha256"][z]:
                    pytest.fail(f"{where}: {k} first differs in slice {z}: sum "
                                f"{int(a[z].sum(dtype=np.int64))} != oracle "
                                f"{rec['slices'][k]['sum'][z]}")
            pytest.fail(f"{where}: {k} differs")
    for k in ("H1", "H2", "H3", "Mt", "slope", "index"):
        assert _sha([got[k]]) == rec["sha256"][k], \
            f"{where}: {k} differs ({int(got[k].sum())} set / sum, oracle hull sizes {rec['hull_voxels']})"


def _geom(g):
    return synth.Geometry(g["nx"], g["ny"], g["nz"], g["sx"], g["sy"], g["sz"], g["T"])


def test_head200_full_size_exact(hd):
    """9e6 histories in one add call from device memory, as the benchmark
    issues them."""
    rec = _golden("head200")
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    assert _sha(h.arrays()) == rec["inputs_sha256"], "generated inputs differ from the oracle's"
    with hd.Scan(g) as s:
        s.add([torch.from_numpy(a).cuda() for a in h.arrays()])
        s.finalize()
        torch.cuda.synchronize()
        _check(rec, _outputs(hd, s), "head200")


@pytest.mark.parametrize("name", ["euclid200", "euclid200_d05"])
def test_euclid200_full_size_exact(hd, name):
    """The head-sized scan set to Euclidean thick rays at d_0 = 2.5 mm (the
    benchmark's euclid workload) and 0.5 mm, 9e6 histories in one add call:
    counts, hulls, thresholds and statistics against the oracle's record."""
    rec = _golden(name)
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    assert _sha(h.arrays()) == rec["inputs_sha256"], "generated inputs differ from the oracle's"
    with hd.Scan(g) as s:
        s.set_thick_distance(rec["d0_mm"])
        s.add([torch.from_numpy(a).cuda() for a in h.arrays()])
        s.finalize()
        torch.cuda.synchronize()
        _check(rec, _outputs(hd, s), name)


def test_thick200_full_size_exact(hd):
    """The head-sized scan set to in-plane thick rays at k = 2 (the
    benchmark's thick workload, tiled thick traversal), 9e6 histories in one
    add call: counts, hulls, thresholds and statistics against the oracle's
    record."""
    rec = _golden("thick200")
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    assert _sha(h.arrays()) == rec["inputs_sha256"], "generated inputs differ from the oracle's"
    with hd.Scan(g) as s:
        s.set_thick(rec["k"])
        s.add([torch.from_numpy(a).cuda() for a in h.arrays()])
        s.finalize()
        torch.cuda.synchronize()
        _check(rec, _outputs(hd, s), "thick200")


def test_rows200_full_size_exact(hd):
    """The system-matrix rows of every history of the head-sized scan inside
    its MSC hull (the benchmark's rows workload: 8.3e8 column indices), in
    path order, against the oracle's record; a mismatch names the first
    block of 2^20 histories whose columns differ."""
    rec = _golden("rows200")
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    assert _sha(h.arrays()) == rec["inputs_sha256"], "generated inputs differ from the oracle's"
    with hd.Scan(g) as s:
        dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
        s.add(dev)
        s.finalize()
        hull = np.asarray(s.mask(hd.HD_MSC), np.uint8)
        assert _sha([hull]) == rec["hull_sha256"], "rows200: MSC hull differs"
        row_ptr, cols = s.system_rows(hd.HD_MSC, dev)
        torch.cuda.synchronize()
        ptr = row_ptr.cpu().numpy().astype(np.int64)
        c = cols.cpu().numpy().astype(np.int32)
    assert len(c) == rec["nnz"], f"rows200: {len(c)} nonzeros != oracle {rec['nnz']}"
    assert _sha([ptr]) == rec["row_ptr_sha256"], "rows200: row lengths differ"
    if _sha([c]) != rec["cols_sha256"]:
        b = rec["cols_block_histories"]
        for k, ref in enumerate(rec["cols_block_sha256"]):
            lo = k * b
            hi = min(lo + b, len(h))
            if _sha([c[ptr[lo]:ptr[hi]]])[:16] != ref:
                pytest.fail(f"rows200: columns first differ in histories {lo}..{hi - 1}")
        pytest.fail("rows200: columns differ")


def test_head400_streamed_full_size_exact(hd):
    """9.9e7 histories added one per-angle chunk at a time (180 calls)."""
    rec = _golden("head400")
    g = synth.geometry_for(3)
    with _pool() as pool, hd.Scan(g) as s:
        for k, chunk in enumerate(pool.imap(synth.config3_chunk, range(180))):
            assert _sha(chunk.arrays()) == rec["chunks_sha256"][k], f"chunk {k} differs"
            s.add([torch.from_numpy(a).cuda() for a in chunk.arrays()])
        s.finalize()
        torch.cuda.synchronize()
        _check(rec, _outputs(hd, s), "head400")


@pytest.fixture(scope="module")
def mix48():
    """The 48 scans of the batched/served mix (host arrays), checked against
    the oracle's input hashes."""
    rec = _golden("batch48")
    jobs = [(k, a, min(90, a + 10)) for k in range(48) for a in range(0, 90, 10)]
    with _pool() as pool:
        parts = pool.map(synth.batch_scan_part, jobs)
    specs = synth.batch_scan_specs(48)
    scans = []
    for k, sp in enumerate(specs):
        h = synth.Histories.concat([p for (kk, _, _), p in zip(jobs, parts) if kk == k])
        assert _sha(h.arrays()) == rec["scans"][k]["inputs_sha256"], f"scan {k} inputs differ"
        assert _geom(rec["scans"][k]["geometry"]) == sp.geometry
        scans.append((sp, h))
    return rec, scans


def test_batch48_full_size_exact(hd, mix48):
    """All 48 scans (1.75e8 histories) in one batched run: one persistent
    traversal over every scan, captured in a CUDA graph, then replayed."""
    rec, scans = mix48
    dev = [[torch.from_numpy(a).cuda() for a in h.arrays()] for _, h in scans]
    objs = [hd.Scan(sp.geometry) for sp, _ in scans]
    stream = torch.cuda.Stream()
    try:
        with hd.Batch(len(objs)) as b:
            for rep in range(2):  # capture, then a replay
                for s, d in zip(objs, dev):
                    b.add(s, d)
                b.run(hd.HD_BATCH_RESET | hd.HD_BATCH_FINALIZE, stream=stream)
                stream.synchronize()
                for k, s in enumerate(objs):
                    _check(rec["scans"][k], _outputs(hd, s), f"batch48 run {rep} scan {k}")
            st = b.stats()
            assert st["graph_captures"] == 1 and st["graph_replays"] == 1
    finally:
        for s in objs:
            s.close()


def test_served48_full_size_exact(hd, mix48):
    """The same 48 scans served: per-angle chunks of 1e4-1e5 histories from
    page-locked host memory (rows of one 6 x n array per scan, so each
    submit is one strided copy), submitted by four client threads round-robin
    over their scans, all scans open at once; every served scan equals the
    oracle."""
    rec, scans = mix48
    rng = np.random.default_rng(20140207)
    payload = []
    for sp, h in scans:
        # rows of one page-locked 6 x n array, as a client would hold them
        block = torch.from_numpy(np.stack(h.arrays())).pin_memory()
        pinned = [block[a] for a in range(6)]
        starts = np.flatnonzero(np.r_[True, h.angle_deg[1:] != h.angle_deg[:-1]])
        ends = np.r_[starts[1:], len(h)]
        chunks = []
        for a0, a1 in zip(starts, ends):
            s0 = a0
            while s0 < a1:
                e0 = min(a1, s0 + int(rng.integers(10_000, 100_001)))
                chunks.append((int(s0), int(e0 - s0)))
                s0 = e0
        payload.append((block, chunks))
    with hd.Server() as srv:
        ids = [srv.open_scan(sp.geometry, None, len(ch)) for (sp, _), (_, ch) in zip(scans, payload)]
        errors = []

        def client(me, nclients=4):
            mine = [k for k in range(len(ids)) if k % nclients == me]
            pos = {k: 0 for k in mine}
            try:
                while mine:
                    for k in list(mine):
                        block, chunks = payload[k]
                        srv.submit_rows(ids[k], block, *chunks[pos[k]])
                        pos[k] += 1
                        if pos[k] == len(chunks):
                            mine.remove(k)
            except Exception as e:  # pragma: no cover - reported below
                errors.append(e)

        threads = [threading.Thread(target=client, args=(i,)) for i in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for k, ((sp, _), sid) in enumerate(zip(scans, ids)):
            assert srv.wait(sid, 600_000) == hd.HD_OK
            _check(rec["scans"][k], _outputs(hd, srv.scan(sid, sp.geometry)), f"served scan {k}")
            srv.close_scan(sid)
        st = srv.stats()
        assert st["scans_done"] == 48
        assert st["launches"] < st["chunks_launched"]  # chunks of several scans per launch
