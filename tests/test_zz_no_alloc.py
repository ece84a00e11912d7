"""The allocation-free entry point (hd_accumulate_noalloc), for callers that
cannot allocate device memory when they run the traversal.  Its counts must
equal those of a regular scan on the same histories, on two calls in a row
(the shared scratch array keeps what the previous call left in it).

This file is collected last on purpose, so a run that stops at its first
failure has already run every other test; it must also pass on its own in a
fresh process."""
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


def _scan_counts(hd, g, dev):
    with hd.Scan(g) as s:
        s.add(dev)
        s.finalize()
        torch.cuda.synchronize()
        return s.counts(hd.HD_MSC), s.counts(hd.HD_SM)


def test_noalloc_matches_scan_twice(hd):
    w = synth.make_config(1, fraction=0.6)  # 108000 histories: under the 262144 limit
    g, h = w.geometry, w.histories
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    N_ref, M_ref = _scan_counts(hd, g, dev)
    assert N_ref.sum() > 0 and M_ref.sum() > 0
    params = hd.hd_params_default()
    for _ in range(2):
        N = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
        M = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
        hd.hd_accumulate_noalloc(g, params, *dev, N, M)
        torch.cuda.synchronize()
        assert np.array_equal(N.cpu().numpy().view(np.uint32), N_ref)
        assert np.array_equal(M.cpu().numpy().view(np.uint32), M_ref)


def test_noalloc_accumulates_chunks_and_limits(hd):
    w = synth.make_config(1, fraction=0.25)
    g, h = w.geometry, w.histories
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    N_ref, M_ref = _scan_counts(hd, g, dev)
    N = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    M = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    params = hd.hd_params_default()
    half = len(h) // 2
    hd.hd_accumulate_noalloc(g, params, *[a[:half] for a in dev], N, M)
    hd.hd_accumulate_noalloc(g, params, *[a[half:] for a in dev], N, M)
    torch.cuda.synchronize()
    assert np.array_equal(N.cpu().numpy().view(np.uint32), N_ref)
    assert np.array_equal(M.cpu().numpy().view(np.uint32), M_ref)
    # beyond the fixed scratch size: a clear error, nothing launched
    big = [torch.zeros(262145, dtype=torch.float32, device="cuda") for _ in range(6)]
    with pytest.raises(hd.HDError) as e:
        hd.hd_accumulate_noalloc(g, params, *big, N, M)
    assert e.value.status == hd.HD_ERR_RANGE
    # a requested class without its output volume
    with pytest.raises(hd.HDError) as e:
        hd.hd_accumulate_noalloc(g, params, *dev, N, None)
    assert e.value.status == hd.HD_ERR_ARG


def test_noalloc_method_subsets_unaligned_inputs_and_oracle(hd, oracle_mod):
    """SM alone with no N volume, on inputs starting one element into their
    arrays (not 16-byte aligned: the ingest kernel's scalar loads), against
    the oracle; then SC alone (N only) on the same inputs."""
    w = synth.make_config(1, fraction=0.3)
    g, h = w.geometry, w.histories
    dev = [torch.from_numpy(a).cuda()[1:] for a in h.arrays()]
    assert dev[0].data_ptr() % 16 != 0
    sub = h.take(np.arange(1, len(h)))
    ref = oracle_mod.run(g, sub, threads=8)
    p = hd.hd_params_default()
    p.methods = hd.HD_SM
    M = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    hd.hd_accumulate_noalloc(g, p, *dev, None, M)
    torch.cuda.synchronize()
    assert np.array_equal(M.cpu().numpy().view(np.uint32), ref["M"])
    p.methods = hd.HD_SC
    N = torch.zeros(g.n_voxels, dtype=torch.int32, device="cuda")
    hd.hd_accumulate_noalloc(g, p, *dev, N, None)
    torch.cuda.synchronize()
    assert np.array_equal(N.cpu().numpy().view(np.uint32), ref["N"])
