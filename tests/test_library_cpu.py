"""CPU-side checks of the C-ABI library: it builds, loads without a GPU and
exports every entry point include/hulld.h declares; host-only calls work."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hd():
    from paper_1402_1720_gb300 import build, hulld
    build.build()
    hulld.load()
    return hulld


def _declared():
    text = open(os.path.join(ROOT, "include", "hulld.h")).read()
    return sorted(set(re.findall(r"HD_API\s+[\w\s\*]+?\b(hd_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    assert "hd_scan_create" in names and "hd_scan_finalize" in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol(hd):
    lib = hd.load()
    for name in _declared():
        assert hasattr(lib, name), name
    # the binding covers the same names
    assert sorted(hd.exported_names()) == sorted(_declared())


def test_host_only_calls(hd):
    p = hd.hd_params_default()
    assert (p.wepl_miss_lt, p.wepl_hit_gt, p.msc_nt, p.msc_nbhd, p.sm_ge, p.sm_per_slice,
            p.methods) == (1.0, 5.0, 50, 6, 1, 1, 7)
    assert hd.hd_status_string(hd.HD_ERR_OVERFLOW) == "HD_ERR_OVERFLOW"
    assert hd.hd_status_string(99) == "HD_ERR_UNKNOWN"


def test_no_gpu_fails_loudly(hd):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1402_1720_gb300 import synth
    with pytest.raises(hd.HDError) as e:
        hd.Scan(synth.geometry_for(1))
    assert e.value.status == hd.HD_ERR_CUDA


def test_oracle_is_not_imported_by_the_product():
    # the library and its binding never reach the oracle
    pkg = os.path.join(ROOT, "paper_1402_1720_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "hull_oracle" not in text, f
