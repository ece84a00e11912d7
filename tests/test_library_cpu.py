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


_CTYPE = {"int32_t": "c_int", "uint32_t": "c_uint", "int64_t": "c_long", "float": "c_float",
          "double": "c_double", "size_t": "c_ulong"}


def _header_structs():
    text = open(os.path.join(ROOT, "include", "hulld.h")).read()
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(\w+);", text, re.S):
        body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
        fields = []
        for decl in body.split(";"):
            parts = decl.split()
            if parts:
                fields += [(parts[0], n.strip()) for n in " ".join(parts[1:]).split(",")]
        out[m.group(2)] = fields
    return out


def test_binding_structs_match_the_header(hd):
    """Every struct of include/hulld.h has a ctypes twin with the same fields
    in the same order and of the same C types (an ABI drift guard)."""
    import ctypes
    structs = _header_structs()
    assert len(structs) >= 11
    for name, fields in structs.items():
        cls = getattr(hd, name)
        got = [(f, t) for f, t in cls._fields_]
        assert [f for f, _ in got] == [n for _, n in fields], name
        for (_, t), (ctype, n) in zip(got, fields):
            want = getattr(ctypes, _CTYPE[ctype])
            assert ctypes.sizeof(t) == ctypes.sizeof(want), (name, n)
            assert (t in (ctypes.c_float, ctypes.c_double)) == (ctype in ("float", "double")), n


def test_binned_params_default_matches_the_oracle(hd, oracle_mod):
    """A host-only call: the paper's bins for a geometry, as the oracle
    derives them."""
    from paper_1402_1720_gb300 import synth
    for g in [synth.geometry_for(1), synth.geometry_for(2), synth.geometry_for(3),
              synth.Geometry(128, 128, 32, 1.0, 1.0, 2.5, 110.0),
              synth.Geometry(33, 70, 5, 0.7, 1.3, 3.0, 80.0)]:
        p = hd.hd_binned_params_default(g)
        bp = oracle_mod.binned_params_for(g)
        assert (p.angle_bin_deg, p.u_bin_mm, p.v_bin_mm, p.k_sigma, p.window,
                p.min_count) == (4.0, 1.0, 5.0, 3, 5, 11)
        assert (p.u_lo_mm, p.v_lo_mm, p.n_u, p.n_v, p.miss_wepl_mm) == \
            (bp.u_lo_mm, bp.v_lo_mm, bp.n_u, bp.v_bins, 1.0)


def test_workspace_queries(hd):
    """Host-only size queries: enough room for the difference arrays, and the
    documented range errors."""
    from paper_1402_1720_gb300 import synth
    g = synth.geometry_for(2)
    V = g.nx * g.ny * g.nz
    assert hd.hd_accumulate_thick_workspace(g) >= 16 * V
    assert hd.hd_sm_canny_workspace((g.nx, g.ny, g.nz)) >= 18 * V
    with pytest.raises(hd.HDError) as e:
        hd.hd_sm_canny_workspace((800, 1000, 1))
    assert e.value.status == hd.HD_ERR_RANGE
    with pytest.raises(hd.HDError) as e:
        hd.hd_binned_params_default(synth.Geometry(0, 4, 4, 1.0, 1.0, 1.0, 10.0))
    assert e.value.status == hd.HD_ERR_RANGE
