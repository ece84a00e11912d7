"""Python binding of libhulld (ctypes), same names as the C ABI in hulld.h.

Argument marshalling only: every step of the hull-detection path runs in the
library's CUDA kernels.  Buffers may be torch CUDA tensors (passed as device
pointers) or numpy arrays (host pointers); streams are torch.cuda.Stream
objects, raw cudaStream_t integers, or None for the current torch stream
(the legacy default stream when torch is not in use).
If the library has not been built, loading fails loudly; there is no
fallback.
"""
from __future__ import annotations

import ctypes
import threading
from pathlib import Path
from typing import Optional, Sequence

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libhulld.so"
_lib = None
_lock = threading.Lock()

HD_OK, HD_ERR_ARG, HD_ERR_RANGE, HD_ERR_NOMEM, HD_ERR_CUDA = 0, 1, 2, 3, 4
HD_ERR_STATE, HD_ERR_TIMEOUT, HD_ERR_ADMISSION, HD_ERR_OVERFLOW = 5, 6, 7, 8
HD_SC, HD_MSC, HD_SM = 1, 2, 4
HD_MASK_U8, HD_MASK_BITS = 0, 1


class HDError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = _lib
        name = lib.hd_status_string(status).decode() if lib else str(status)
        cuda = lib.hd_last_cuda_error().decode() if lib else ""
        super().__init__(f"{where}: {name}" + (f" [{cuda}]" if cuda and status == HD_ERR_CUDA else ""))


class hd_geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("sx", ctypes.c_float), ("sy", ctypes.c_float), ("sz", ctypes.c_float),
                ("tracker_half_sep_mm", ctypes.c_float)]


class hd_params(ctypes.Structure):
    _fields_ = [("wepl_miss_lt", ctypes.c_float), ("wepl_hit_gt", ctypes.c_float),
                ("msc_nt", ctypes.c_int32), ("msc_nbhd", ctypes.c_int32),
                ("sm_ge", ctypes.c_int32), ("sm_per_slice", ctypes.c_int32),
                ("methods", ctypes.c_uint32)]


class hd_stats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("n_miss", ctypes.c_int64), ("n_hit", ctypes.c_int64),
                ("n_none", ctypes.c_int64), ("n_reject", ctypes.c_int64),
                ("steps_miss", ctypes.c_int64), ("steps_hit", ctypes.c_int64),
                ("pairs_general", ctypes.c_int64), ("runs", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class hd_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("trace_launches", ctypes.c_int64),
                ("ms_ingest", ctypes.c_double), ("ms_trace", ctypes.c_double),
                ("ms_finalize", ctypes.c_double), ("ms_trace_global", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hd_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("refill", ctypes.c_int32),
                ("job_size", ctypes.c_int32), ("slab_depth", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class hd_batch_stats(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int64), ("graph_captures", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


HD_BATCH_RESET, HD_BATCH_FINALIZE = 1, 2


class hd_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_chunk", ctypes.c_int64),
                ("max_batch", ctypes.c_int32), ("max_in_flight", ctypes.c_int32),
                ("min_batch", ctypes.c_int32), ("segment_histories", ctypes.c_int64),
                ("staging_bytes", ctypes.c_size_t), ("submit_timeout_ms", ctypes.c_int64)]


class hd_server_scan_info(ctypes.Structure):
    _fields_ = [("t_open", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_first_chunk", ctypes.c_double), ("t_last_chunk", ctypes.c_double),
                ("t_ready", ctypes.c_double), ("histories", ctypes.c_int64),
                ("chunks_submitted", ctypes.c_int32), ("chunks_done", ctypes.c_int32),
                ("state", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hd_server_stats(ctypes.Structure):
    _fields_ = [("scans_opened", ctypes.c_int64), ("scans_admitted", ctypes.c_int64),
                ("scans_done", ctypes.c_int64), ("chunks_submitted", ctypes.c_int64),
                ("chunks_launched", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("issue_seconds", ctypes.c_double),
                ("submit_seconds", ctypes.c_double), ("items_launched", ctypes.c_int64),
                ("copy_seconds", ctypes.c_double), ("alloc_seconds", ctypes.c_double),
                ("scans_reused", ctypes.c_int64), ("bytes_pooled", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

class hd_binned_params(ctypes.Structure):
    _fields_ = [("angle_bin_deg", ctypes.c_float), ("u_bin_mm", ctypes.c_float),
                ("v_bin_mm", ctypes.c_float), ("u_lo_mm", ctypes.c_float),
                ("v_lo_mm", ctypes.c_float), ("n_u", ctypes.c_int32), ("n_v", ctypes.c_int32),
                ("k_sigma", ctypes.c_int32), ("miss_wepl_mm", ctypes.c_float),
                ("window", ctypes.c_int32), ("min_count", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hd_binned_stats(ctypes.Structure):
    _fields_ = [("histories_binned", ctypes.c_int64), ("histories_cut", ctypes.c_int64),
                ("bins", ctypes.c_int64), ("bins_used", ctypes.c_int64),
                ("bins_missed", ctypes.c_int64), ("lines", ctypes.c_int64),
                ("lines_outside", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


# exported symbols and their signatures
_VP, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_SIGS = {
    "hd_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "hd_last_cuda_error": ([], ctypes.c_char_p),
    "hd_params_default": ([ctypes.POINTER(hd_params)], ctypes.c_int),
    "hd_scan_create": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_params),
                        ctypes.POINTER(_VP)], ctypes.c_int),
    "hd_scan_destroy": ([_VP], ctypes.c_int),
    "hd_scan_reset": ([_VP, _VP], ctypes.c_int),
    "hd_scan_reserve": ([_VP, _I64, _VP], ctypes.c_int),
    "hd_probe_atomics": ([_I32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "hd_scan_system_rows": ([_VP, _I32] + [_VP] * 5 + [_I64, _VP, _VP, _I64,
                            ctypes.POINTER(ctypes.c_int64), _VP], ctypes.c_int),
    "hd_scan_add_histories": ([_VP] + [_VP] * 6 + [_I64, _I32, _VP], ctypes.c_int),
    "hd_scan_finalize": ([_VP, _VP], ctypes.c_int),
    "hd_scan_get_mask": ([_VP, _I32, _I32, _VP, _SZ, _I32, _VP], ctypes.c_int),
    "hd_scan_get_counts": ([_VP, _I32, _VP, _I64, _I32, _VP], ctypes.c_int),
    "hd_scan_set_counts": ([_VP, _I32, _VP, _I64, _I32, _VP], ctypes.c_int),
    "hd_scan_get_thresholds": ([_VP, _VP, _VP, _VP, _I32, _VP], ctypes.c_int),
    "hd_scan_get_stats": ([_VP, ctypes.POINTER(hd_stats), _VP], ctypes.c_int),
    "hd_scan_get_hull_indices": ([_VP, _I32, _VP, _I64, ctypes.POINTER(_I64), _I32, _VP],
                                 ctypes.c_int),
    "hd_classify": ([_VP, _I64, ctypes.POINTER(hd_params), _VP, _I32, _VP], ctypes.c_int),
    "hd_accumulate_noalloc": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_params)] +
                              [_VP] * 6 + [_I64, _VP, _VP, _VP], ctypes.c_int),
    "hd_scan_set_profiling": ([_VP, _I32], ctypes.c_int),
    "hd_scan_set_thick": ([_VP, _I32], ctypes.c_int),
    "hd_scan_set_tuning": ([_VP, ctypes.POINTER(hd_tuning)], ctypes.c_int),
    "hd_scan_get_tuning": ([_VP, ctypes.POINTER(hd_tuning)], ctypes.c_int),
    "hd_batch_create": ([_I32, ctypes.POINTER(_VP)], ctypes.c_int),
    "hd_batch_destroy": ([_VP], ctypes.c_int),
    "hd_batch_add": ([_VP, _VP] + [_VP] * 6 + [_I64], ctypes.c_int),
    "hd_batch_run": ([_VP, _I32, _VP], ctypes.c_int),
    "hd_batch_set_graph": ([_VP, _I32], ctypes.c_int),
    "hd_batch_get_stats": ([_VP, ctypes.POINTER(hd_batch_stats)], ctypes.c_int),
    "hd_batch_add_item": ([_VP, _VP] + [_VP] * 6 + [_I64, _I32], ctypes.c_int),
    "hd_server_config_default": ([ctypes.POINTER(hd_server_config)], ctypes.c_int),
    "hd_server_create": ([ctypes.POINTER(hd_server_config), ctypes.POINTER(_VP)], ctypes.c_int),
    "hd_server_destroy": ([_VP], ctypes.c_int),
    "hd_server_open_scan": ([_VP, ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_params), _I32,
                             ctypes.POINTER(_I64)], ctypes.c_int),
    "hd_server_submit_chunk": ([_VP, _I64] + [_VP] * 6 + [_I64, _I32], ctypes.c_int),
    "hd_server_submit_rows": ([_VP, _I64, _VP, _I64, _I64, _I32], ctypes.c_int),
    "hd_server_poll": ([_VP, _I64, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_int)],
                       ctypes.c_int),
    "hd_server_wait": ([_VP, _I64, _I64], ctypes.c_int),
    "hd_server_scan": ([_VP, _I64, ctypes.POINTER(_VP)], ctypes.c_int),
    "hd_server_get_info": ([_VP, _I64, ctypes.POINTER(hd_server_scan_info)], ctypes.c_int),
    "hd_server_get_stats": ([_VP, ctypes.POINTER(hd_server_stats)], ctypes.c_int),
    "hd_server_close_scan": ([_VP, _I64], ctypes.c_int),
    "hd_scan_get_profile": ([_VP, ctypes.POINTER(hd_profile)], ctypes.c_int),
    "hd_hull_compare": ([_VP, _VP, _I32, _I32, _I32, _VP, _VP], ctypes.c_int),
    "hd_accumulate_thick_workspace": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(_SZ)],
                                      ctypes.c_int),
    "hd_accumulate_thick": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_params), _I32] +
                            [_VP] * 6 + [_I64, _VP, _VP, _VP, _SZ, _VP, _VP], ctypes.c_int),
    "hd_accumulate_euclid": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_params),
                              ctypes.c_float] + [_VP] * 6 + [_I64, _VP, _VP, _VP, _SZ, _VP, _VP],
                             ctypes.c_int),
    "hd_scan_set_thick_distance": ([_VP, ctypes.c_float], ctypes.c_int),
    "hd_sm_canny_workspace": ([_I32, _I32, _I32, ctypes.POINTER(_SZ)], ctypes.c_int),
    "hd_sm_canny": ([_VP, _I32, _I32, _I32, _I32, _VP, _SZ, _VP, _VP, _VP, _VP], ctypes.c_int),
    "hd_fill_enclosed": ([_VP, _I32, _I32, _I32, _VP, _VP], ctypes.c_int),
    "hd_binned_params_default": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_binned_params)],
                                 ctypes.c_int),
    "hd_binned_create": ([ctypes.POINTER(hd_geometry), ctypes.POINTER(hd_binned_params),
                          ctypes.POINTER(_VP)], ctypes.c_int),
    "hd_binned_destroy": ([_VP], ctypes.c_int),
    "hd_binned_reset": ([_VP, _VP], ctypes.c_int),
    "hd_binned_add_histories": ([_VP] + [_VP] * 6 + [_I64, _VP], ctypes.c_int),
    "hd_binned_cut_histories": ([_VP] + [_VP] * 6 + [_I64, _VP], ctypes.c_int),
    "hd_binned_finalize": ([_VP, _VP], ctypes.c_int),
    "hd_binned_run": ([_VP] + [_VP] * 6 + [_I64, _VP], ctypes.c_int),
    "hd_binned_get_image": ([_VP, _I32, _VP, _I64, _I32, _VP], ctypes.c_int),
    "hd_binned_get_bins": ([_VP, _VP, _I64, _I32, _VP], ctypes.c_int),
    "hd_binned_get_stats": ([_VP, ctypes.POINTER(hd_binned_stats), _VP], ctypes.c_int),
}


def exported_names() -> Sequence[str]:
    return list(_SIGS)


def lib_path() -> Path:
    return _LIB_PATH


def load():
    """Load libhulld.so (built by paper_1402_1720_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not _LIB_PATH.exists():
                raise RuntimeError(f"libhulld.so not built ({_LIB_PATH}); run "
                                   "paper_1402_1720_gb300.build.build() first")
            L = ctypes.CDLL(str(_LIB_PATH))
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != HD_OK:
        raise HDError(status, where)


# ---------------------------------------------------------- marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(address, on_device) of a torch tensor or numpy array (contiguous)."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _geometry(g) -> hd_geometry:
    if isinstance(g, hd_geometry):
        return g
    return hd_geometry(int(g.nx), int(g.ny), int(g.nz), float(g.sx), float(g.sy), float(g.sz),
                       float(getattr(g, "tracker_half_sep_mm", getattr(g, "T", 0.0))))


def _params(p) -> hd_params:
    if p is None:
        return hd_params_default()
    if isinstance(p, hd_params):
        return p
    return hd_params(float(p.tau_l), float(p.tau_h), int(p.nt), int(p.nbhd), int(p.sm_ge),
                     int(p.sm_per_slice), int(p.methods))


# --------------------------------------------------- C-ABI, same names
def hd_status_string(status: int) -> str:
    return load().hd_status_string(status).decode()


def hd_last_cuda_error() -> str:
    return load().hd_last_cuda_error().decode()


def hd_params_default() -> hd_params:
    p = hd_params()
    _check(load().hd_params_default(ctypes.byref(p)), "hd_params_default")
    return p


def hd_scan_create(geometry, params=None) -> int:
    h = _VP()
    g = _geometry(geometry)
    p = _params(params)
    _check(load().hd_scan_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)),
           "hd_scan_create")
    return h.value


def hd_scan_destroy(scan: int) -> None:
    _check(load().hd_scan_destroy(scan), "hd_scan_destroy")


def hd_scan_reset(scan: int, stream=None) -> None:
    _check(load().hd_scan_reset(scan, _stream(stream)), "hd_scan_reset")


HD_PROBE_SMEM_RANDOM, HD_PROBE_SMEM_COHERENT, HD_PROBE_L2_RANDOM, HD_PROBE_HBM_RANDOM = 0, 1, 2, 3


def hd_probe_atomics(kind: int) -> float:
    """Atomics per second of one probe kind (see include/hulld.h)."""
    out = ctypes.c_double(0.0)
    _check(load().hd_probe_atomics(int(kind), ctypes.byref(out)), "hd_probe_atomics")
    return out.value


def hd_scan_system_rows(scan: int, method: int, angle_deg, u_in, v_in, u_out, v_out,
                        row_ptr, cols=None, stream=None) -> int:
    """CSR rows of the hull-restricted system matrix into device tensors
    (row_ptr: n + 1 int64; cols: int32, may be None to size it first).
    Returns the total; raises HDError(HD_ERR_RANGE) when cols is too small."""
    arrs = [angle_deg, u_in, v_in, u_out, v_out]
    ptrs = [_ptr(a) for a in arrs]
    if any(on == 0 for _, on in ptrs):
        raise ValueError("histories must be device arrays")
    rp, on = _ptr(row_ptr)
    if not on:
        raise ValueError("row_ptr must be a device array")
    cp, cap = (0, 0)
    if cols is not None:
        cp, on = _ptr(cols)
        if not on:
            raise ValueError("cols must be a device array")
        cap = len(cols)
    nnz = ctypes.c_int64(0)
    _check(load().hd_scan_system_rows(scan, int(method), *[p for p, _ in ptrs], len(arrs[0]),
                                      rp, cp or None, cap, ctypes.byref(nnz), _stream(stream)),
           "hd_scan_system_rows")
    return nnz.value


def hd_scan_reserve(scan: int, n: int, stream=None) -> None:
    _check(load().hd_scan_reserve(scan, int(n), _stream(stream)), "hd_scan_reserve")


def hd_scan_add_histories(scan: int, angle_deg, u_in, v_in, u_out, v_out, wepl,
                          stream=None) -> None:
    arrs = [angle_deg, u_in, v_in, u_out, v_out, wepl]
    ptrs = [_ptr(a) for a in arrs]
    ons = {o for _, o in ptrs}
    if len(ons) != 1:
        raise ValueError("all six arrays must be on the device or all on the host")
    n = len(arrs[0])
    for a in arrs:
        if len(a) != n:
            raise ValueError("arrays differ in length")
        dt = str(a.dtype)
        if dt not in ("float32", "torch.float32"):
            raise TypeError("history arrays must be float32")
    _check(load().hd_scan_add_histories(scan, *[p for p, _ in ptrs], n, ons.pop(),
                                        _stream(stream)), "hd_scan_add_histories")


def hd_scan_finalize(scan: int, stream=None) -> None:
    _check(load().hd_scan_finalize(scan, _stream(stream)), "hd_scan_finalize")


def hd_scan_get_mask(scan: int, method: int, layout: int, dst, stream=None) -> None:
    p, on = _ptr(dst)
    nbytes = dst.numel() * dst.element_size() if _is_torch(dst) else dst.nbytes
    _check(load().hd_scan_get_mask(scan, method, layout, p, nbytes, on, _stream(stream)),
           "hd_scan_get_mask")


def hd_scan_get_counts(scan: int, method: int, dst, stream=None) -> None:
    p, on = _ptr(dst)
    n = dst.numel() if _is_torch(dst) else dst.size
    _check(load().hd_scan_get_counts(scan, method, p, n, on, _stream(stream)),
           "hd_scan_get_counts")


def hd_scan_set_counts(scan: int, method: int, src, stream=None) -> None:
    p, on = _ptr(src)
    n = src.numel() if _is_torch(src) else src.size
    _check(load().hd_scan_set_counts(scan, method, p, n, on, _stream(stream)),
           "hd_scan_set_counts")


def hd_scan_get_thresholds(scan: int, nz: int, stream=None):
    mt = np.zeros(nz, np.uint32)
    slope = np.zeros(nz, np.uint32)
    index = np.zeros(nz, np.int64)
    _check(load().hd_scan_get_thresholds(scan, mt.ctypes.data, slope.ctypes.data,
                                         index.ctypes.data, nz, _stream(stream)),
           "hd_scan_get_thresholds")
    return mt, slope, index


def hd_scan_get_stats(scan: int, stream=None) -> dict:
    st = hd_stats()
    _check(load().hd_scan_get_stats(scan, ctypes.byref(st), _stream(stream)),
           "hd_scan_get_stats")
    return st.as_dict()


def hd_scan_get_hull_indices(scan: int, method: int, dst=None, stream=None):
    """Returns (count, dst); with dst None a host int32 array is allocated."""
    count = _I64()
    if dst is None:
        # query the size first, then fetch
        _check(load().hd_scan_get_hull_indices(scan, method, None, 0, ctypes.byref(count), 0,
                                               _stream(stream)), "hd_scan_get_hull_indices")
        dst = np.zeros(max(1, count.value), np.int32)
    p, on = _ptr(dst)
    cap = dst.numel() if _is_torch(dst) else dst.size
    _check(load().hd_scan_get_hull_indices(scan, method, p, cap, ctypes.byref(count), on,
                                           _stream(stream)), "hd_scan_get_hull_indices")
    return count.value, dst


def hd_scan_set_tuning(scan: int, tuning: hd_tuning) -> None:
    _check(load().hd_scan_set_tuning(scan, ctypes.byref(tuning)), "hd_scan_set_tuning")


def hd_scan_get_tuning(scan: int) -> dict:
    t = hd_tuning()
    _check(load().hd_scan_get_tuning(scan, ctypes.byref(t)), "hd_scan_get_tuning")
    return t.as_dict()


def hd_scan_set_thick(scan: int, k: int) -> None:
    _check(load().hd_scan_set_thick(scan, int(k)), "hd_scan_set_thick")


def hd_scan_set_thick_distance(scan: int, d0_mm: float) -> None:
    _check(load().hd_scan_set_thick_distance(scan, float(d0_mm)), "hd_scan_set_thick_distance")


def hd_scan_set_profiling(scan: int, enable: bool) -> None:
    _check(load().hd_scan_set_profiling(scan, 1 if enable else 0), "hd_scan_set_profiling")


def hd_scan_get_profile(scan: int) -> dict:
    p = hd_profile()
    _check(load().hd_scan_get_profile(scan, ctypes.byref(p)), "hd_scan_get_profile")
    return p.as_dict()


def hd_accumulate_noalloc(geometry, params, angle_deg, u_in, v_in, u_out, v_out, wepl, N, M,
                          stream=None) -> None:
    """Allocation-free accumulation into caller-owned device count volumes
    (for callers that cannot allocate; see hulld.h).  All arrays are torch
    CUDA tensors; N or M may be None when its class is not requested."""
    g = _geometry(geometry)
    p = _params(params)
    arrs = [angle_deg, u_in, v_in, u_out, v_out, wepl]
    ptrs = []
    for a in arrs:
        ptr, on = _ptr(a)
        if not on:
            raise ValueError("hd_accumulate_noalloc takes device arrays")
        ptrs.append(ptr)
    n = len(arrs[0])
    np_ = _ptr(N)[0] if N is not None else None
    mp_ = _ptr(M)[0] if M is not None else None
    _check(load().hd_accumulate_noalloc(ctypes.byref(g), ctypes.byref(p), *ptrs, n, np_, mp_,
                                        _stream(stream)), "hd_accumulate_noalloc")


def hd_classify(wepl, params=None, cls_out=None, stream=None):
    p = _params(params)
    wp, on = _ptr(wepl)
    n = wepl.numel() if _is_torch(wepl) else wepl.size
    if cls_out is None:
        if on:
            import torch
            cls_out = torch.empty(n, dtype=torch.uint8, device=wepl.device)
        else:
            cls_out = np.zeros(n, np.uint8)
    cp, con = _ptr(cls_out)
    if con != on:
        raise ValueError("wepl and cls_out must both be device or both host buffers")
    _check(load().hd_classify(wp, n, ctypes.byref(p), cp, on, _stream(stream)), "hd_classify")
    return cls_out


def hd_batch_create(max_items: int) -> int:
    h = _VP()
    _check(load().hd_batch_create(int(max_items), ctypes.byref(h)), "hd_batch_create")
    return h.value


def hd_batch_destroy(batch: int) -> None:
    _check(load().hd_batch_destroy(batch), "hd_batch_destroy")


def hd_batch_add(batch: int, scan: int, angle_deg, u_in, v_in, u_out, v_out, wepl) -> None:
    arrs = [angle_deg, u_in, v_in, u_out, v_out, wepl]
    ptrs = []
    for a in arrs:
        p, on = _ptr(a)
        if not on:
            raise ValueError("batch items take device arrays")
        ptrs.append(p)
    _check(load().hd_batch_add(batch, scan, *ptrs, len(arrs[0])), "hd_batch_add")


def hd_batch_run(batch: int, flags: int = 0, stream=None) -> None:
    _check(load().hd_batch_run(batch, int(flags), _stream(stream)), "hd_batch_run")


def hd_batch_set_graph(batch: int, enable: bool) -> None:
    _check(load().hd_batch_set_graph(batch, 1 if enable else 0), "hd_batch_set_graph")


def hd_batch_get_stats(batch: int) -> dict:
    st = hd_batch_stats()
    _check(load().hd_batch_get_stats(batch, ctypes.byref(st)), "hd_batch_get_stats")
    return st.as_dict()


def hd_batch_add_item(batch: int, scan: int, angle_deg, u_in, v_in, u_out, v_out, wepl,
                      flags: int = 0) -> None:
    arrs = [angle_deg, u_in, v_in, u_out, v_out, wepl]
    ptrs = []
    for a in arrs:
        p, on = _ptr(a)
        if not on:
            raise ValueError("batch items take device arrays")
        ptrs.append(p)
    _check(load().hd_batch_add_item(batch, scan, *ptrs, len(arrs[0]), int(flags)),
           "hd_batch_add_item")


# ------------------------------------------------------------------ serving
def hd_server_config_default() -> hd_server_config:
    c = hd_server_config()
    _check(load().hd_server_config_default(ctypes.byref(c)), "hd_server_config_default")
    return c


def hd_server_create(cfg: hd_server_config = None) -> int:
    cfg = cfg or hd_server_config_default()
    h = _VP()
    _check(load().hd_server_create(ctypes.byref(cfg), ctypes.byref(h)), "hd_server_create")
    return h.value


def hd_server_destroy(server: int) -> None:
    _check(load().hd_server_destroy(server), "hd_server_destroy")


def hd_server_open_scan(server: int, geometry, params, n_chunks: int) -> int:
    g = _geometry(geometry)
    p = _params(params)
    sid = _I64()
    _check(load().hd_server_open_scan(server, ctypes.byref(g), ctypes.byref(p), int(n_chunks),
                                      ctypes.byref(sid)), "hd_server_open_scan")
    return sid.value


def hd_server_submit_chunk(server: int, scan_id: int, angle_deg, u_in, v_in, u_out, v_out,
                           wepl) -> None:
    arrs = [angle_deg, u_in, v_in, u_out, v_out, wepl]
    ptrs = [_ptr(a) for a in arrs]
    ons = {o for _, o in ptrs}
    if len(ons) != 1:
        raise ValueError("all six arrays must be on the device or all on the host")
    _check(load().hd_server_submit_chunk(server, int(scan_id), *[p for p, _ in ptrs],
                                         len(arrs[0]), ons.pop()), "hd_server_submit_chunk")


def hd_server_submit_rows(server: int, scan_id: int, rows, start: int, n: int) -> None:
    """Submit histories start .. start + n of a 6 x N float32 array `rows`
    (host or device torch tensor, or numpy array; row a is column a of the
    structure of arrays) with one strided copy."""
    if getattr(rows, "ndim", 0) != 2 or rows.shape[0] != 6:
        raise ValueError("rows must be a 6 x N array")
    stride = rows.stride(0) if _is_torch(rows) else rows.strides[0] // rows.itemsize
    inner = rows.stride(1) if _is_torch(rows) else rows.strides[1] // rows.itemsize
    if inner != 1 or start < 0 or start + n > rows.shape[1]:
        raise ValueError("rows must be contiguous along histories and hold the range")
    base, on = _ptr(rows)
    _check(load().hd_server_submit_rows(server, int(scan_id), int(base) + 4 * int(start),
                                        int(stride), int(n), on), "hd_server_submit_rows")


def hd_server_poll(server: int, scan_id: int):
    done = _I32()
    st = ctypes.c_int()
    _check(load().hd_server_poll(server, int(scan_id), ctypes.byref(done), ctypes.byref(st)),
           "hd_server_poll")
    return bool(done.value), st.value


def hd_server_wait(server: int, scan_id: int, timeout_ms: int) -> int:
    """Returns the status (HD_OK, HD_ERR_TIMEOUT or the scan's error)."""
    return load().hd_server_wait(server, int(scan_id), int(timeout_ms))


def hd_server_scan(server: int, scan_id: int) -> int:
    h = _VP()
    _check(load().hd_server_scan(server, int(scan_id), ctypes.byref(h)), "hd_server_scan")
    return h.value


def hd_server_get_info(server: int, scan_id: int) -> dict:
    i = hd_server_scan_info()
    _check(load().hd_server_get_info(server, int(scan_id), ctypes.byref(i)), "hd_server_get_info")
    return i.as_dict()


def hd_server_get_stats(server: int) -> dict:
    st = hd_server_stats()
    _check(load().hd_server_get_stats(server, ctypes.byref(st)), "hd_server_get_stats")
    return st.as_dict()


def hd_server_close_scan(server: int, scan_id: int) -> None:
    _check(load().hd_server_close_scan(server, int(scan_id)), "hd_server_close_scan")


class ScanView:
    """Read access to a scan owned by someone else (e.g. the server)."""

    def __init__(self, handle: int, geometry):
        g = _geometry(geometry)
        self.handle = handle
        self.dims = (g.nx, g.ny, g.nz)
        self.V = g.nx * g.ny * g.nz

    def mask(self, method: int, layout: int = HD_MASK_U8, out=None, stream=None):
        return Scan.mask(self, method, layout, out, stream)

    def counts(self, method: int, out=None, stream=None):
        return Scan.counts(self, method, out, stream)

    def thresholds(self, stream=None):
        return hd_scan_get_thresholds(self.handle, self.dims[2], stream)

    def stats(self, stream=None):
        return hd_scan_get_stats(self.handle, stream)

    def sync(self, stream=None):
        hd_scan_get_stats(self.handle, stream)


class Server:
    """Owning handle of one hd_server."""

    def __init__(self, cfg: hd_server_config = None):
        self.handle = hd_server_create(cfg)

    def close(self):
        if self.handle:
            hd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def open_scan(self, geometry, params=None, n_chunks: int = 1) -> int:
        return hd_server_open_scan(self.handle, geometry, params, n_chunks)

    def submit(self, scan_id: int, arrays):
        hd_server_submit_chunk(self.handle, scan_id, *arrays)

    def submit_rows(self, scan_id: int, rows, start: int, n: int):
        """Histories start .. start + n of a 6 x N array (one strided copy)."""
        hd_server_submit_rows(self.handle, scan_id, rows, start, n)

    def wait(self, scan_id: int, timeout_ms: int) -> int:
        return hd_server_wait(self.handle, scan_id, timeout_ms)

    def poll(self, scan_id: int):
        return hd_server_poll(self.handle, scan_id)

    def scan(self, scan_id: int, geometry) -> ScanView:
        return ScanView(hd_server_scan(self.handle, scan_id), geometry)

    def info(self, scan_id: int) -> dict:
        return hd_server_get_info(self.handle, scan_id)

    def stats(self) -> dict:
        return hd_server_get_stats(self.handle)

    def close_scan(self, scan_id: int):
        hd_server_close_scan(self.handle, scan_id)


class Batch:
    """Owning handle of one hd_batch."""

    def __init__(self, max_items: int = 64):
        self.handle = hd_batch_create(max_items)

    def close(self):
        if self.handle:
            hd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, scan: "Scan", arrays):
        hd_batch_add(self.handle, scan.handle, *arrays)

    def run(self, flags: int = HD_BATCH_FINALIZE, stream=None):
        hd_batch_run(self.handle, flags, stream)

    def set_graph(self, enable: bool):
        hd_batch_set_graph(self.handle, enable)

    def stats(self) -> dict:
        return hd_batch_get_stats(self.handle)


# ------------------------------------------------------------- wrapper
class Scan:
    """Owning handle of one hd_scan."""

    def __init__(self, geometry, params=None):
        self.geometry = geometry
        self.params = _params(params)
        self.handle = hd_scan_create(geometry, self.params)
        g = _geometry(geometry)
        self.dims = (g.nx, g.ny, g.nz)
        self.V = g.nx * g.ny * g.nz

    def close(self):
        if self.handle:
            hd_scan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self, stream=None):
        hd_scan_reset(self.handle, stream)

    def reserve(self, n: int, stream=None):
        hd_scan_reserve(self.handle, n, stream)

    def set_thick(self, k: int):
        """Thick rays: A_i dilated by k voxels in-plane (before any add)."""
        hd_scan_set_thick(self.handle, k)

    def set_thick_distance(self, d0_mm: float):
        """Thick rays by Euclidean distance d0 (mm) from voxel centres to the
        path (before any add); 0 restores thin paths."""
        hd_scan_set_thick_distance(self.handle, d0_mm)

    def system_rows(self, method: int, hist_arrays: Sequence, stream=None):
        """(row_ptr, cols) device tensors of the hull-restricted system
        matrix for device histories (angle, u_in, v_in, u_out, v_out, ...)."""
        import torch
        h = list(hist_arrays)[:5]
        n = len(h[0])
        row_ptr = torch.empty(n + 1, dtype=torch.int64, device=h[0].device)
        try:
            total = hd_scan_system_rows(self.handle, method, *h, row_ptr, None, stream)
        except HDError as e:
            if e.status != HD_ERR_RANGE:
                raise
            total = int(row_ptr[-1].item())
        cols = torch.empty(max(1, total), dtype=torch.int32, device=h[0].device)
        hd_scan_system_rows(self.handle, method, *h, row_ptr, cols, stream)
        return row_ptr, cols[:total]

    def add(self, hist_arrays: Sequence, stream=None):
        hd_scan_add_histories(self.handle, *hist_arrays, stream=stream)

    def finalize(self, stream=None):
        hd_scan_finalize(self.handle, stream)

    def mask(self, method: int, layout: int = HD_MASK_U8, out=None, stream=None):
        if out is None:
            n = self.V if layout == HD_MASK_U8 else 4 * ((self.V + 31) // 32)
            out = np.zeros(n if layout == HD_MASK_U8 else n // 4,
                           np.uint8 if layout == HD_MASK_U8 else np.uint32)
        hd_scan_get_mask(self.handle, method, layout, out, stream)
        if not _is_torch(out):
            self.sync(stream)
        return out

    def counts(self, method: int, out=None, stream=None):
        if out is None:
            out = np.zeros(self.V, np.uint32)
        hd_scan_get_counts(self.handle, method, out, stream)
        if not _is_torch(out):
            self.sync(stream)
        return out

    def thresholds(self, stream=None):
        return hd_scan_get_thresholds(self.handle, self.dims[2], stream)

    def stats(self, stream=None):
        return hd_scan_get_stats(self.handle, stream)

    def hull_indices(self, method: int, dst=None, stream=None):
        return hd_scan_get_hull_indices(self.handle, method, dst, stream)

    def set_profiling(self, enable: bool):
        hd_scan_set_profiling(self.handle, enable)

    def profile(self) -> dict:
        return hd_scan_get_profile(self.handle)

    def sync(self, stream=None):
        # D2H copies into pageable numpy memory are complete when the call
        # returns; pinned destinations need a stream sync, done via stats
        hd_scan_get_stats(self.handle, stream)


# ------------------------------------------------------------ binned SC
HD_BINNED_HULL, HD_BINNED_CARVED = 0, 1


def hd_binned_params_default(geometry) -> hd_binned_params:
    p = hd_binned_params()
    g = _geometry(geometry)
    _check(load().hd_binned_params_default(ctypes.byref(g), ctypes.byref(p)),
           "hd_binned_params_default")
    return p


def _binned_params(p, geometry) -> hd_binned_params:
    if p is None:
        return hd_binned_params_default(geometry)
    if isinstance(p, hd_binned_params):
        return p
    return hd_binned_params(float(p.angle_bin_deg), float(p.u_bin_mm), float(p.v_bin_mm),
                            float(p.u_lo_mm), float(p.v_lo_mm), int(p.n_u), int(p.v_bins),
                            int(p.k_sigma), float(p.miss_wepl_mm), int(p.window),
                            int(p.min_count))


def hd_binned_create(geometry, params=None) -> int:
    h = _VP()
    g = _geometry(geometry)
    p = _binned_params(params, geometry)
    _check(load().hd_binned_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)),
           "hd_binned_create")
    return h.value


def hd_binned_destroy(b: int) -> None:
    _check(load().hd_binned_destroy(b), "hd_binned_destroy")


def hd_binned_reset(b: int, stream=None) -> None:
    _check(load().hd_binned_reset(b, _stream(stream)), "hd_binned_reset")


def _hist_ptrs(arrs):
    if len(arrs) != 6:
        raise ValueError("six history arrays (angle, u_in, v_in, u_out, v_out, wepl)")
    n = None
    ptrs = []
    for a in arrs:
        p, _ = _ptr(a)
        m = int(a.numel() if _is_torch(a) else a.size)
        n = m if n is None else n
        if m != n:
            raise ValueError("history arrays differ in length")
        ptrs.append(p)
    return ptrs, n or 0


def hd_binned_add_histories(b: int, angle_deg, u_in, v_in, u_out, v_out, wepl,
                            stream=None) -> None:
    ptrs, n = _hist_ptrs([angle_deg, u_in, v_in, u_out, v_out, wepl])
    _check(load().hd_binned_add_histories(b, *ptrs, n, _stream(stream)),
           "hd_binned_add_histories")


def hd_binned_cut_histories(b: int, angle_deg, u_in, v_in, u_out, v_out, wepl,
                            stream=None) -> None:
    ptrs, n = _hist_ptrs([angle_deg, u_in, v_in, u_out, v_out, wepl])
    _check(load().hd_binned_cut_histories(b, *ptrs, n, _stream(stream)),
           "hd_binned_cut_histories")


def hd_binned_finalize(b: int, stream=None) -> None:
    _check(load().hd_binned_finalize(b, _stream(stream)), "hd_binned_finalize")


def hd_binned_run(b: int, angle_deg, u_in, v_in, u_out, v_out, wepl, stream=None) -> None:
    ptrs, n = _hist_ptrs([angle_deg, u_in, v_in, u_out, v_out, wepl])
    _check(load().hd_binned_run(b, *ptrs, n, _stream(stream)), "hd_binned_run")


def hd_binned_get_image(b: int, which: int, dst, stream=None) -> None:
    p, on = _ptr(dst)
    n = int(dst.numel() if _is_torch(dst) else dst.size)
    _check(load().hd_binned_get_image(b, int(which), p, n, on, _stream(stream)),
           "hd_binned_get_image")


def hd_binned_get_bins(b: int, dst, stream=None) -> None:
    p, on = _ptr(dst)
    n = int(dst.numel() if _is_torch(dst) else dst.size) // 9
    _check(load().hd_binned_get_bins(b, p, n, on, _stream(stream)), "hd_binned_get_bins")


def hd_binned_get_stats(b: int, stream=None) -> dict:
    out = hd_binned_stats()
    _check(load().hd_binned_get_stats(b, ctypes.byref(out), _stream(stream)),
           "hd_binned_get_stats")
    return out.as_dict()


class Binned:
    """Binned SC object (owns an hd_binned handle)."""

    def __init__(self, geometry, params=None):
        self.geometry = geometry
        self.params = _binned_params(params, geometry)
        self.handle = hd_binned_create(geometry, self.params)
        n_ang = int(round(360.0 / self.params.angle_bin_deg))
        self.n_bins = n_ang * self.params.n_u * self.params.n_v

    def close(self):
        if self.handle:
            hd_binned_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, arrays, stream=None):
        hd_binned_run(self.handle, *arrays, stream=stream)

    def add(self, arrays, stream=None):
        hd_binned_add_histories(self.handle, *arrays, stream=stream)

    def cut(self, arrays, stream=None):
        hd_binned_cut_histories(self.handle, *arrays, stream=stream)

    def finalize(self, stream=None):
        hd_binned_finalize(self.handle, stream)

    def image(self, which: int = HD_BINNED_HULL, stream=None) -> np.ndarray:
        g = self.geometry
        out = np.zeros(int(g.nx) * int(g.ny) * int(g.nz), np.uint8)
        hd_binned_get_image(self.handle, which, out, stream)
        self._sync(stream)
        return out

    def bins(self, stream=None) -> np.ndarray:
        out = np.zeros((self.n_bins, 9), np.int64)
        hd_binned_get_bins(self.handle, out, stream)
        self._sync(stream)
        return out

    def stats(self, stream=None) -> dict:
        return hd_binned_get_stats(self.handle, stream)

    def _sync(self, stream):
        hd_binned_get_stats(self.handle, stream)  # synchronises the stream


# ------------------------------------------------------- hull diagnostics
def _dev_ptr(x, what):
    p, on = _ptr(x)
    if not on:
        raise ValueError(f"{what} must be a device tensor")
    return p


def hd_hull_compare(hull, obj, dims, counts=None, stream=None):
    """Extra/missing voxels per slice and in total (device tensors); returns
    the counts tensor (2 nz + 2 int64, on the device)."""
    import torch
    nx, ny, nz = (int(d) for d in dims)
    if counts is None:
        counts = torch.empty(2 * nz + 2, dtype=torch.int64, device=hull.device)
    _check(load().hd_hull_compare(_dev_ptr(hull, "hull"), _dev_ptr(obj, "object"), nx, ny, nz,
                                  _dev_ptr(counts, "counts"), _stream(stream)), "hd_hull_compare")
    return counts


def hd_fill_enclosed(mask, dims, out=None, stream=None):
    """Per slice, the mask voxels not joined to the border (device tensors)."""
    import torch
    nx, ny, nz = (int(d) for d in dims)
    src = _dev_ptr(mask, "mask")
    if out is None:
        out = torch.empty_like(mask)
    _check(load().hd_fill_enclosed(src, nx, ny, nz, _dev_ptr(out, "out"), _stream(stream)),
           "hd_fill_enclosed")
    return out


def hd_sm_canny_workspace(dims) -> int:
    nx, ny, nz = (int(d) for d in dims)
    out = _SZ(0)
    _check(load().hd_sm_canny_workspace(nx, ny, nz, ctypes.byref(out)), "hd_sm_canny_workspace")
    return out.value


def hd_sm_canny(M, dims, q_pct: int = 50, workspace=None, stream=None):
    """SM threshold by the documented edge-detection picker on a device
    uint32 M volume; returns (mt, has_edge, H3) device tensors."""
    import torch
    nx, ny, nz = (int(d) for d in dims)
    src = _dev_ptr(M, "M")
    need = hd_sm_canny_workspace(dims)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=M.device)
    mt = torch.empty(nz, dtype=torch.int32, device=M.device)
    he = torch.empty(nz, dtype=torch.uint8, device=M.device)
    H3 = torch.empty(nx * ny * nz, dtype=torch.uint8, device=M.device)
    _check(load().hd_sm_canny(src, nx, ny, nz, int(q_pct), _dev_ptr(workspace, "workspace"),
                              int(workspace.numel() * workspace.element_size()), _dev_ptr(mt, "mt"),
                              _dev_ptr(he, "has_edge"), _dev_ptr(H3, "H3"), _stream(stream)),
           "hd_sm_canny")
    return mt, he, H3


# ------------------------------------------------------------ thick rays
def hd_accumulate_thick_workspace(geometry) -> int:
    g = _geometry(geometry)
    out = _SZ(0)
    _check(load().hd_accumulate_thick_workspace(ctypes.byref(g), ctypes.byref(out)),
           "hd_accumulate_thick_workspace")
    return out.value


def hd_accumulate_thick(geometry, params, k: int, arrays, N, M, workspace=None, stream=None,
                        intervals=None):
    """Adds thick-ray counts (A_i dilated by k voxels in-plane) of device
    history arrays into device N, M (uint32 viewed as int32 tensors);
    `intervals` (a one-element int64 device tensor) receives the number of
    row intervals emitted."""
    import torch
    g = _geometry(geometry)
    p = _params(params)
    ptrs, n = _hist_ptrs(list(arrays))
    if workspace is None:
        workspace = torch.empty(hd_accumulate_thick_workspace(geometry), dtype=torch.uint8,
                                device="cuda")
    nptr = _dev_ptr(N, "N") if N is not None else None
    mptr = _dev_ptr(M, "M") if M is not None else None
    iptr = _dev_ptr(intervals, "intervals") if intervals is not None else None
    _check(load().hd_accumulate_thick(ctypes.byref(g), ctypes.byref(p), int(k), *ptrs, n, nptr,
                                      mptr, _dev_ptr(workspace, "workspace"),
                                      int(workspace.numel() * workspace.element_size()), iptr,
                                      _stream(stream)), "hd_accumulate_thick")


def hd_accumulate_euclid(geometry, params, d0_mm: float, arrays, N, M, workspace=None,
                         stream=None, rows=None):
    """Adds Euclidean thick-ray counts (voxel centres within d0_mm of the path)
    of device history arrays into device N, M (uint32 viewed as int32
    tensors); `rows` (a one-element int64 device tensor) receives the number
    of row intervals added."""
    import torch
    g = _geometry(geometry)
    p = _params(params)
    ptrs, n = _hist_ptrs(list(arrays))
    if workspace is None:
        workspace = torch.empty(hd_accumulate_thick_workspace(geometry), dtype=torch.uint8,
                                device="cuda")
    nptr = _dev_ptr(N, "N") if N is not None else None
    mptr = _dev_ptr(M, "M") if M is not None else None
    rptr = _dev_ptr(rows, "rows") if rows is not None else None
    _check(load().hd_accumulate_euclid(ctypes.byref(g), ctypes.byref(p), float(d0_mm), *ptrs, n,
                                       nptr, mptr, _dev_ptr(workspace, "workspace"),
                                       int(workspace.numel() * workspace.element_size()), rptr,
                                       _stream(stream)), "hd_accumulate_euclid")
