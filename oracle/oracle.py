"""Python face of the CPU oracle (test infrastructure only).

The arithmetic lives in hull_oracle.c, compiled here with gcc and called
through ctypes.  The CORDIC constants are computed below with exact integer
arithmetic from their definitions; nothing is shared with the CUDA library.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading
from pathlib import Path
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "hull_oracle.c"
_OUT = _HERE / "_build" / "liboracle.so"
_lib = None
_lock = threading.Lock()

SC, MSC, SM = 1, 2, 4


# ------------------------------------------------------------------ build
def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C99 + __int128, no arch flags)."""
    if force or not _OUT.exists() or _OUT.stat().st_mtime < _SRC.stat().st_mtime:
        _OUT.parent.mkdir(exist_ok=True)
        tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                               "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(str(build()))
            i64p = ctypes.POINTER(ctypes.c_int64)
            f32p = ctypes.POINTER(ctypes.c_float)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            L.oracle_cordic.argtypes = [ctypes.c_int64, i64p, ctypes.c_int64, i64p, i64p]
            L.oracle_cordic.restype = None
            L.oracle_grid_endpoints.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int64] + \
                [ctypes.c_float] * 5 + [i64p, i64p]
            L.oracle_grid_endpoints.restype = ctypes.c_int
            L.oracle_voxel_set.argtypes = [i64p, i64p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, i64p, ctypes.c_int64]
            L.oracle_voxel_set.restype = ctypes.c_int64
            L.oracle_segment_meets_voxel.argtypes = [i64p, i64p, ctypes.c_int64,
                                                     ctypes.c_int64, ctypes.c_int64]
            L.oracle_segment_meets_voxel.restype = ctypes.c_int
            L.oracle_classify.argtypes = [ctypes.c_float] * 3
            L.oracle_classify.restype = ctypes.c_int
            L.oracle_accumulate.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                                            ctypes.c_int32, i64p, ctypes.c_int64] + \
                [f32p] * 6 + [ctypes.c_int64, u32p, u32p, u8p, i64p]
            L.oracle_accumulate.restype = ctypes.c_int
            L.oracle_sc_from_counts.argtypes = [u32p, ctypes.c_int64, u8p]
            L.oracle_sc_from_counts.restype = None
            L.oracle_msc_decide.argtypes = [u32p] + [ctypes.c_int32] * 5 + [u8p]
            L.oracle_msc_decide.restype = None
            L.oracle_sm_decide.argtypes = [u32p] + [ctypes.c_int32] * 6 + [u32p, u32p, i64p, u8p]
            L.oracle_sm_decide.restype = None
            L.oracle_count_through_voxel.argtypes = [ctypes.c_void_p, ctypes.c_float,
                                                     ctypes.c_float, i64p, ctypes.c_int64] + \
                [f32p] * 6 + [ctypes.c_int64, ctypes.c_int32] + [ctypes.c_int64] * 3
            L.oracle_count_through_voxel.restype = ctypes.c_int64
            L.oracle_voxel_path.argtypes = [i64p, i64p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, i64p, ctypes.c_int64]
            L.oracle_voxel_path.restype = ctypes.c_int64
            L.oracle_system_rows.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int64] + \
                [f32p] * 5 + [ctypes.c_int64, u8p, i64p, ctypes.POINTER(ctypes.c_int32)]
            L.oracle_system_rows.restype = ctypes.c_int
            f64p = ctypes.POINTER(ctypes.c_double)
            L.oracle_grid_endpoints_fp64.argtypes = [ctypes.c_void_p] + [ctypes.c_float] * 5 + \
                [f64p, f64p]
            L.oracle_grid_endpoints_fp64.restype = ctypes.c_int
            L.oracle_voxel_set_fp64.argtypes = [f64p, f64p, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, i64p, ctypes.c_int64]
            L.oracle_voxel_set_fp64.restype = ctypes.c_int64
            L.oracle_compare_fp64.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                                              ctypes.c_int32, i64p, ctypes.c_int64] + \
                [f32p] * 6 + [ctypes.c_int64, u32p, u32p, i64p]
            L.oracle_compare_fp64.restype = ctypes.c_int
            L.oracle_accumulate_thick.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                                                  ctypes.c_int32, i64p, ctypes.c_int64,
                                                  ctypes.c_int32] + [f32p] * 6 + \
                [ctypes.c_int64, u32p, u32p, i64p]
            L.oracle_accumulate_thick.restype = ctypes.c_int
            L.oracle_in_capsule.argtypes = [i64p, i64p, i64p, ctypes.c_int64]
            L.oracle_in_capsule.restype = ctypes.c_int
            L.oracle_capsule_of.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int64] + \
                [ctypes.c_float] * 6 + [i64p, i64p, i64p]
            L.oracle_capsule_of.restype = ctypes.c_int
            L.oracle_accumulate_euclid.argtypes = [ctypes.c_void_p, ctypes.c_float,
                                                   ctypes.c_float, ctypes.c_int32, i64p,
                                                   ctypes.c_int64, ctypes.c_float] + \
                [f32p] * 6 + [ctypes.c_int64, u32p, u32p, i64p]
            L.oracle_accumulate_euclid.restype = ctypes.c_int
            L.oracle_segment_meets_box.argtypes = [i64p, i64p, i64p, i64p]
            L.oracle_segment_meets_box.restype = ctypes.c_int
            L.oracle_count_thick_voxels.argtypes = [ctypes.c_void_p, ctypes.c_float,
                                                    ctypes.c_float, i64p, ctypes.c_int64,
                                                    ctypes.c_int32] + [f32p] * 6 + \
                [ctypes.c_int64, ctypes.c_int32, i64p, ctypes.c_int64, i64p]
            L.oracle_count_thick_voxels.restype = None
            L.oracle_sm_canny.argtypes = [u32p] + [ctypes.c_int32] * 4 + [u32p, u8p, u8p] + \
                [i64p] * 4 + [u8p, u8p]
            L.oracle_sm_canny.restype = ctypes.c_int
            L.oracle_hull_compare.argtypes = [u8p, u8p] + [ctypes.c_int32] * 3 + [i64p]
            L.oracle_hull_compare.restype = None
            L.oracle_fill_enclosed.argtypes = [u8p] + [ctypes.c_int32] * 3 + [u8p]
            L.oracle_fill_enclosed.restype = ctypes.c_int
            L.oracle_bin_line.argtypes = [ctypes.c_void_p, ctypes.c_int64, f32p, f32p]
            L.oracle_bin_line.restype = None
            L.oracle_slice_bin.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           f32p]
            L.oracle_slice_bin.restype = ctypes.c_int64
            L.oracle_sc_binned.argtypes = [ctypes.c_void_p, ctypes.c_void_p, i64p,
                                           ctypes.c_int64] + [f32p] * 6 + \
                [ctypes.c_int64, i64p, u8p, u8p, i64p]
            L.oracle_sc_binned.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ------------------------------------------------------ CORDIC constants
def _atan_inv_fixed(m: int, bits: int) -> int:
    """atan(1/m) * 2^bits by its Taylor series, exact integer arithmetic
    (error below the number of terms in the last place)."""
    one = 1 << bits
    total, k = 0, 0
    power = m
    while True:
        term = one // (power * (2 * k + 1))
        if term == 0:
            break
        total += -term if k & 1 else term
        k += 1
        power *= m * m
    return total


def cordic_table(bits: int = 256) -> Tuple[Tuple[int, ...], int]:
    """theta_i = round(atan(2^-i) * 180/pi * 2^30), i = 0..31, and
    K = round(2^30 * prod_i (1 + 2^-2i)^(-1/2)), from exact series:
    pi by Machin's formula pi/4 = 4 atan(1/5) - atan(1/239)."""
    pi = 4 * (4 * _atan_inv_fixed(5, bits) - _atan_inv_fixed(239, bits))
    theta = [45 << 30]  # atan(1) = pi/4 = 45 degrees exactly
    for i in range(1, 32):
        a = _atan_inv_fixed(1 << i, bits)
        theta.append((2 * a * 180 * (1 << 30) + pi) // (2 * pi))
    P = 1
    for i in range(32):
        P *= (1 << (2 * i)) + 1
    Qexp = 2 * sum(range(32))
    m = 64
    # K = round(sqrt(2^60 * 2^Qexp / P))
    s = math.isqrt(((1 << (60 + Qexp + 2 * m)) // P))
    K = (s + (1 << (m - 1))) >> m
    return tuple(theta), K


_TABLE = None


def _table_arrays():
    global _TABLE
    if _TABLE is None:
        theta, K = cordic_table()
        _TABLE = (np.asarray(theta, dtype=np.int64), int(K))
    return _TABLE


def cordic(angle_q16: int) -> Tuple[int, int]:
    """(cos, sin) with 30 fractional bits of an angle in degrees * 2^16."""
    th, K = _table_arrays()
    c = ctypes.c_int64()
    s = ctypes.c_int64()
    lib().oracle_cordic(int(angle_q16), _p(th, ctypes.c_int64), K, ctypes.byref(c),
                        ctypes.byref(s))
    return c.value, s.value


# ------------------------------------------------------------- geometry
class _OGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("sx", ctypes.c_float), ("sy", ctypes.c_float), ("sz", ctypes.c_float),
                ("T", ctypes.c_float)]


def _ogeom(g) -> _OGeom:
    return _OGeom(int(g.nx), int(g.ny), int(g.nz), float(g.sx), float(g.sy), float(g.sz),
                  float(g.T))


def grid_endpoints(g, angle, u_in, v_in, u_out, v_out):
    """(rejected, gin[3], gout[3]) of one history in grid Q16 coordinates."""
    th, K = _table_arrays()
    gin = np.zeros(3, np.int64)
    gout = np.zeros(3, np.int64)
    og = _ogeom(g)
    r = lib().oracle_grid_endpoints(ctypes.byref(og), _p(th, ctypes.c_int64), K,
                                    float(angle), float(u_in), float(v_in), float(u_out),
                                    float(v_out), _p(gin, ctypes.c_int64),
                                    _p(gout, ctypes.c_int64))
    return bool(r), gin, gout


def voxel_set(gin, gout, nx: int, ny: int, nz: int) -> np.ndarray:
    """Sorted linear indices (x fastest) of A_i for the closed segment."""
    gin = np.ascontiguousarray(gin, dtype=np.int64)
    gout = np.ascontiguousarray(gout, dtype=np.int64)
    cap = nx + ny + nz + 8
    out = np.zeros(cap, np.int64)
    m = lib().oracle_voxel_set(_p(gin, ctypes.c_int64), _p(gout, ctypes.c_int64), nx, ny, nz,
                               _p(out, ctypes.c_int64), cap)
    if m < 0 or m > cap:
        raise RuntimeError("oracle_voxel_set failed")
    return out[:m].copy()


def segment_meets_voxel(gin, gout, x: int, y: int, z: int) -> bool:
    gin = np.ascontiguousarray(gin, dtype=np.int64)
    gout = np.ascontiguousarray(gout, dtype=np.int64)
    return bool(lib().oracle_segment_meets_voxel(_p(gin, ctypes.c_int64),
                                                 _p(gout, ctypes.c_int64), x, y, z))


def voxel_set_bruteforce(gin, gout, nx: int, ny: int, nz: int) -> np.ndarray:
    """A_i by testing every voxel of the grid with the slab test."""
    gin = np.ascontiguousarray(gin, dtype=np.int64)
    gout = np.ascontiguousarray(gout, dtype=np.int64)
    f = lib().oracle_segment_meets_voxel
    pi, po = _p(gin, ctypes.c_int64), _p(gout, ctypes.c_int64)
    out = [x + nx * (y + ny * z) for z in range(nz) for y in range(ny) for x in range(nx)
           if f(pi, po, x, y, z)]
    return np.asarray(out, dtype=np.int64)


def count_through_voxel(g, hist, cls: int, x: int, y: int, z: int,
                        params: Params = None) -> int:
    """|C(v)| of one voxel by testing every history of class `cls`
    (1 missed -> N(v), 2 hit -> M(v)) with the slab test."""
    params = params or Params()
    th, K = _table_arrays()
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    return int(lib().oracle_count_through_voxel(
        ctypes.byref(og), params.tau_l, params.tau_h, _p(th, ctypes.c_int64), K,
        *[_p(a, ctypes.c_float) for a in arrs], len(hist), cls, x, y, z))


def classify(wepl, tau_l: float = 1.0, tau_h: float = 5.0) -> np.ndarray:
    """0 neither, 1 missed (Eq. 3.1), 2 hit (Eq. 3.7), one history at a time."""
    f = lib().oracle_classify
    return np.asarray([f(float(w), tau_l, tau_h) for w in np.asarray(wepl, np.float32)],
                      dtype=np.uint8)


# ---------------------------------------------------------------- params
@dataclasses.dataclass(frozen=True)
class Params:
    tau_l: float = 1.0      # missed cutoff on WEPL, mm (Sec. 3.3)
    tau_h: float = 5.0      # hit cutoff on WEPL, mm (Sec. 3.4)
    nt: int = 50            # MSC neighbour-difference threshold N_t (Sec. 3.3)
    nbhd: int = 6           # B(v): 6 face neighbours (index units) or 4 in-plane
    sm_ge: int = 1          # H_3 uses M >= M_t (1) or M > M_t (0)
    sm_per_slice: int = 1   # SM threshold per slice (1) or over the volume (0)
    methods: int = SC | MSC | SM


# ----------------------------------------------------------- accumulation
def accumulate(g, hist, params: Params = Params(), want_h1: bool = True) -> Dict:
    """N, M, carved H1 and stats over all histories (single thread)."""
    V = g.nx * g.ny * g.nz
    N = np.zeros(V, np.uint32)
    M = np.zeros(V, np.uint32)
    H1 = np.ones(V, np.uint8) if want_h1 else None
    stats = np.zeros(8, np.int64)
    _accumulate_into(g, hist, 0, len(hist), params, N, M, H1, stats)
    return _pack_acc(N, M, H1, stats)


def _pack_acc(N, M, H1, stats):
    return {"N": N, "M": M, "H1_carved": H1,
            "stats": {"n_in": int(stats[0]), "n_miss": int(stats[1]), "n_hit": int(stats[2]),
                      "n_none": int(stats[3]), "n_reject": int(stats[4]),
                      "steps_miss": int(stats[5]), "steps_hit": int(stats[6])}}


def _accumulate_into(g, hist, s, e, params, N, M, H1, stats):
    th, K = _table_arrays()
    arrs = [np.ascontiguousarray(a[s:e], dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    r = lib().oracle_accumulate(ctypes.byref(og), params.tau_l, params.tau_h, params.methods,
                                _p(th, ctypes.c_int64), K,
                                *[_p(a, ctypes.c_float) for a in arrs], e - s,
                                _p(N, ctypes.c_uint32), _p(M, ctypes.c_uint32),
                                _p(H1, ctypes.c_uint8) if H1 is not None else None,
                                _p(stats, ctypes.c_int64))
    if r != 0:
        raise MemoryError("oracle_accumulate")


def accumulate_parallel(g, hist, params: Params = Params(), threads: Optional[int] = None,
                        want_h1: bool = True) -> Dict:
    """The same sums split over history ranges, each thread with its own
    volumes, added at the end (integer sums, so the result is identical)."""
    n = len(hist)
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, n // 1000 + 1))
    V = g.nx * g.ny * g.nz
    parts = []
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    for t in range(threads):
        parts.append((np.zeros(V, np.uint32), np.zeros(V, np.uint32),
                      np.ones(V, np.uint8) if want_h1 else None, np.zeros(8, np.int64)))
    ths = [threading.Thread(target=_accumulate_into,
                            args=(g, hist, int(bounds[t]), int(bounds[t + 1]), params) + parts[t])
           for t in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    N = np.zeros(V, np.uint32)
    M = np.zeros(V, np.uint32)
    H1 = np.ones(V, np.uint8) if want_h1 else None
    stats = np.zeros(8, np.int64)
    for pN, pM, pH, ps in parts:
        N += pN
        M += pM
        if want_h1:
            H1 &= pH
        stats += ps
    return _pack_acc(N, M, H1, stats)


# -------------------------------------------------------------- decisions
def sc_from_counts(N: np.ndarray) -> np.ndarray:
    N = np.ascontiguousarray(N, np.uint32)
    H1 = np.zeros(N.shape[0], np.uint8)
    lib().oracle_sc_from_counts(_p(N, ctypes.c_uint32), N.shape[0], _p(H1, ctypes.c_uint8))
    return H1


def msc_decide(N: np.ndarray, dims, nt: int = 50, nbhd: int = 6) -> np.ndarray:
    nx, ny, nz = dims
    N = np.ascontiguousarray(N, np.uint32).reshape(-1)
    H2 = np.zeros(N.shape[0], np.uint8)
    lib().oracle_msc_decide(_p(N, ctypes.c_uint32), nx, ny, nz, nt, nbhd, _p(H2, ctypes.c_uint8))
    return H2


def sm_decide(M: np.ndarray, dims, per_slice: int = 1, nbhd: int = 6, ge: int = 1) -> Dict:
    nx, ny, nz = dims
    M = np.ascontiguousarray(M, np.uint32).reshape(-1)
    H3 = np.zeros(M.shape[0], np.uint8)
    Mt = np.zeros(nz, np.uint32)
    slope = np.zeros(nz, np.uint32)
    index = np.zeros(nz, np.int64)
    lib().oracle_sm_decide(_p(M, ctypes.c_uint32), nx, ny, nz, per_slice, nbhd, ge,
                           _p(Mt, ctypes.c_uint32), _p(slope, ctypes.c_uint32),
                           _p(index, ctypes.c_int64), _p(H3, ctypes.c_uint8))
    return {"H3": H3, "Mt": Mt, "slope": slope, "index": index}


def run(g, hist, params: Params = Params(), threads: Optional[int] = 1) -> Dict:
    """Everything the hull-detection path returns for one scan."""
    if threads == 1:
        acc = accumulate(g, hist, params)
    else:
        acc = accumulate_parallel(g, hist, params, threads)
    dims = (g.nx, g.ny, g.nz)
    out = dict(acc)
    out["H1"] = sc_from_counts(acc["N"])
    out["H2"] = msc_decide(acc["N"], dims, params.nt, params.nbhd)
    sm = sm_decide(acc["M"], dims, params.sm_per_slice, params.nbhd, params.sm_ge)
    out.update(sm)
    return out


# ------------------------------------------- FP64 geometry (reported only)
def grid_endpoints_fp64(g, angle, u_in, v_in, u_out, v_out):
    """(rejected, gin, gout) with unquantised FP64 geometry (voxel units)."""
    gin = np.zeros(3, np.float64)
    gout = np.zeros(3, np.float64)
    og = _ogeom(g)
    r = lib().oracle_grid_endpoints_fp64(ctypes.byref(og), float(angle), float(u_in),
                                         float(v_in), float(u_out), float(v_out),
                                         _p(gin, ctypes.c_double), _p(gout, ctypes.c_double))
    return bool(r), gin, gout


def voxel_set_fp64(gin, gout, nx: int, ny: int, nz: int) -> np.ndarray:
    gin = np.ascontiguousarray(gin, np.float64)
    gout = np.ascontiguousarray(gout, np.float64)
    cap = nx + ny + nz + 8
    out = np.zeros(cap, np.int64)
    m = lib().oracle_voxel_set_fp64(_p(gin, ctypes.c_double), _p(gout, ctypes.c_double),
                                    nx, ny, nz, _p(out, ctypes.c_int64), cap)
    if m < 0 or m > cap:
        raise MemoryError("oracle_voxel_set_fp64")
    return out[:m].copy()


def _compare_into(g, hist, s, e, params, N64, M64, cmp):
    th, K = _table_arrays()
    arrs = [np.ascontiguousarray(a[s:e], dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    r = lib().oracle_compare_fp64(ctypes.byref(og), params.tau_l, params.tau_h, params.methods,
                                  _p(th, ctypes.c_int64), K,
                                  *[_p(a, ctypes.c_float) for a in arrs], e - s,
                                  _p(N64, ctypes.c_uint32), _p(M64, ctypes.c_uint32),
                                  _p(cmp, ctypes.c_int64))
    if r != 0:
        raise MemoryError("oracle_compare_fp64")


def compare_fp64(g, hist, params: Params = Params(), threads: Optional[int] = None,
                 fixed: Optional[Dict] = None) -> Dict:
    """How much the fixed-point geometry changes the result against the
    same set definition on FP64 geometry (reported, not a parity check):
    the fraction of voxel memberships in exactly one of the two sets, the
    fraction of histories whose sets differ, and the fraction of voxels whose
    H_1, H_2 or H_3 decision differs.  `fixed` may pass the fixed-point
    result (oracle.run or the GPU's) to skip recomputing it."""
    n = len(hist)
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, n // 1000 + 1))
    V = g.nx * g.ny * g.nz
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    parts = [(np.zeros(V, np.uint32), np.zeros(V, np.uint32), np.zeros(8, np.int64))
             for _ in range(threads)]
    ths = [threading.Thread(target=_compare_into,
                            args=(g, hist, int(bounds[t]), int(bounds[t + 1]), params) + parts[t])
           for t in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    N64 = sum(p[0] for p in parts)
    M64 = sum(p[1] for p in parts)
    cmp = sum(p[2] for p in parts)
    if fixed is None:
        fixed = run(g, hist, params, threads=threads)
    dims = (g.nx, g.ny, g.nz)
    H1 = sc_from_counts(N64)
    H2 = msc_decide(N64, dims, params.nt, params.nbhd)
    H3 = sm_decide(M64, dims, params.sm_per_slice, params.nbhd, params.sm_ge)["H3"]
    out = {"histories": int(cmp[0]), "memberships": int(cmp[1]),
           "membership_diff": int(cmp[2]),
           "membership_diff_frac": float(cmp[2]) / max(1, int(cmp[1])),
           "histories_differing_frac": float(cmp[3]) / max(1, int(cmp[0])),
           "histories_one_geometry_only": int(cmp[4]), "voxels": V}
    for k, h in (("H1", H1), ("H2", H2), ("H3", H3)):
        ref = np.asarray(fixed[k])
        d = int(np.count_nonzero(ref != h))
        out[f"{k}_voxels_differing"] = d
        out[f"{k}_diff_frac_of_hull"] = d / max(1, int(np.count_nonzero(ref)))
    return out


# ------------------------ hull-restricted system-matrix rows (next row f1)
def voxel_path(gin, gout, nx: int, ny: int, nz: int) -> np.ndarray:
    """The voxels of A_i in the order the path meets them."""
    gin = np.ascontiguousarray(gin, np.int64)
    gout = np.ascontiguousarray(gout, np.int64)
    cap = nx + ny + nz + 8
    out = np.zeros(cap, np.int64)
    m = lib().oracle_voxel_path(_p(gin, ctypes.c_int64), _p(gout, ctypes.c_int64), nx, ny, nz,
                                _p(out, ctypes.c_int64), cap)
    if m < 0 or m > cap:
        raise MemoryError("oracle_voxel_path")
    return out[:m].copy()


def _rows_range(g, hist, s, e, hull):
    th, K = _table_arrays()
    arrs = [np.ascontiguousarray(a[s:e], dtype=np.float32) for a in hist.arrays()[:5]]
    og = _ogeom(g)
    nnz = np.zeros(e - s, np.int64)
    f = lib().oracle_system_rows
    args = [ctypes.byref(og), _p(th, ctypes.c_int64), K] + [_p(a, ctypes.c_float) for a in arrs]
    if f(*args, e - s, _p(hull, ctypes.c_uint8), _p(nnz, ctypes.c_int64), None) != 0:
        raise MemoryError("oracle_system_rows")
    cols = np.zeros(max(1, int(nnz.sum())), np.int32)
    if f(*args, e - s, _p(hull, ctypes.c_uint8), _p(nnz, ctypes.c_int64),
         _p(cols, ctypes.c_int32)) != 0:
        raise MemoryError("oracle_system_rows")
    return nnz, cols[:int(nnz.sum())]


def system_rows(g, hist, hull, threads: Optional[int] = 1) -> Tuple[np.ndarray, np.ndarray]:
    """Rows of the hull-restricted system matrix (CSR): row i lists, in path
    order, the voxels of A_i that are in the hull (uint8 mask of V voxels).
    Returns (row_ptr int64 of n + 1, cols int32)."""
    hull = np.ascontiguousarray(hull, np.uint8)
    n = len(hist)
    threads = max(1, min(threads or os.cpu_count() or 1, n // 1000 + 1))
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    parts = [None] * threads

    def work(t):
        parts[t] = _rows_range(g, hist, int(bounds[t]), int(bounds[t + 1]), hull)
    ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    nnz = np.concatenate([p[0] for p in parts]) if n else np.zeros(0, np.int64)
    cols = np.concatenate([p[1] for p in parts]) if n else np.zeros(0, np.int32)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(nnz, out=row_ptr[1:])
    return row_ptr, cols


# ---------------------------------------------- thick rays (next row f4)
def accumulate_thick(g, hist, k: int, params: Params = Params()) -> Dict:
    """N and M with thick rays: A_i dilated by k voxels in-plane (Chebyshev)
    within each slice; k = 0 gives the counts of accumulate."""
    th, K = _table_arrays()
    V = g.nx * g.ny * g.nz
    N = np.zeros(V, np.uint32)
    M = np.zeros(V, np.uint32)
    stats = np.zeros(8, np.int64)
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    if lib().oracle_accumulate_thick(ctypes.byref(og), params.tau_l, params.tau_h,
                                     params.methods, _p(th, ctypes.c_int64), K, int(k),
                                     *[_p(a, ctypes.c_float) for a in arrs], len(hist),
                                     _p(N, ctypes.c_uint32), _p(M, ctypes.c_uint32),
                                     _p(stats, ctypes.c_int64)):
        raise MemoryError("oracle_accumulate_thick")
    return {"N": N, "M": M, "stats": stats}


def segment_meets_box(gin, gout, lo, hi) -> bool:
    """Slab test of the closed segment against the half-open box [lo, hi)."""
    arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in (gin, gout, lo, hi)]
    return bool(lib().oracle_segment_meets_box(*[_p(a, ctypes.c_int64) for a in arrs]))


def count_thick_voxels(g, hist, k: int, cls: int, voxels, params: Params = None) -> np.ndarray:
    """For each voxel (linear index), the histories of class cls (1 missed,
    2 hit) whose thick set A_i(k) holds it, by the slab test of the dilated
    box against every history."""
    params = params or Params()
    th, K = _table_arrays()
    vox = np.ascontiguousarray(voxels, dtype=np.int64)
    counts = np.zeros(len(vox), np.int64)
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    lib().oracle_count_thick_voxels(ctypes.byref(og), params.tau_l, params.tau_h,
                                    _p(th, ctypes.c_int64), K, int(k),
                                    *[_p(a, ctypes.c_float) for a in arrs], len(hist), int(cls),
                                    _p(vox, ctypes.c_int64), len(vox), _p(counts, ctypes.c_int64))
    return counts


def run_thick(g, hist, k: int, params: Params = Params()) -> Dict:
    """run() with every A_i replaced by its thick set A_i(k): counts from
    accumulate_thick, then the same decisions (H_1 = [N = 0])."""
    acc = accumulate_thick(g, hist, k, params)
    dims = (g.nx, g.ny, g.nz)
    out = dict(acc)
    out["H1"] = sc_from_counts(acc["N"])
    out["H2"] = msc_decide(acc["N"], dims, params.nt, params.nbhd)
    out.update(sm_decide(acc["M"], dims, params.sm_per_slice, params.nbhd, params.sm_ge))
    return out


# ------------------------------ thick rays, Euclidean distance (next row f4)
def in_capsule(A, B, C, R) -> bool:
    """Is the point C within R of the closed segment A-B (integer coordinates,
    the doubled mm * 2^16 units of capsule_of)?"""
    arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in (A, B, C)]
    return bool(lib().oracle_in_capsule(*[_p(a, ctypes.c_int64) for a in arrs], int(R)))


def capsule_of(g, d0: float, angle, u_in, v_in, u_out, v_out):
    """(rejected, A, B, R): the doubled world entry and exit points (mm * 2^17)
    and the doubled radius 2 q16(d0) of one history."""
    th, K = _table_arrays()
    A = np.zeros(3, np.int64)
    B = np.zeros(3, np.int64)
    R = np.zeros(1, np.int64)
    og = _ogeom(g)
    rej = lib().oracle_capsule_of(ctypes.byref(og), _p(th, ctypes.c_int64), K, float(d0),
                                  float(angle), float(u_in), float(v_in), float(u_out),
                                  float(v_out), _p(A, ctypes.c_int64), _p(B, ctypes.c_int64),
                                  _p(R, ctypes.c_int64))
    return bool(rej), A, B, int(R[0])


def voxel_centre2(g, x: int, y: int, z: int) -> np.ndarray:
    """Doubled centre of voxel (x, y, z) in mm * 2^16 units: (2 i + 1 - n) q16(s)."""
    q = lambda s: int(np.rint(np.float64(np.float32(s)) * 65536.0))
    return np.array([(2 * x + 1 - g.nx) * q(g.sx), (2 * y + 1 - g.ny) * q(g.sy),
                     (2 * z + 1 - g.nz) * q(g.sz)], np.int64)


def _accumulate_euclid_into(g, hist, s, e, d0, params, N, M, stats):
    th, K = _table_arrays()
    arrs = [np.ascontiguousarray(a[s:e], dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    lib().oracle_accumulate_euclid(ctypes.byref(og), params.tau_l, params.tau_h, params.methods,
                                   _p(th, ctypes.c_int64), K, float(d0),
                                   *[_p(a, ctypes.c_float) for a in arrs], e - s,
                                   _p(N, ctypes.c_uint32), _p(M, ctypes.c_uint32),
                                   _p(stats, ctypes.c_int64))


def accumulate_euclid(g, hist, d0: float, params: Params = Params(),
                      threads: Optional[int] = 1) -> Dict:
    """N and M with Euclidean thick rays (Eq. 3.2, d the Euclidean distance
    from the voxel centre to the closed segment, d_0 in mm): every voxel of
    each capsule's bounding box tested exactly; split over `threads` history
    ranges with private volumes (integer sums, so the result is the same)."""
    n = len(hist)
    threads = max(1, min(threads or os.cpu_count() or 1, n // 200 + 1))
    V = g.nx * g.ny * g.nz
    parts = [(np.zeros(V, np.uint32), np.zeros(V, np.uint32), np.zeros(8, np.int64))
             for _ in range(threads)]
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    ths = [threading.Thread(target=_accumulate_euclid_into,
                            args=(g, hist, int(bounds[t]), int(bounds[t + 1]), d0, params) + parts[t])
           for t in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    N = np.zeros(V, np.uint32)
    M = np.zeros(V, np.uint32)
    stats = np.zeros(8, np.int64)
    for pN, pM, ps in parts:
        N += pN
        M += pM
        stats += ps
    return {"N": N, "M": M, "stats": stats}


def run_euclid(g, hist, d0: float, params: Params = Params(), threads: Optional[int] = 1) -> Dict:
    """run() with every A_i replaced by its Euclidean thick set A_i(d0)."""
    acc = accumulate_euclid(g, hist, d0, params, threads)
    dims = (g.nx, g.ny, g.nz)
    out = dict(acc)
    out["H1"] = sc_from_counts(acc["N"])
    out["H2"] = msc_decide(acc["N"], dims, params.nt, params.nbhd)
    out.update(sm_decide(acc["M"], dims, params.sm_per_slice, params.nbhd, params.sm_ge))
    return out


# ------------------------------------------ hull diagnostics (next row f3)
def hull_compare(hull, obj, dims) -> Dict:
    """Extra (hull, not object) and missing (object, not hull) voxels per
    slice and in total (the counts of Tables 1-2)."""
    nx, ny, nz = dims
    h = np.ascontiguousarray(hull, np.uint8).ravel()
    o = np.ascontiguousarray(obj, np.uint8).ravel()
    counts = np.zeros(2 * nz + 2, np.int64)
    lib().oracle_hull_compare(_p(h, ctypes.c_uint8), _p(o, ctypes.c_uint8), nx, ny, nz,
                              _p(counts, ctypes.c_int64))
    return {"extra_per_slice": counts[:nz].copy(), "missing_per_slice": counts[nz:2 * nz].copy(),
            "extra": int(counts[2 * nz]), "missing": int(counts[2 * nz + 1])}


def fill_enclosed(mask, dims) -> np.ndarray:
    """Mask voxels not joined to their slice's border through the mask
    (4-connected), per slice."""
    nx, ny, nz = dims
    m = np.ascontiguousarray(mask, np.uint8).ravel()
    out = np.zeros_like(m)
    if lib().oracle_fill_enclosed(_p(m, ctypes.c_uint8), nx, ny, nz, _p(out, ctypes.c_uint8)):
        raise MemoryError("oracle_fill_enclosed")
    return out


def sm_canny(M, dims, q_pct: int = 50, debug: bool = False) -> Dict:
    """SM threshold per slice by the documented edge-detection picker: M_t,
    whether the slice has an edge, H_3 = [M >= M_t]; with debug, the smoothed
    image, Sobel derivatives, magnitude, NMS and edge masks."""
    nx, ny, nz = dims
    V = nx * ny * nz
    M = np.ascontiguousarray(M, np.uint32).ravel()
    mt = np.zeros(nz, np.uint32)
    he = np.zeros(nz, np.uint8)
    H3 = np.zeros(V, np.uint8)
    dbg = [np.zeros(V, np.int64) for _ in range(4)] + [np.zeros(V, np.uint8) for _ in range(2)]
    ptrs = [_p(a, ctypes.c_int64) for a in dbg[:4]] + [_p(a, ctypes.c_uint8) for a in dbg[4:]]
    if not debug:
        ptrs = [None] * 6
    if lib().oracle_sm_canny(_p(M, ctypes.c_uint32), nx, ny, nz, int(q_pct),
                             _p(mt, ctypes.c_uint32), _p(he, ctypes.c_uint8),
                             _p(H3, ctypes.c_uint8), *ptrs):
        raise MemoryError("oracle_sm_canny")
    out = {"Mt": mt, "has_edge": he, "H3": H3}
    if debug:
        for k, a in zip(("S", "gx", "gy", "mag", "nms", "edge"), dbg):
            out[k] = a
    return out


# ------------------------------------ SC as the paper ran it (next row f2)
class _OBinned(ctypes.Structure):
    _fields_ = [("n_ang", ctypes.c_int32), ("n_u", ctypes.c_int32), ("n_v", ctypes.c_int32),
                ("ang_q", ctypes.c_int64), ("u_q", ctypes.c_int64), ("v_q", ctypes.c_int64),
                ("u_lo_q", ctypes.c_int64), ("v_lo_q", ctypes.c_int64), ("k", ctypes.c_int32),
                ("miss_q8", ctypes.c_int64), ("w", ctypes.c_int32),
                ("min_count", ctypes.c_int32)]


@dataclasses.dataclass(frozen=True)
class BinnedParams:
    """Bins of the data cuts and of SC's lines (Sec. 2.2, Sec. 3.1: 4 degree
    angular, 1 mm lateral and 5 mm vertical bins), the 3 sigma cuts, the 1 mm
    cutoff on a bin's mean WEPL (Sec. 3.2) and the 5 x 5 average thresholded
    at 0.4 (a window of 25 needs more than 10 uncarved voxels)."""
    angle_bin_deg: float = 4.0
    u_bin_mm: float = 1.0
    v_bin_mm: float = 5.0
    u_lo_mm: float = -142.0
    v_lo_mm: float = -40.0
    n_u: int = 284
    v_bins: int = 16
    k_sigma: int = 3
    miss_wepl_mm: float = 1.0
    window: int = 5
    min_count: int = 11

    def q(self) -> _OBinned:
        """Integer form; the parameters are float32 values, scaled exactly
        and rounded to nearest even."""
        def fx(v, scale):
            return int(np.rint(np.float64(np.float32(v)) * scale))
        ang_q = fx(self.angle_bin_deg, 65536)
        n_ang = (360 * 65536) // ang_q
        if n_ang * ang_q != 360 * 65536:
            raise ValueError("angle bins must tile 360 degrees")
        return _OBinned(n_ang, self.n_u, self.v_bins, ang_q, fx(self.u_bin_mm, 65536),
                        fx(self.v_bin_mm, 65536), fx(self.u_lo_mm, 65536),
                        fx(self.v_lo_mm, 65536), self.k_sigma, fx(self.miss_wepl_mm, 256),
                        self.window, self.min_count)

    @property
    def n_bins(self) -> int:
        b = self.q()
        return b.n_ang * b.n_u * b.n_v


def binned_params_for(g, **kw) -> BinnedParams:
    """Displacement bins covering the volume's lateral half-diagonal and its
    height, at the paper's bin sizes (overridable by keyword)."""
    p = BinnedParams(**kw)
    half_u = math.ceil(math.hypot(g.nx * g.sx, g.ny * g.sy) / 2 / p.u_bin_mm) * p.u_bin_mm
    half_v = math.ceil(g.nz * g.sz / 2 / p.v_bin_mm) * p.v_bin_mm
    return dataclasses.replace(p, u_lo_mm=-half_u, n_u=int(round(2 * half_u / p.u_bin_mm)),
                               v_lo_mm=-half_v, v_bins=int(round(2 * half_v / p.v_bin_mm)),
                               **kw)


def bin_line(bp: BinnedParams, bi: int) -> Tuple[float, float]:
    """(centre angle, lateral centre) of bin bi's lines."""
    ob = bp.q()
    la, lu = ctypes.c_float(), ctypes.c_float()
    lib().oracle_bin_line(ctypes.byref(ob), int(bi), ctypes.byref(la), ctypes.byref(lu))
    return la.value, lu.value


def slice_bin(g, bp: BinnedParams, z: int) -> Tuple[int, float]:
    """(vertical bin or -1, centre height) of slice z."""
    og, ob = _ogeom(g), bp.q()
    zc = ctypes.c_float()
    iv = lib().oracle_slice_bin(ctypes.byref(og), ctypes.byref(ob), int(z), ctypes.byref(zc))
    return int(iv), zc.value


def sc_binned(g, hist, bp: BinnedParams) -> Dict:
    """Binned SC with data cuts and the averaging filter.  Returns the hull
    mask, the carved image (1 = not carved), the bin table (n_bins x 9 int64:
    n, S and Q of WEPL / lateral / vertical slope, kept n, kept WEPL sum) and
    counters."""
    th, K = _table_arrays()
    ob = bp.q()
    nb = ob.n_ang * ob.n_u * ob.n_v
    V = g.nx * g.ny * g.nz
    acc = np.zeros((nb, 9), np.int64)
    carved = np.zeros(V, np.uint8)
    mask = np.zeros(V, np.uint8)
    stats = np.zeros(6, np.int64)
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in hist.arrays()]
    og = _ogeom(g)
    r = lib().oracle_sc_binned(ctypes.byref(og), ctypes.byref(ob), _p(th, ctypes.c_int64), K,
                               *[_p(a, ctypes.c_float) for a in arrs], len(hist),
                               _p(acc, ctypes.c_int64), _p(carved, ctypes.c_uint8),
                               _p(mask, ctypes.c_uint8), _p(stats, ctypes.c_int64))
    if r != 0:
        raise MemoryError("oracle_sc_binned")
    return {"mask": mask, "carved": carved, "bins": acc,
            "stats": {"binned": int(stats[0]), "cut": int(stats[1]),
                      "bins_used": int(stats[2]), "bins_missed": int(stats[3]),
                      "lines": int(stats[4]), "lines_outside": int(stats[5])}}
