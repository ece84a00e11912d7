"""Autotuner for the traversal's launch parameters (hd_tuning).

For one volume class (grid size) it times a scan of a sample workload with
each candidate setting through the C ABI (CUDA events around reset + add +
finalize on the scan's stream) and keeps the fastest, searching one
parameter at a time (slab depth, block size, refill threshold, job size)
from the library's defaults.  Results are cached in a JSON file keyed by the
grid and the GPU name, so a batch of scans tunes each class once.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional, Sequence

from . import hulld

DEFAULT = {"threads": 1024, "refill": 12, "job_size": 32767, "slab_depth": 0}
SPACE = {
    "slab_depth": [0, 2, 4],
    "threads": [256, 512, 768, 1024],
    "refill": [4, 8, 12, 16, 24],
    "job_size": [4096, 8192, 16384, 32767],
}


def _key(geometry, device_name: str) -> str:
    g = hulld._geometry(geometry)
    return f"{device_name}|{g.nx}x{g.ny}x{g.nz}"


def _tuning(d: Dict[str, int]) -> "hulld.hd_tuning":
    return hulld.hd_tuning(int(d["threads"]), int(d["refill"]), int(d["job_size"]),
                           int(d["slab_depth"]))


def time_setting(geometry, arrays: Sequence, setting: Dict[str, int], params=None,
                 repeats: int = 3, warmup: int = 1) -> float:
    """Mean ms of reset + add + finalize with `setting` (device arrays)."""
    import torch
    stream = torch.cuda.Stream()
    with hulld.Scan(geometry, params) as s:
        hulld.hd_scan_set_tuning(s.handle, _tuning(setting))
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                s.reset(stream)
                s.add(arrays, stream)
                s.finalize(stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(repeats):
                s.reset(stream)
                s.add(arrays, stream)
                s.finalize(stream)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / repeats


def autotune(geometry, arrays: Sequence, params=None, space: Optional[Dict] = None,
             repeats: int = 3, order: Iterable[str] = ("slab_depth", "threads", "refill",
                                                       "job_size")) -> Dict:
    """Coordinate search from the defaults; returns the best setting and its
    time, plus every trial."""
    space = space or SPACE
    best = dict(DEFAULT)
    best_ms = time_setting(geometry, arrays, best, params, repeats)
    trials = [(dict(best), best_ms)]
    for name in order:
        for v in space[name]:
            if v == best[name]:
                continue
            cand = dict(best)
            cand[name] = v
            ms = time_setting(geometry, arrays, cand, params, repeats)
            trials.append((cand, ms))
            if ms < best_ms:
                best, best_ms = cand, ms
    return {"setting": best, "ms": best_ms, "trials": trials}


def cache_path() -> str:
    return os.environ.get("HULLD_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hulld_tuning.json"))


def load_cache(path: Optional[str] = None) -> Dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_setting(geometry, sample_arrays: Optional[Sequence] = None, params=None,
                  path: Optional[str] = None, repeats: int = 3) -> Dict[str, int]:
    """The cached setting of this volume class on this GPU; tuned now (on
    the sample) when missing, defaults when there is no sample."""
    import torch
    dev = torch.cuda.get_device_name()
    key = _key(geometry, dev)
    cache = load_cache(path)
    if key in cache:
        return cache[key]["setting"]
    if sample_arrays is None:
        return dict(DEFAULT)
    res = autotune(geometry, sample_arrays, params, repeats=repeats)
    cache = load_cache(path)
    cache[key] = {"setting": res["setting"], "ms": res["ms"]}
    save_cache(cache, path)
    return res["setting"]


def apply(scan: "hulld.Scan", setting: Dict[str, int]) -> None:
    hulld.hd_scan_set_tuning(scan.handle, _tuning(setting))
