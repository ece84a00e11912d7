#!/usr/bin/env python
"""Throughput of the GB300 hull-detection path (SC + MSC + SM) on the
head-sized workload (200x200x32 voxels of 1x1x2.5 mm, 90 angles x 100k =
9e6 float32 histories, synthetic head phantom).

One step = one scan: reset the counts, add all histories (classify, traverse,
accumulate N and M), finalize the three hulls.  `value` is histories/s over
all ranks; `e2e` is the same metric through the C ABI from pinned host
buffers with the host->device copy of the histories and the device->host
read of the three masks inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hulld|reference]

Under torchrun (N > 1) every rank runs its own scan (independent problems,
no collective on the data path); the step time is the maximum over ranks.
`--impl reference` times the CPU oracle (the plain C statement of the
method) on a bounded sample of the same workload.

The default line also carries the traversal kernel's roofline (voxel-steps
per second against the random-address shared-memory atomic rate measured
by hd_probe_atomics in the same run), the oracle on the host cores, and two
sections on the 48-scan mix (48 scans of {64x64x16, 128x128x32, 256x256x64}
voxels, log-uniform 2e5-2e7 histories each): batched in one persistent
launch against one scan at a time, and served as per-angle chunks with
Poisson arrivals (time-to-hull percentiles).  Other workloads:
--workload batched-48 | serving | rows | binned | diagnostics | thick |
euclid | configs | large.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "proton histories/s (SC+MSC+SM hull detection)"
UNIT = "histories/s"
WORKLOAD = "head-200x200x32 voxels 1x1x2.5mm, 90 angles x 100000 = 9e6 float32 histories"

def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "sm_max_mhz": float(p.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM traffic of the traversal kernel comes from one ncu capture, summarised
# in profiles/trace_tiles_head200.md together with a hash of the kernel
# sources it was taken on; it is reported only while those sources are
# unchanged (null otherwise: the counters describe another kernel).
KERNEL_SOURCES = ["paper_1402_1720_gb300/csrc/hd_tiles.cu", "paper_1402_1720_gb300/csrc/hd_geom.cuh",
                  "paper_1402_1720_gb300/csrc/hd_internal.cuh"]
TRACE_PROFILE = "profiles/trace_tiles_head200.md"


def _kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_fields():
    """Fields of the committed ncu summary of the traversal kernel, when it
    was captured on the current kernel sources (None otherwise)."""
    path = os.path.join(ROOT, TRACE_PROFILE)
    try:
        text = open(path).read()
    except OSError:
        return None, "no capture summary"
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel sources sha256") != _kernel_sources_hash():
        return None, f"{TRACE_PROFILE} was captured on other kernel sources"
    return fields, TRACE_PROFILE


def _profiled_traffic():
    fields, note = _profile_fields()
    if fields is None:
        return None, note
    try:
        return int(fields["dram bytes per full launch"]), note
    except (KeyError, ValueError):
        return None, "no traffic figure in the capture summary"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The CPU oracle on a bounded sample of the same workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1402_1720_gb300 import synth
    oracle.build()
    frac = args.ref_fraction
    w = synth.make_config(2, fraction=frac)
    cores = os.cpu_count() or 1
    g, h = w.geometry, w.histories
    for _ in range(args.warmup):
        oracle.run(g, h, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.run(g, h, threads=cores)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = len(h) / dt
    sample = (f"{len(h)} histories per step = every angle, {frac:g} of each angle's "
              f"100000 histories, full 200x200x32 grid")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_fraction": frac},
            "voxel_steps_per_s": (r["stats"]["steps_miss"] + r["stats"]["steps_hit"]) / dt,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(seconds_target: float):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    import oracle
    from paper_1402_1720_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    frac = 0.01
    w = synth.make_config(2, fraction=frac)
    t0 = time.perf_counter()
    r = oracle.run(w.geometry, w.histories, threads=cores)
    dt = time.perf_counter() - t0
    # grow the sample toward the target CPU time (bounded)
    if dt < seconds_target / 4:
        frac = min(1.0, frac * seconds_target / max(dt, 1e-3) / 2)
        w = synth.make_config(2, fraction=frac)
        t0 = time.perf_counter()
        r = oracle.run(w.geometry, w.histories, threads=cores)
        dt = time.perf_counter() - t0
    n = len(w.histories)
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} histories (every angle, {frac:.4g} of each angle's histories) "
                      f"of the same workload on the full 200x200x32 grid, {dt:.1f} s wall",
            "voxel_steps_per_s": (r["stats"]["steps_miss"] + r["stats"]["steps_hit"]) / dt}


def mix48(args, pool=None):
    """The 48 scans of the batched/served mix (volumes from {64x64x16,
    128x128x32, 256x256x64} voxels, random ellipsoid phantoms, log-uniform
    2e5-2e7 histories each) as host arrays, generated in parallel by `pool`
    when one is given."""
    from paper_1402_1720_gb300 import synth
    specs = synth.batch_scan_specs(48, fraction=args.batch_fraction)
    if pool is not None:
        hosts = synth.batch_scans_parallel(pool, fraction=args.batch_fraction)
    else:
        hosts = [synth.scan_histories(sp) for sp in specs]
    return specs, hosts


def measure_batched(args, specs, hosts, steps, warmup):
    """One batched run per step (all scans, one persistent traversal,
    CUDA-graph replay) against the same scans one at a time on the same
    GPU; inputs resident in HBM."""
    import torch
    from paper_1402_1720_gb300 import autotune, hulld
    dev = [[torch.from_numpy(a).cuda() for a in h.arrays()] for h in hosts]
    total = sum(len(h) for h in hosts)
    scans = [hulld.Scan(sp.geometry) for sp in specs]
    # launch parameters per volume class, from the autotuner (tuned on the
    # class's largest scan, cached per grid and GPU)
    tuning = {}
    if not args.no_tune:
        for cls in sorted({(sp.geometry.nx, sp.geometry.ny, sp.geometry.nz) for sp in specs}):
            k = max((i for i, sp in enumerate(specs)
                     if (sp.geometry.nx, sp.geometry.ny, sp.geometry.nz) == cls),
                    key=lambda i: len(hosts[i]))
            tuning["x".join(map(str, cls))] = autotune.tuned_setting(specs[k].geometry, dev[k],
                                                                     repeats=2)
        for s, sp in zip(scans, specs):
            autotune.apply(s, tuning["x".join(map(str, (sp.geometry.nx, sp.geometry.ny,
                                                        sp.geometry.nz)))])
    stream = torch.cuda.Stream()
    batch = hulld.Batch(len(scans))
    flags = hulld.HD_BATCH_RESET | hulld.HD_BATCH_FINALIZE

    def batched_step():
        for s, d in zip(scans, dev):
            batch.add(s, d)
        batch.run(flags, stream=stream)

    def sequential_step():
        for s, d in zip(scans, dev):
            s.reset(stream)
            s.add(d, stream)
            s.finalize(stream)

    def timed(step, k, w):
        with torch.cuda.stream(stream):
            for _ in range(w):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    for _ in range(warmup):
        batched_step()
    torch.cuda.synchronize()
    st0 = batch.stats()
    ms_b = timed(batched_step, steps, 0)
    launches = (batch.stats()["kernel_launches"] - st0["kernel_launches"]) // max(1, steps)
    steps_total = sum(s.stats()["steps_miss"] + s.stats()["steps_hit"] for s in scans)
    ms_s = timed(sequential_step, steps, warmup)
    out = {"workload": "48 scans, grids {64x64x16,128x128x32,256x256x64} of 1x1x2.5 mm, "
                       f"log-uniform 2e5-2e7 histories each (x{args.batch_fraction:g}), "
                       "90 angles, inputs resident in HBM",
           "total_histories": total, "steps": steps, "warmup": warmup,
           "ms": ms_b, "histories_per_s": total / (ms_b * 1e-3),
           "voxel_steps_per_s": steps_total / (ms_b * 1e-3),
           "sequential_ms": ms_s, "sequential_histories_per_s": total / (ms_s * 1e-3),
           "speedup": ms_s / ms_b, "tuning": tuning, "graph": batch.stats(),
           "gpu_launches_per_step": launches,
           "grids": [f"{sp.geometry.nx}x{sp.geometry.ny}x{sp.geometry.nz}" for sp in specs]}
    batch.close()
    for s in scans:
        s.close()
    del dev
    torch.cuda.empty_cache()
    return out


def measure_serving(args, specs, hosts):
    """Poisson arrivals of the scans, each streamed as per-angle chunks of
    1e4-1e5 histories from page-locked host memory, served by the
    continuous-batching server.  First the saturated throughput X is
    measured (all scans at once); then scans arrive at rate
    load * X / (mean histories per scan).  time-to-hull = hull ready - last
    chunk submitted (and - first chunk).  Also: the same chunks added one
    scan at a time through the plain scan calls."""
    import queue
    import torch
    from paper_1402_1720_gb300 import hulld
    rng = np.random.default_rng(20140207)
    scans = []  # (spec, [chunk views of pinned tensors])
    total = 0
    for sp, h in zip(specs, hosts):
        # the six columns of a scan as rows of one page-locked 6 x n array:
        # a chunk is submitted with one strided copy (hd_server_submit_rows)
        block = torch.from_numpy(np.stack(h.arrays())).pin_memory()
        pinned = [block[a] for a in range(6)]
        bounds = []
        angles = h.angle_deg
        starts = np.flatnonzero(np.r_[True, angles[1:] != angles[:-1]])
        ends = np.r_[starts[1:], len(h)]
        for a0, a1 in zip(starts, ends):
            s0 = a0
            while s0 < a1:
                e0 = min(a1, s0 + int(rng.integers(10_000, 100_001)))
                bounds.append((s0, e0))
                s0 = e0
        scans.append((sp, [[p[a:b] for p in pinned] for a, b in bounds], block, bounds))
        total += len(h)
    cfg = hulld.hd_server_config_default()
    cfg.max_chunk = 100_000

    # one long-lived server for every experiment (as in deployment): its
    # staging pool, streams and loaded kernels carry over; statistics are
    # reported per experiment as differences
    srv = hulld.Server(cfg)

    def serve(arrivals):
        """Run one experiment; arrivals[k] = start time (s) of scan k."""
        before = srv.stats()
        ids = {}
        t0 = time.perf_counter()

        def client(me):
            # round-robin over this thread's arrived scans, one chunk each
            active = []  # [k, next chunk]
            done = False
            while not done or active:
                try:
                    while True:
                        k = work[me].get_nowait()
                        if k is None:
                            done = True
                            break
                        sp, chunks = scans[k][0], scans[k][1]
                        ids[k] = srv.open_scan(sp.geometry, None, len(chunks))
                        active.append([k, 0])
                except queue.Empty:
                    pass
                if not active:
                    if not done:
                        time.sleep(0.0002)
                    continue
                for item in list(active):
                    k, j = item
                    a, b = scans[k][3][j]
                    srv.submit_rows(ids[k], scans[k][2], int(a), int(b - a))
                    item[1] += 1
                    if item[1] == len(scans[k][1]):
                        active.remove(item)

        nthreads = args.serve_clients
        work = [queue.Queue() for _ in range(nthreads)]
        threads = [threading.Thread(target=client, args=(i,)) for i in range(nthreads)]
        for t in threads:
            t.start()
        for k in np.argsort(arrivals):
            delay = arrivals[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            work[int(k) % nthreads].put(int(k))
        for q in work:
            q.put(None)
        for t in threads:
            t.join()
        infos = []
        for k in range(len(scans)):
            sid = ids[k]
            assert srv.wait(sid, 600_000) == hulld.HD_OK
            infos.append(srv.info(sid))
            srv.close_scan(sid)
        after = srv.stats()
        st = {key: after[key] - before[key] if key != "bytes_in_use" else after[key]
              for key in after}
        return infos, st

    # warm-up: the whole saturated experiment once through the same server,
    # not measured (kernel loading, staging segments, upload streams, and a
    # pooled scan for every volume class, as a long-running server has)
    serve(np.zeros(len(scans)))

    # saturated throughput: every scan at time zero
    infos, st_sat = serve(np.zeros(len(scans)))
    t_start = min(i["t_open"] for i in infos)
    makespan = max(i["t_ready"] for i in infos) - t_start
    X = total / makespan
    mean_h = total / len(scans)
    lam = args.serve_load * X / mean_h
    arrivals = np.cumsum(rng.exponential(1.0 / lam, len(scans)))
    arrivals -= arrivals[0]
    infos, st = serve(arrivals)
    srv.close()
    # one scan at a time through the plain scan calls, the same chunks from
    # the same pinned host memory: each chunk added as it comes, the hulls
    # after the scan's last chunk
    seq_stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    t_seq = time.perf_counter()
    with torch.cuda.stream(seq_stream):
        for sp, chunks, _, _ in scans:
            with hulld.Scan(sp.geometry) as s:
                for c in chunks:
                    s.add(c, seq_stream)
                s.finalize(seq_stream)
                seq_stream.synchronize()
    seq_s = time.perf_counter() - t_seq
    ttl = np.array([i["t_ready"] - i["t_last_chunk"] for i in infos])
    ttf = np.array([i["t_ready"] - i["t_first_chunk"] for i in infos])
    span = max(i["t_ready"] for i in infos) - min(i["t_open"] for i in infos)
    return {"workload": f"{len(scans)} scans from the 48-scan mix, Poisson arrivals at "
                        f"{args.serve_load:g} x saturated throughput, per-angle chunks of "
                        "1e4-1e5 histories from pinned host memory",
            "total_histories": total, "chunks": int(st["chunks_submitted"]),
            "client_threads": args.serve_clients, "load": args.serve_load,
            "p50_ms": float(np.percentile(ttl, 50)) * 1e3,
            "p99_ms": float(np.percentile(ttl, 99)) * 1e3,
            "max_ms": float(ttl.max()) * 1e3,
            "from_first_chunk_ms": {"p50": float(np.percentile(ttf, 50)) * 1e3,
                                    "p99": float(np.percentile(ttf, 99)) * 1e3},
            "histories_per_s": total / span,
            "saturated_histories_per_s": X, "arrival_rate_scans_per_s": lam,
            "sequential_histories_per_s": total / seq_s, "sequential_seconds": seq_s,
            "sequential_what": "one scan at a time, each chunk added from pinned host memory "
                               "through the plain scan calls",
            "saturated_over_sequential": X / (total / seq_s),
            "server": st, "server_saturated": st_sat}


def run_batched(args):
    """The 48-scan mix, batched against one at a time (its own JSON line)."""
    import multiprocessing as mp
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        specs, hosts = mix48(args, pool)
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    sampler = ClockSampler(local)
    sampler.start()
    b = measure_batched(args, specs, hosts, args.steps, args.warmup)
    clocks = sampler.stop()
    line = {"metric": "proton histories/s (48 batched scans, SC+MSC+SM)",
            "value": b["histories_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": b["workload"], "total_histories": b["total_histories"],
                       "tuning": b["tuning"], "grids": b["grids"]},
            "voxel_steps_per_s": b["voxel_steps_per_s"],
            "sequential_48": {"value": b["sequential_histories_per_s"], "unit": UNIT,
                              "ms_per_step": b["sequential_ms"]},
            "batched_over_sequential": b["speedup"], "graph": b["graph"],
            "gpu_launches_per_step": b["gpu_launches_per_step"],
            "gpu_launches": b["gpu_launches_per_step"] * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """The 48-scan mix served (its own JSON line)."""
    import multiprocessing as mp
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        specs, hosts = mix48(args, pool)
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    sv = measure_serving(args, specs[:args.serve_scans], hosts[:args.serve_scans])
    line = {"metric": "served time-to-hull p50 (hull ready - last chunk), 48-scan mix",
            "value": sv["p50_ms"], "unit": "ms", "n_gpus": 1,
            "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": sv["workload"], "total_histories": sv["total_histories"],
                       "chunks": sv["chunks"], "client_threads": sv["client_threads"]},
            "time_to_hull_ms": {"p50": sv["p50_ms"], "p99": sv["p99_ms"], "max": sv["max_ms"]},
            "time_from_first_chunk_ms": sv["from_first_chunk_ms"],
            "served_histories_per_s": sv["histories_per_s"],
            "saturated_histories_per_s": sv["saturated_histories_per_s"],
            "arrival_rate_scans_per_s": sv["arrival_rate_scans_per_s"],
            "sequential_streamed": {"histories_per_s": sv["sequential_histories_per_s"],
                                    "seconds": sv["sequential_seconds"],
                                    "what": sv["sequential_what"]},
            "saturated_over_sequential": sv["saturated_over_sequential"],
            "server": sv["server"], "server_saturated": sv["server_saturated"]}
    print(json.dumps(line), flush=True)


def run_rows(args):
    """Hull-restricted system-matrix rows of the head-sized scan: the scan
    (SC+MSC+SM) is built once, then each step emits the CSR rows of all 9e6
    histories inside its MSC hull through the C ABI (count, offsets, emit,
    and the read of the total)."""
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld, synth
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    w = synth.make_config(2, fraction=args.fraction)
    g, h = w.geometry, w.histories
    n = len(h)
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    scan = hulld.Scan(g)
    scan.add(dev)
    scan.finalize()
    torch.cuda.synchronize()
    row_ptr, cols = scan.system_rows(hulld.HD_MSC, dev)
    nnz = len(cols)
    stream = torch.cuda.Stream()

    def step():
        hulld.hd_scan_system_rows(scan.handle, hulld.HD_MSC, *dev[:5], row_ptr, cols, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    peaks = _peaks()
    out_bytes = 4.0 * nnz + 8.0 * (n + 1)
    line = {"metric": "histories/s (hull-restricted system-matrix rows, MSC hull)",
            "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; rows of every history inside the MSC hull",
                       "histories": n, "nnz": nnz,
                       "hull_voxels": int(scan.mask(hulld.HD_MSC).sum())},
            "nnz_per_s": nnz / (ms * 1e-3),
            "output": {"bytes_per_step": out_bytes,
                       "gbs": out_bytes / (ms * 1e-3) / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"]},
            "gpu_launches": 5 * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    scan.close()


def run_binned(args):
    """SC as the paper ran it on the head-sized scan: each step bins all 9e6
    histories, applies the 3 sigma cuts, carves the missed bins' lines and
    filters (hd_binned_run: statistics, cuts, bin decisions, carve, filter),
    inputs resident in HBM (216 MB, read twice, larger than L2).  e2e: the
    same with the inputs copied from page-locked host memory and the hull
    read back every step."""
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld, synth
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    w = synth.make_config(2, fraction=args.fraction)
    g, h = w.geometry, w.histories
    n = len(h)
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    b = hulld.Binned(g)
    stream = torch.cuda.Stream()

    def step():
        hulld.hd_binned_run(b.handle, *dev, stream=stream)

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        ms = timed(step, args.steps)
        clocks = sampler.stop()
        st = b.stats()
        # phases, each timed alone over the same resident inputs
        hulld.hd_binned_reset(b.handle, stream)
        t_stats = timed(lambda: hulld.hd_binned_add_histories(b.handle, *dev, stream=stream),
                        1)
        t_cut = timed(lambda: hulld.hd_binned_cut_histories(b.handle, *dev, stream=stream), 1)
        t_fin = timed(lambda: hulld.hd_binned_finalize(b.handle, stream), 3)
        e2e = None
        if not args.no_e2e:
            host = [torch.from_numpy(a).pin_memory() for a in h.arrays()]
            out = torch.empty(g.nx * g.ny * g.nz, dtype=torch.uint8).pin_memory()

            def e2e_step():
                for d, hh in zip(dev, host):
                    d.copy_(hh, non_blocking=True)
                hulld.hd_binned_run(b.handle, *dev, stream=stream)
                hulld.hd_binned_get_image(b.handle, hulld.HD_BINNED_HULL, out, stream)
            for _ in range(args.warmup):
                e2e_step()
            torch.cuda.synchronize()
            ms_e2e = timed(e2e_step, args.steps)
            e2e = {"value": n / (ms_e2e * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": int(out.numel())}
    peaks = _peaks()
    atomics = 7 * st["histories_binned"] + 2 * (st["histories_binned"] - st["histories_cut"])
    l2_rate = hulld.hd_probe_atomics(hulld.HD_PROBE_L2_RANDOM)
    stats_atomics = 7 * st["histories_binned"]
    line = {"metric": "histories/s (SC with binning, data cuts and filter, as the paper ran it)",
            "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; binned SC (4 deg x 1 mm x 5 mm bins)",
                       "histories": n, "bins": st["bins"], "l2": "inputs larger than L2"},
            "stats": st,
            "phases_ms": {"statistics": t_stats, "cuts": t_cut, "carve_and_filter": t_fin},
            "atomic_rate": {"atomics_per_step": atomics,
                            "per_s": atomics / ((t_stats + t_cut) * 1e-3)},
            "roofline": {"bound": "l2_atomic", "kernel": "binned_stats_kernel",
                         "achieved": stats_atomics / (t_stats * 1e-3), "peak": l2_rate,
                         "unit": "atomics/s", "frac": stats_atomics / (t_stats * 1e-3) / l2_rate,
                         "atomics_per_launch": stats_atomics,
                         "peak_source": "hd_probe_atomics L2 random (measured in this run)"},
            "input": {"bytes_per_step": 2 * 24 * n,
                      "gbs": 2 * 24 * n / ((t_stats + t_cut) * 1e-3) / 1e9,
                      "hbm_peak_gbs": peaks["hbm_gbs"]},
            "e2e": e2e, "gpu_launches": 5 * args.steps, "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        import time as _time
        sub = synth.make_config(2, fraction=0.05)
        bp = oracle.binned_params_for(g)
        t0 = _time.perf_counter()
        oracle.sc_binned(g, sub.histories, bp)
        dt = _time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sub.histories) / dt, "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(sub.histories)} histories (5% per angle)"}
    print(json.dumps(line), flush=True)
    b.close()


def run_thick(args):
    """Thick rays on the head-sized scan: each step adds the missed and hit
    counts of all 9e6 histories with A_i dilated by k voxels in-plane
    (hd_accumulate_thick: clear the difference arrays, walk, prefix sums)."""
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld, synth
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    w = synth.make_config(2, fraction=args.fraction)
    g, h = w.geometry, w.histories
    n = len(h)
    k = args.thick_k
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    V = g.nx * g.ny * g.nz
    N = torch.zeros(V, dtype=torch.int32, device="cuda")
    M = torch.zeros(V, dtype=torch.int32, device="cuda")
    ws = torch.empty(hulld.hd_accumulate_thick_workspace(g), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()

    counter = torch.zeros(1, dtype=torch.int64, device="cuda")

    def step():
        hulld.hd_accumulate_thick(g, None, k, dev, N, M, ws, stream, counter)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        N.zero_()
        M.zero_()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    voxels = (int(N.sum().item()) + int(M.sum().item())) // args.steps
    atomics = 2 * int(counter.item())
    peaks = _peaks()
    l2_rate = hulld.hd_probe_atomics(hulld.HD_PROBE_L2_RANDOM)
    # the whole method on thick sets: a scan set to thick rays (SC, MSC, SM,
    # the tiled thick traversal on this grid), reset, add and finalize per step
    scan = hulld.Scan(g)
    scan.set_thick(k)

    def scan_step():
        hulld.hd_scan_reset(scan.handle, stream)
        hulld.hd_scan_add_histories(scan.handle, *dev, stream=stream)
        hulld.hd_scan_finalize(scan.handle, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            scan_step()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            scan_step()
        f1.record(stream)
        torch.cuda.synchronize()
        clocks_scan = sampler.stop()
    ms_scan = f0.elapsed_time(f1) / args.steps
    scan_stats = scan.stats()
    scan.close()
    line = {"metric": f"histories/s (SC+MSC+SM on thick rays, k = {k} voxels in-plane)",
            "value": n / (ms_scan * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_scan, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD + f"; thick rays k = {k}", "histories": n,
                       "fraction": args.fraction,
                       "step": "a scan set to thick rays (hd_scan_set_thick): reset, add, "
                               "finalize; the tiled thick traversal on this grid"},
            "thick_voxels_per_s": (scan_stats["steps_miss"] + scan_stats["steps_hit"])
            / (ms_scan * 1e-3),
            "standalone": {"what": "hd_accumulate_thick (counts only; a lane per history "
                                   "over the whole grid)",
                           "ms_per_step": ms, "histories_per_s": n / (ms * 1e-3),
                           "thick_voxels_per_s": voxels / (ms * 1e-3),
                           "roofline": {"bound": "l2_atomic", "kernel": "thick_kernel",
                                        "achieved": atomics / (ms * 1e-3), "peak": l2_rate,
                                        "unit": "atomics/s",
                                        "frac": atomics / (ms * 1e-3) / l2_rate,
                                        "atomics_per_step": atomics,
                                        "peak_source": "hd_probe_atomics L2 random "
                                                       "(measured in this run)",
                                        "hbm_peak_gbs": peaks["hbm_gbs"]}},
            "gpu_launches": 12 * args.steps, "clocks": clocks_scan,
            "clocks_standalone": clocks}
    if not args.no_cpu_baseline:
        import oracle
        import time as _time
        sub = synth.make_config(2, fraction=0.005)
        t0 = _time.perf_counter()
        oracle.accumulate_thick(g, sub.histories, k)
        dt = _time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sub.histories) / dt, "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(sub.histories)} histories (0.5% per angle)"}
    print(json.dumps(line), flush=True)


def run_euclid(args):
    """Thick rays by Euclidean distance on the head-sized scan: each step adds
    the missed and hit counts of all 9e6 histories with A_i(d_0) = the voxels
    whose centre lies within d_0 mm of the path (hd_accumulate_euclid: clear,
    rows of every capsule, prefix sums); then a scan set to the same distance
    (reset, add, finalize of SC, MSC and SM)."""
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld, synth
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    w = synth.make_config(2, fraction=args.fraction)
    g, h = w.geometry, w.histories
    n = len(h)
    d0 = args.thick_mm
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    V = g.nx * g.ny * g.nz
    N = torch.zeros(V, dtype=torch.int32, device="cuda")
    M = torch.zeros(V, dtype=torch.int32, device="cuda")
    ws = torch.empty(hulld.hd_accumulate_thick_workspace(g), dtype=torch.uint8, device="cuda")
    rows = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    def step():
        hulld.hd_accumulate_euclid(g, None, d0, dev, N, M, ws, stream, rows)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        N.zero_()
        M.zero_()
        sampler = ClockSampler(local)
        sampler.start()
        ms = timed(step, args.steps)
        clocks = sampler.stop()
    voxels = (int(N.sum().item()) + int(M.sum().item())) // args.steps
    n_rows = int(rows.item())
    scan = hulld.Scan(g)
    scan.set_thick_distance(d0)

    def scan_step():
        hulld.hd_scan_reset(scan.handle, stream)
        hulld.hd_scan_add_histories(scan.handle, *dev, stream=stream)
        hulld.hd_scan_finalize(scan.handle, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            scan_step()
        torch.cuda.synchronize()
        ms_scan = timed(scan_step, args.steps)
    scan.close()
    line = {"metric": f"histories/s (SC+MSC+SM on Euclidean thick rays, d_0 = {d0:g} mm)",
            "value": n / (ms_scan * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_scan, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/int128",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + f"; voxel centres within {d0:g} mm of each path",
                       "histories": n, "fraction": args.fraction,
                       "step": "a scan set to the distance (hd_scan_set_thick_distance): "
                               "reset, add, finalize"},
            "standalone": {"what": "hd_accumulate_euclid (counts only)", "ms_per_step": ms,
                           "histories_per_s": n / (ms * 1e-3),
                           "thick_voxels_per_s": voxels / (ms * 1e-3),
                           "rows_per_s": n_rows / (ms * 1e-3), "rows_per_step": n_rows,
                           "voxels_per_row": voxels / n_rows if n_rows else None},
            "gpu_launches": 4 * args.steps, "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        import time as _time
        sub = synth.make_config(2, fraction=0.0005)
        t0 = _time.perf_counter()
        oracle.accumulate_euclid(g, sub.histories, d0)
        dt = _time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sub.histories) / dt, "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(sub.histories)} histories (50 per angle)"}
    print(json.dumps(line), flush=True)


def run_diagnostics(args):
    """Extra and missing voxels of every hull against the synthetic object
    (the measures of Tables 1-2) on the head-sized scan, all computed on the
    GPU: SC, MSC (Eq. 3.6 literal and its enclosed part), SM (the slope
    picker of Alg. 3 and the documented edge-detection picker) and SC as the
    paper ran it; plus the device time of the diagnostic operations."""
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld, synth
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    w = synth.make_config(2, fraction=args.fraction)
    g, h = w.geometry, w.histories
    dims = (g.nx, g.ny, g.nz)
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    obj = torch.from_numpy(synth.object_mask(g, w.phantom)).cuda()
    scan = hulld.Scan(g)
    scan.add(dev)
    scan.finalize()
    hulls = {}
    for name, m in (("SC", hulld.HD_SC), ("MSC", hulld.HD_MSC), ("SM", hulld.HD_SM)):
        hulls[name] = torch.from_numpy(scan.mask(m)).cuda()
    Mvol = torch.from_numpy(scan.counts(hulld.HD_SM).view(np.int32)).cuda()
    stream = torch.cuda.Stream()
    ws = torch.empty(hulld.hd_sm_canny_workspace(dims), dtype=torch.uint8, device="cuda")
    b = hulld.Binned(g)

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    out = {}
    fill = torch.empty_like(hulls["MSC"])
    out["fill_enclosed_ms"] = timed(lambda: hulld.hd_fill_enclosed(hulls["MSC"], dims, fill,
                                                                   stream), args.steps)
    hulls["MSC enclosed"] = fill
    res = {}
    for q in (0, 25, 50):
        holder = {}

        def canny():
            holder["r"] = hulld.hd_sm_canny(Mvol, dims, q, ws, stream)
        t = timed(canny, args.steps)
        if q == 50:
            out["sm_canny_ms"] = t
        res[q] = holder["r"]
        hulls[f"SM edge q={q}"] = holder["r"][2]
    with torch.cuda.stream(stream):
        b.run(dev, stream)
    torch.cuda.synchronize()
    hulls["SC binned"] = torch.from_numpy(b.image(hulld.HD_BINNED_HULL)).cuda()
    counts = torch.empty(2 * g.nz + 2, dtype=torch.int64, device="cuda")
    out["hull_compare_ms"] = timed(lambda: hulld.hd_hull_compare(hulls["SC"], obj, dims, counts,
                                                                 stream), args.steps)
    table = {}
    for name, hm in hulls.items():
        c = hulld.hd_hull_compare(hm, obj, dims).cpu().numpy()
        table[name] = {"hull": int(hm.sum().item()), "extra": int(c[2 * g.nz]),
                       "missing": int(c[2 * g.nz + 1])}
    line = {"metric": "extra/missing voxels against the synthetic object (Tables 1-2 measures)",
            "config": {"workload": WORKLOAD, "fraction": args.fraction,
                       "object_voxels": int(obj.sum().item())},
            "hulls": table, "device_ms": out, "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(line), flush=True)
    b.close()
    scan.close()


def run_configs(args):
    """Per-configuration figures beside the head-sized benchmark: the tiny
    scan (64x64x8 voxels, 1.8e5 histories) and the large streamed scan
    (400x400x128 voxels, 9.9e7 histories added in 180 per-angle chunks from
    device memory) timed on the GPU, and the oracle as it stands, on one
    host thread and on all of them, on bounded samples of the tiny, the
    head-sized and the large scan."""
    import multiprocessing as mp
    import numpy as _np
    # the large scan's chunks are generated by a spawn pool started before
    # any CUDA call, and collected before the first timed region
    pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
    from paper_1402_1720_gb300 import synth
    chunks_job = pool.map_async(synth.config3_chunk, range(180))
    import torch
    import oracle
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    oracle.build()
    cores = os.cpu_count() or 1
    chunks = chunks_job.get()
    pool.close()
    pool.join()

    def gpu_ms(g, parts, steps, warmup):
        devs = [[torch.from_numpy(a).cuda() for a in p.arrays()] for p in parts]
        stream = torch.cuda.current_stream()
        with hulld.Scan(g) as s:
            def step():
                s.reset()
                for d in devs:
                    s.add(d)
                s.finalize()
            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            st = s.stats()
        return e0.elapsed_time(e1) / steps, st

    def oracle_rate(g, h, every, threads):
        sub = h.take(_np.arange(0, len(h), every))
        t0 = time.perf_counter()
        oracle.run(g, sub, threads=threads)
        dt = time.perf_counter() - t0
        return {"histories_per_s": len(sub) / dt, "threads": threads,
                "sample": f"{len(sub)} histories (every {every}th), {dt:.1f} s wall"}

    out = {}
    w1 = synth.make_config(1)
    ms1, st1 = gpu_ms(w1.geometry, [w1.histories], args.steps, args.warmup)
    out["tiny 64x64x8, 1.8e5 histories"] = {
        "gpu_ms_per_scan": ms1, "gpu_histories_per_s": len(w1.histories) / (ms1 * 1e-3),
        "oracle_1_thread": oracle_rate(w1.geometry, w1.histories, 4, 1),
        "oracle_all_threads": oracle_rate(w1.geometry, w1.histories, 1, cores)}
    w2 = synth.make_config(2)
    out["head 200x200x32, 9e6 histories"] = {
        "oracle_1_thread": oracle_rate(w2.geometry, w2.histories, 400, 1),
        "oracle_all_threads": oracle_rate(w2.geometry, w2.histories, 25, cores)}
    g3 = synth.geometry_for(3)
    ms3, st3 = gpu_ms(g3, chunks, 3, 1)
    n3 = sum(len(c) for c in chunks)
    big = synth.Histories.concat(chunks[::45])
    out["large 400x400x128, 9.9e7 histories in 180 chunks"] = {
        "gpu_ms_per_scan": ms3, "gpu_histories_per_s": n3 / (ms3 * 1e-3),
        "gpu_voxel_steps_per_s": (st3["steps_miss"] + st3["steps_hit"]) / (ms3 * 1e-3),
        "oracle_1_thread": oracle_rate(g3, big, 200, 1),
        "oracle_all_threads": oracle_rate(g3, big, 10, cores)}
    line = {"metric": "per-configuration throughput (GPU and the oracle as it stands)",
            "unit": UNIT, "host_cores": cores, "configs": out,
            "data": "synthetic", "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(line), flush=True)


def run_large(args):
    """The large streamed scan alone (400x400x128 voxels of 0.5x0.5x1.25 mm,
    9.9e7 histories added in 180 per-angle chunks from device memory, one add
    per chunk): reset, the adds and finalize per step, timed on the GPU, with
    the traversal's voxel-steps per second against the random-address
    shared-memory atomic rate hd_probe_atomics measures in the same run."""
    import multiprocessing as mp
    # the chunks come from a spawn pool started before any CUDA call
    pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
    from paper_1402_1720_gb300 import synth
    chunks = pool.map(synth.config3_chunk, range(180))
    pool.close()
    pool.join()
    import torch
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld
    _, _, local = _dist()
    torch.cuda.set_device(local)
    hbuild.build()
    hulld.load()
    g3 = synth.geometry_for(3)
    devs = [[torch.from_numpy(a).cuda() for a in p.arrays()] for p in chunks]
    n = sum(len(c) for c in chunks)
    stream = torch.cuda.current_stream()
    with hulld.Scan(g3) as s:
        def step():
            s.reset()
            for d in devs:
                s.add(d)
            s.finalize()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        st = s.stats()
    ms = e0.elapsed_time(e1) / args.steps
    steps_per_scan = (st["steps_miss"] + st["steps_hit"])
    smem_rate = hulld.hd_probe_atomics(hulld.HD_PROBE_SMEM_RANDOM)
    line = {"metric": "histories/s (large streamed scan, SC+MSC+SM)", "value": n / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/int64", "data": "synthetic",
            "config": {"workload": "large 400x400x128 voxels 0.5x0.5x1.25 mm, 9.9e7 float32 "
                                   "histories added in 180 per-angle chunks from device memory",
                       "histories": n, "chunks": len(chunks)},
            "voxel_steps_per_scan": steps_per_scan,
            "voxel_steps_per_s": steps_per_scan / (ms * 1e-3),
            "smem_atomic_rate": smem_rate,
            "gpu_launches": 6 * len(chunks) * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hulld", choices=["hulld", "reference"])
    ap.add_argument("--ref-fraction", type=float, default=0.004)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-method", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="head-200",
                    choices=["head-200", "batched-48", "serving", "rows", "binned",
                             "diagnostics", "thick", "euclid", "configs", "large"])
    ap.add_argument("--batch-fraction", type=float, default=1.0)
    ap.add_argument("--fraction", type=float, default=1.0,
                    help="head-200 workload: keep this fraction of the histories "
                         "(small profiling captures; 1.0 for the benchmark)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--thick-k", type=int, default=2,
                    help="thick workload: in-plane dilation in voxels")
    ap.add_argument("--thick-mm", type=float, default=2.5,
                    help="euclid workload: distance d_0 from voxel centres to the path, mm")
    ap.add_argument("--serve-scans", type=int, default=48)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-clients", type=int, default=8)
    ap.add_argument("--no-mix", action="store_true",
                    help="head-200 workload: skip the batched and served 48-scan sections")
    ap.add_argument("--mix-steps", type=int, default=5,
                    help="head-200 workload: timed batched steps of the 48-scan section")
    args = ap.parse_args()

    if args.workload == "configs":
        run_configs(args)
        return
    if args.workload == "large":
        run_large(args)
        return
    if args.workload == "batched-48":
        run_batched(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "rows":
        run_rows(args)
        return
    if args.workload == "binned":
        run_binned(args)
        return
    if args.workload == "diagnostics":
        run_diagnostics(args)
        return
    if args.workload == "thick":
        run_thick(args)
        return
    if args.workload == "euclid":
        run_euclid(args)
        return

    if args.impl == "reference":
        run_reference(args)
        return

    # the 48-scan mix for the batched and served sections, generated on the
    # host cores by spawned processes while the GPU measures the head scan
    ws0, _, _ = _dist()
    mix_pool = mix_job = None
    if ws0 == 1 and not args.no_mix:
        import multiprocessing as mp
        from paper_1402_1720_gb300 import synth as _synth
        mix_pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
        jobs = [(k, a, min(90, a + 10), args.batch_fraction) for k in range(48)
                for a in range(0, 90, 10)]
        mix_job = (jobs, mix_pool.map_async(_synth.batch_scan_part, jobs))

    import torch
    import torch.distributed as dist
    from paper_1402_1720_gb300 import build as hbuild
    from paper_1402_1720_gb300 import hulld, synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hbuild.build()
    hulld.load()

    w = synth.make_config(2, fraction=args.fraction) if args.fraction < 1.0 else synth.make_config(2)
    g, h = w.geometry, w.histories
    n = len(h)
    dev = [torch.from_numpy(a).cuda() for a in h.arrays()]
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def timed(scan, steps, warmup, profile=False, sampler=None):
        for _ in range(warmup):
            scan.reset()
            scan.add(dev)
            scan.finalize()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if profile:
            scan.set_profiling(True)
        l0 = scan.profile()["kernel_launches"]
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            scan.reset()
            scan.add(dev)
            scan.finalize()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1) / steps
        prof = scan.profile()
        if profile:
            scan.set_profiling(False)
        return ms, prof, prof["kernel_launches"] - l0, clocks

    # the mix's generation ends before any timed region, so that no host
    # core is busy with it while kernels are launched and timed
    mix_parts = None
    if mix_job is not None:
        mix_parts = mix_job[1].get()
        mix_pool.close()
        mix_pool.join()

    # ---- main measurement: all three methods
    scan = hulld.Scan(g)
    sampler = ClockSampler(local)
    ms, prof, launches, clocks = timed(scan, args.steps, args.warmup, profile=True,
                                       sampler=sampler)
    ms = max_over_ranks(ms)
    st = scan.stats()
    steps_per_scan = st["steps_miss"] + st["steps_hit"]
    value = ws * n / (ms * 1e-3)

    # roofline of the dominant kernel (the traversal).  Its algorithmic work
    # is one counter update per voxel-step (the oracle's exact sum |A_i|;
    # one launch covers the whole scan), and the ceiling of a design that
    # privatises the counts in shared memory is the random-address
    # shared-memory atomic rate, measured here by the same process.
    peaks = _peaks()
    trace_ms = prof["ms_trace"] / max(1, prof["trace_launches"])
    runs = st.get("runs", 0)
    probes = {name: hulld.hd_probe_atomics(kind) for name, kind in
              [("smem_random", hulld.HD_PROBE_SMEM_RANDOM),
               ("smem_coherent", hulld.HD_PROBE_SMEM_COHERENT),
               ("l2_random", hulld.HD_PROBE_L2_RANDOM),
               ("hbm_random", hulld.HD_PROBE_HBM_RANDOM)]}
    vsteps = steps_per_scan / (trace_ms * 1e-3)
    traffic, traffic_note = _profiled_traffic()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = {"bound": "smem_atomic", "achieved": vsteps, "peak": probes["smem_random"],
                "unit": "atomics/s", "frac": vsteps / probes["smem_random"],
                "traffic": traffic, "traffic_source": traffic_note,
                "kernel": "trace_tiles_kernel", "kernel_ms": trace_ms,
                "voxel_steps_per_launch": steps_per_scan,
                "work_per_unit": "one counter update per voxel-step (sum |A_i| of the scan)",
                "peak_source": "hd_probe_atomics shared-memory random-address rate, measured "
                               "in this run (1024-thread blocks, xorshift addresses, best of 3)",
                "sm_count": sms}
    fields, _ = _profile_fields()
    if fields and "executed thread instructions per voxel-step" in fields:
        roofline["executed_thread_instructions_per_voxel_step"] = float(
            fields["executed thread instructions per voxel-step"])
    atomic_roofline = {
        "ceilings_atomics_per_s": probes,
        "voxel_steps_per_s": vsteps,
        "voxel_steps_over_l2_random_ceiling": vsteps / probes["l2_random"],
        "runs_per_scan": runs,
        "voxels_per_run": steps_per_scan / runs if runs else None,
        "trace_smem_atomics_per_s": 2.0 * runs / (trace_ms * 1e-3),
        "trace_smem_atomics_over_smem_random_ceiling":
            2.0 * runs / (trace_ms * 1e-3) / probes["smem_random"]}

    # prepare = ingest + plan + scatter (everything before the traversal)
    phases = {"prepare_ms": prof["ms_ingest"] / args.steps, "trace_ms": trace_ms,
              "trace_global_ms": prof["ms_trace_global"] / args.steps,
              "finalize_ms": prof["ms_finalize"] / args.steps}
    # input bytes (24 per history) over the prepare phase, against the HBM copy peak
    phases["prepare_input_gbs"] = 24.0 * n / (phases["prepare_ms"] * 1e-3) / 1e9
    phases["hbm_peak_gbs"] = peaks["hbm_gbs"]

    # ---- per method
    per_method = {}
    if not args.no_per_method:
        for name, m in [("sc", hulld.HD_SC), ("msc", hulld.HD_MSC), ("sm", hulld.HD_SM)]:
            p = hulld.hd_params_default()
            p.methods = m
            s2 = hulld.Scan(g, p)
            k = max(3, args.steps // 2)
            mms, _, _, _ = timed(s2, k, 3)
            mms = max_over_ranks(mms)
            sst = s2.stats()
            per_method[name] = {"histories_per_s": ws * n / (mms * 1e-3),
                                "voxel_steps_per_s": ws * (sst["steps_miss"] + sst["steps_hit"]) /
                                (mms * 1e-3), "ms_per_step": mms}
            s2.close()

    # ---- end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        host = [torch.from_numpy(a).pin_memory() for a in h.arrays()]
        masks = [torch.empty(g.n_voxels, dtype=torch.uint8).pin_memory() for _ in range(3)]
        s3 = hulld.Scan(g)

        def e2e_step():
            s3.reset()
            s3.add(host)
            s3.finalize()
            for mk, meth in zip(masks, (hulld.HD_SC, hulld.HD_MSC, hulld.HD_SM)):
                hulld.hd_scan_get_mask(s3.handle, meth, hulld.HD_MASK_U8, mk)
            stream.synchronize()

        for _ in range(max(3, args.warmup)):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        k = max(3, args.steps // 2)
        for _ in range(k):
            e2e_step()
        dt = max_over_ranks((time.perf_counter() - t0) / k)
        e2e = {"value": ws * n / dt, "unit": UNIT, "h2d_bytes_per_step": 24 * n,
               "d2h_bytes_per_step": 3 * g.n_voxels, "ms_per_step": dt * 1e3}
        s3.close()

    # ---- the 48-scan mix: batched (one persistent launch, graph replay)
    # against one scan at a time, and served (Poisson arrivals of streamed
    # scans) with its time-to-hull percentiles
    batched = serving = None
    if mix_job is not None:
        jobs, parts = mix_job[0], mix_parts
        from paper_1402_1720_gb300 import synth as _synth
        specs = _synth.batch_scan_specs(48, fraction=args.batch_fraction)
        hosts = [_synth.Histories.concat([p for j, p in zip(jobs, parts) if j[0] == k])
                 for k in range(48)]
        del parts, mix_parts
        b = measure_batched(args, specs, hosts, args.mix_steps, 2)
        batched = {k: b[k] for k in ("workload", "total_histories", "steps", "ms",
                                     "histories_per_s", "sequential_ms",
                                     "sequential_histories_per_s", "speedup",
                                     "gpu_launches_per_step", "tuning")}
        batched["graph_replays"] = b["graph"]["graph_replays"]
        sv = measure_serving(args, specs, hosts)
        serving = {k: sv[k] for k in ("workload", "total_histories", "chunks", "load",
                                      "client_threads", "p50_ms", "p99_ms", "max_ms",
                                      "histories_per_s", "saturated_histories_per_s",
                                      "sequential_histories_per_s",
                                      "saturated_over_sequential")}
        serving["server_launches"] = sv["server"]["launches"]
        del hosts

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "methods": "SC+MSC+SM",
                           "histories": n, "fraction": args.fraction,
                           "inputs": f"{n:.3g} x 24 B = {n * 24 / 1e6:.0f} MB resident in HBM"
                                     + (", larger than L2" if n * 24 > 129e6 else ""),
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
                "voxel_steps_per_s": ws * steps_per_scan / (ms * 1e-3),
                "voxel_steps_per_scan": steps_per_scan,
                "per_method": per_method, "phases": phases,
                "roofline": roofline, "atomic_roofline": atomic_roofline,
                "cpu_baseline": cpu, "e2e": e2e,
                "batched": batched, "serving": serving,
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    scan.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
