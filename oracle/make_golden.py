"""Full-size expected values for the GPU parity tests (test infrastructure).

Runs the CPU oracle over the head-sized scan (200x200x32 voxels, 9e6
histories), the large streamed scan (400x400x128 voxels, 180 per-angle
chunks of 550 000 histories), the 48 scans of the batched/served mix
(grids 64x64x16, 128x128x32, 256x256x64; 2e5-2e7 histories each) and, on
request, the head-sized scan with Euclidean thick rays at d_0 = 2.5 mm
and 0.5 mm (euclid200, euclid200_d05) and with in-plane thick rays at k = 2 (thick200), and the
system-matrix rows of the head-sized scan inside its MSC hull (rows200),
and writes to tests/golden/ what the GPU tests compare against:

* the SHA-256 of the generated inputs (the whole scan, every chunk or every
  scan), so a test first checks that it fed the GPU the same histories;
* the SHA-256 of each output array: N and M (uint32, Eq. 3.4 and 3.9),
  H_1, H_2, H_3 (uint8, Eq. 3.3, 3.6, 3.10), and the per-slice SM threshold
  M_t, its steepest drop and its voxel index (Alg. 3);
* per slice, the SHA-256 and the sum of N and of M, so that a mismatch can
  be located;
* the oracle's statistics: histories in, missed, hit, unused, rejected, and
  the voxel memberships sum |A_i| of each class.

Only `oracle` and the seeded input generator are called; nothing here reads
or runs the CUDA library.

    python oracle/make_golden.py [head200] [head400] [batch48] [euclid200] [euclid200_d05]
                                 [thick200] [rows200] [--threads N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1402_1720_gb300 import synth  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")


def sha(arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def output_record(g, res) -> dict:
    """Hashes, per-slice hashes and sums, and statistics of one oracle result."""
    plane = g.nx * g.ny
    arrays = {"N": np.asarray(res["N"], np.uint32), "M": np.asarray(res["M"], np.uint32),
              "H1": np.asarray(res["H1"], np.uint8), "H2": np.asarray(res["H2"], np.uint8),
              "H3": np.asarray(res["H3"], np.uint8), "Mt": np.asarray(res["Mt"], np.uint32),
              "slope": np.asarray(res["slope"], np.uint32),
              "index": np.asarray(res["index"], np.int64)}
    rec = {"sha256": {k: sha([v]) for k, v in arrays.items()},
           "slices": {}, "stats": dict(res["stats"]),
           "hull_voxels": {k: int(arrays[k].sum(dtype=np.int64)) for k in ("H1", "H2", "H3")}}
    for k in ("N", "M"):
        a = arrays[k].reshape(g.nz, plane)
        rec["slices"][k] = {"sha256": [sha([a[z]])[:16] for z in range(g.nz)],
                            "sum": [int(a[z].sum(dtype=np.int64)) for z in range(g.nz)]}
    return rec


def geometry_record(g) -> dict:
    return {"nx": g.nx, "ny": g.ny, "nz": g.nz, "sx": g.sx, "sy": g.sy, "sz": g.sz, "T": g.T}


def decisions(g, acc) -> dict:
    """H_1, H_2 and the SM threshold and hull from accumulated counts."""
    dims = (g.nx, g.ny, g.nz)
    out = dict(acc)
    out["H1"] = oracle.sc_from_counts(acc["N"])
    out["H2"] = oracle.msc_decide(acc["N"], dims)
    out.update(oracle.sm_decide(acc["M"], dims))
    return out


# ------------------------------------------------------------- generators
def _c3_chunk(k):
    return synth.config3_chunk(k)



# -------------------------------------------------------------- workloads
def head200(threads: int) -> dict:
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    res = oracle.run(g, h, threads=threads)
    return {"workload": "head-200x200x32, 90 angles x 100000 histories (config 2)",
            "geometry": geometry_record(g), "histories": len(h),
            "inputs_sha256": sha(h.arrays()), **output_record(g, res)}


def euclid200(threads: int, d0: float = 2.5) -> dict:
    """The head-sized scan with A_i the Euclidean thick set A_i(d_0) (Eq.
    3.2, d the distance from a voxel's centre to the closed segment), the
    hulls decided from its counts."""
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    res = oracle.run_euclid(g, h, d0, threads=threads)
    s = [int(x) for x in res["stats"]]
    res["stats"] = {"n_in": s[0], "n_miss": s[1], "n_hit": s[2], "n_none": s[3],
                    "n_reject": s[4], "steps_miss": s[5], "steps_hit": s[6]}
    return {"workload": "head-200x200x32, 90 angles x 100000 histories (config 2), Euclidean "
                        f"thick rays, d_0 = {d0:g} mm",
            "d0_mm": d0, "geometry": geometry_record(g), "histories": len(h),
            "inputs_sha256": sha(h.arrays()), **output_record(g, res)}


def thick200(threads: int) -> dict:
    """The head-sized scan with A_i the in-plane Chebyshev thick set A_i(k),
    k = 2 voxels (reading 13a of Eq. 3.2 with d_0 > 0), the hulls decided
    from its counts (the oracle's thick accumulation runs on one thread)."""
    del threads
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    k = 2
    res = oracle.run_thick(g, h, k)
    s = [int(x) for x in res["stats"]]
    res["stats"] = {"n_in": s[0], "n_miss": s[1], "n_hit": s[2], "n_none": s[3],
                    "n_reject": s[4], "steps_miss": s[5], "steps_hit": s[6]}
    return {"workload": "head-200x200x32, 90 angles x 100000 histories (config 2), in-plane "
                        "thick rays, k = 2",
            "k": k, "geometry": geometry_record(g), "histories": len(h),
            "inputs_sha256": sha(h.arrays()), **output_record(g, res)}


def rows200(threads: int) -> dict:
    """The rows of the hull-restricted system matrix of every history of the
    head-sized scan inside its MSC hull (the hull the oracle decides), in
    path order; hashes of the row offsets and of the column indices, the
    latter also per block of 2^20 histories so that a mismatch can be
    located."""
    w = synth.make_config(2)
    g, h = w.geometry, w.histories
    res = oracle.run(g, h, threads=threads)
    hull = np.asarray(res["H2"], np.uint8)
    ptr, cols = oracle.system_rows(g, h, hull, threads=threads)
    ptr = np.asarray(ptr, np.int64)
    cols = np.asarray(cols, np.int32)
    block = 1 << 20
    blocks = [sha([cols[ptr[b]:ptr[min(b + block, len(h))]]])[:16]
              for b in range(0, len(h), block)]
    return {"workload": "head-200x200x32, 90 angles x 100000 histories (config 2): system-matrix "
                        "rows inside the MSC hull",
            "geometry": geometry_record(g), "histories": len(h),
            "inputs_sha256": sha(h.arrays()), "hull_sha256": sha([hull]),
            "nnz": int(len(cols)), "row_ptr_sha256": sha([ptr]), "cols_sha256": sha([cols]),
            "cols_block_histories": block, "cols_block_sha256": blocks}


def head400(threads: int, pool) -> dict:
    g = synth.geometry_for(3)
    V = g.nx * g.ny * g.nz
    N = np.zeros(V, np.uint32)
    M = np.zeros(V, np.uint32)
    stats = None
    chunk_sha = []
    n = 0
    for chunk in pool.imap(_c3_chunk, range(180)):
        chunk_sha.append(sha(chunk.arrays()))
        acc = oracle.accumulate_parallel(g, chunk, threads=threads, want_h1=False)
        N += acc["N"]
        M += acc["M"]
        stats = acc["stats"] if stats is None else {k: stats[k] + acc["stats"][k] for k in stats}
        n += len(chunk)
    res = decisions(g, {"N": N, "M": M, "stats": stats})
    return {"workload": "head-400x400x128, 180 per-angle chunks x 550000 histories (config 3)",
            "geometry": geometry_record(g), "histories": n, "chunks_sha256": chunk_sha,
            **output_record(g, res)}


def batch48(threads: int, pool) -> dict:
    specs = synth.batch_scan_specs(48)
    scans = []
    for k, sp in enumerate(specs):
        parts = pool.map(synth.batch_scan_part, [(k, a, min(90, a + 10)) for a in range(0, 90, 10)])
        h = synth.Histories.concat(parts)
        res = oracle.run(sp.geometry, h, threads=threads)
        scans.append({"scan": k, "geometry": geometry_record(sp.geometry), "histories": len(h),
                      "inputs_sha256": sha(h.arrays()), **output_record(sp.geometry, res)})
        print(f"  scan {k}: {len(h)} histories, {sp.geometry.nx}x{sp.geometry.ny}x"
              f"{sp.geometry.nz}", flush=True)
    return {"workload": "48 scans, grids {64x64x16, 128x128x32, 256x256x64} of 1x1x2.5 mm, "
                        "log-uniform 2e5-2e7 histories (configs 4 and 5)",
            "scans": scans}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="*", default=["head200", "head400", "batch48"])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(4, args.threads // 2))) as pool:
        for name in args.which:
            t0 = time.perf_counter()
            if name == "head200":
                rec = head200(args.threads)
            elif name == "head400":
                rec = head400(args.threads, pool)
            elif name == "batch48":
                rec = batch48(args.threads, pool)
            elif name == "euclid200":
                rec = euclid200(args.threads)
            elif name == "euclid200_d05":
                rec = euclid200(args.threads, 0.5)
            elif name == "thick200":
                rec = thick200(args.threads)
            elif name == "rows200":
                rec = rows200(args.threads)
            else:
                raise SystemExit(f"unknown workload {name}")
            rec["made_by"] = "oracle/make_golden.py (CPU oracle only)"
            path = os.path.join(GOLDEN, f"fullsize_{name}.json")
            with open(path, "w") as f:
                json.dump(rec, f, indent=0, sort_keys=True)
                f.write("\n")
            print(f"{name}: {time.perf_counter() - t0:.0f} s -> {path}", flush=True)


if __name__ == "__main__":
    main()
