"""Report how much the fixed-point geometry changes the hull-detection result
against the same set definition on unquantised FP64 geometry (libm cos/sin,
no rounding).  Reported, not a parity reference: the method as built is the
fixed-point one, which the CUDA path matches bit for bit.

Test infrastructure: calls only the oracle and the seeded input generator.

    python oracle/fp64_report.py [config ...]      (default: 1 2)
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1402_1720_gb300 import synth  # noqa: E402


def report(cid: int, threads: int) -> dict:
    w = synth.make_config(cid)
    t0 = time.time()
    r = oracle.compare_fp64(w.geometry, w.histories, threads=threads)
    r["config"] = cid
    r["seconds"] = round(time.time() - t0, 1)
    r["threads"] = threads
    return r


def main(argv):
    cids = [int(a) for a in argv] or [1, 2]
    threads = os.cpu_count() or 1
    for cid in cids:
        print(json.dumps(report(cid, threads)), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
