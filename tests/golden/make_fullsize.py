#!/usr/bin/env python
"""Writes the oracle's full solves of the two large workloads as golden files.

Calls only ``oracle`` (the CPU FP64 revised simplex, OpenMP build, which is
bit-identical to the serial one) and ``lpgen`` (the seeded inputs); nothing
here touches the CUDA path.  For each workload it stores

  <name>.json        status, pivot and reinversion counts, rule counters,
                     objective and the certificate residuals of the oracle's
                     own solution;
  <name>_trace.npz   the whole pivot sequence: entering q, leaving row r,
                     trace flags, and the oracle's separation margins
                     margin_q = (d_q - best other eligible d) / max(1, |d_q|)
                     margin_r = min relative separation of r from the other rows
                     at every pivot (a choice is only unique where its margin
                     exceeds the 1e-12 tie tolerance).

  python tests/golden/make_fullsize.py [--only NAME] [--threads T]

Workloads (the method's settings: reinversion every 64 pivots, tabu tenure 7,
Bland net after 50 degenerate pivots, tolerances 1e-9 / 1e-9 / 1e-12):
  dense_real_4096x8192    A_ij ~ U[0,1) with 10% zeros, b ~ U[n/4, n/2], c ~ U[0,1), seed 1
  degenerate_2048x4096    A_ij in {-5..10}, 30% of b_i = 0, the rest U[1,100], c_j in {1..20}, seed 2
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "dense_real_4096x8192": dict(kind="real", m=4096, n=8192, seed=1),
    "degenerate_2048x4096": dict(kind="degenerate", m=2048, n=4096, seed=2),
}


def main():
    import lpgen
    import oracle
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None, choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: every host core)")
    args = ap.parse_args()
    for name, w in WORKLOADS.items():
        if args.only and name != args.only:
            continue
        A, b, c = lpgen.make(w["kind"], w["m"], w["n"], w["seed"])
        opts = oracle.Options()
        t0 = time.time()
        s = oracle.solve(A, b, c, opts, trace_cap=4_000_000, threads=args.threads)
        dt = time.time() - t0
        cert = oracle.certificate(A, b, c, s.x, s.y)
        tr = s.trace
        np.savez_compressed(os.path.join(HERE, f"{name}_trace.npz"),
                            q=tr["q"].astype(np.int32), r=tr["r"].astype(np.int32),
                            flags=tr["flags"].astype(np.int32),
                            margin_q=tr["margin_q"], margin_r=tr["margin_r"])
        summary = {
            "workload": name, **w,
            "options": {"reinvert_every": opts.reinvert_every, "tabu_tenure": opts.tabu_tenure,
                        "bland_after": opts.bland_after, "tol_d": opts.tol_d, "tol_piv": opts.tol_piv,
                        "tol_tie": opts.tol_tie},
            "status": oracle.STATUS_NAMES.get(s.status, str(s.status)),
            "iterations": int(s.iterations), "reinversions": int(s.reinversions),
            "degenerate": int(s.degenerate), "tabu_pushes": int(s.tabu_pushes),
            "bland_fallbacks": int(s.bland_fallbacks), "aspirations": int(s.aspirations),
            "objective": float(s.objective),
            "certificate": {k: float(v) for k, v in cert.items()},
            "unseparated_pivots": {
                "margin_q_le_1e-12": int(np.sum(tr["margin_q"] <= 1e-12)),
                "margin_r_le_1e-12": int(np.sum(tr["margin_r"] <= 1e-12))},
            "writer": "tests/golden/make_fullsize.py (oracle OpenMP build, "
                      f"{oracle.threads_used(args.threads)} threads, {dt:.0f} s)",
        }
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(summary, f, indent=1)
            f.write("\n")
        print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
