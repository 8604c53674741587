"""Anti-cycling rules compared on the GPU: the tabu rule of Sections 2.2 and
3.4 (the method, with its Bland safety net) against the lexicographic rule.

For each workload and rule: outcome, pivots, degenerate pivots, tabu pushes,
safety-net activations, device seconds and objective.  The degenerate
workload (2048 x 4096, integer A in -5..10, 30% of the rows with b_i = 0) has
x = 0 as its only feasible point, so every pivot is degenerate and the rule
decides how long the method takes to prove optimality; the dense workload has
no ties, and both rules make the same pivots there.

    python -m paper_1803_04378_gb300.compare_rules [--out FILE]
"""
from __future__ import annotations

import argparse
import json


WORKLOADS = [("degenerate", 2048, 4096, 2), ("degenerate", 1024, 2048, 2), ("real", 4096, 8192, 1)]


def run(kind, m, n, seed, anticycling, max_iters=2_000_000):
    import torch

    import lpgen
    from . import lpgb
    A, b, c = lpgen.make(kind, m, n, seed)
    At, bt, ct = (torch.from_numpy(v).cuda() for v in (A, b, c))
    with lpgb.LP(At, bt, ct, anticycling=anticycling, max_iters=max_iters) as lp:
        lp.solve()  # warm-up
        lp.reset()
        res = lp.solve()
        z = lp.solution()[2] if res.status == lpgb.LP_OPTIMAL else None
    return {"status": res.status_name, "pivots": res.iterations, "degenerate": res.degenerate,
            "tabu_pushes": res.tabu_pushes, "bland_fallbacks": res.bland_fallbacks,
            "seconds": res.seconds, "objective": z,
            "engine": {2: "slack-structured persistent", 1: "dense persistent", 0: "captured graphs"}[res.persistent]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    from . import build, lpgb
    build.build()
    out = []
    for kind, m, n, seed in WORKLOADS:
        row = {"workload": f"{kind}_{m}x{n}", "seed": seed}
        for name, rule in (("tabu", lpgb.LP_ANTICYCLING_TABU), ("lexicographic", lpgb.LP_ANTICYCLING_LEXICOGRAPHIC)):
            row[name] = run(kind, m, n, seed, rule)
        out.append(row)
        print(json.dumps(row), flush=True)
    if args.out:
        json.dump(out, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
