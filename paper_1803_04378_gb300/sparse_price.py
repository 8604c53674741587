"""Sparse FP64 PRICE on the paper's sparser dense classes (20% and 60% zeros,
m = 4096, n = 8192): the dense persistent engine with the dense PRICE and
with the compressed sparse column PRICE (price_mode 2), beside the default
slack-structured engine.

For each: pivots, seconds to optimum, microseconds per pivot without the
reinversions, the persistent kernel's algorithmic GB/s and the objective.

    python -m paper_1803_04378_gb300.sparse_price [--out FILE]
"""
from __future__ import annotations

import argparse
import json

RUNS = [("structured engine", dict(engine=2, price_mode=0)),
        ("dense engine, dense PRICE", dict(engine=0, price_mode=0)),
        ("dense engine, sparse PRICE", dict(engine=0, price_mode=2))]


def run(kind, m, n, seed, opts):
    import torch

    import lpgen
    from . import lpgb
    A, b, c = lpgen.make(kind, m, n, seed)
    At, bt, ct = (torch.from_numpy(v).cuda() for v in (A, b, c))
    with lpgb.LP(At, bt, ct, kernel_timing=64, **opts) as lp:
        lp.solve()  # warm-up
        lp.reset()
        r = lp.solve()
        z = lp.solution()[2]
    return {"pivots": r.iterations, "seconds": r.seconds, "objective": z,
            "us_per_pivot_excl_reinversion": 1e6 * (r.seconds - r.reinvert_seconds) / max(1, r.iterations),
            "reinversion_seconds": r.reinvert_seconds,
            "chain_gbs": r.chain_bytes / r.chain_seconds / 1e9 if r.chain_seconds else None,
            "engine": {2: "slack-structured persistent", 1: "dense persistent", 0: "captured graphs"}[r.persistent]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    from . import build
    build.build()
    out = []
    for kind in ("s20", "s60"):
        row = {"workload": f"{kind}_4096x8192", "seed": 1}
        for name, opts in RUNS:
            row[name] = run(kind, 4096, 8192, 1, opts)
        out.append(row)
        print(json.dumps(row), flush=True)
    if args.out:
        json.dump(out, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
