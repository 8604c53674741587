"""Learned warm start for a family of perturbed LPs.

A base LP (A0, b0, c0) defines a family whose instances multiply every entry
by an independent N(1, sigma^2) draw.  A small network (lp_mlp_*: 2(m+n)
features -> 512 -> 512 -> n+m logits) learns, from (instance -> optimal basis)
pairs that the solver itself produces, which variables are basic at the
optimum.  A new instance starts from the basis the network proposes
(lp_family_propose on the device; lp_set_basis_repair: negative basic values
are repaired by slack pivots, and a proposal that needs more than a capped
number of them falls back to the slack basis, which bounds what a poor
proposal costs).  The plain method then runs to its certified optimum; the
guided variants also price the predicted columns first (lp_set_priority).

Everything here is orchestration: instances are drawn and featurised on the
GPU (lp_family_*), solved by the CUDA solver, and the network is trained and
served by the library's own kernels.
"""
from __future__ import annotations

import time

import numpy as np

import lpgen
from . import lpgb


class Family:
    """Device-resident base LP, one scratch instance and a reusable solver handle."""

    def __init__(self, base, sigma: float = 0.05, stream=None):
        import torch
        A0, b0, c0 = base
        self.m, self.n = A0.shape
        self.sigma = sigma
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.A0 = torch.from_numpy(np.ascontiguousarray(A0)).cuda()
        self.b0 = torch.from_numpy(np.ascontiguousarray(b0)).cuda()
        self.c0 = torch.from_numpy(np.ascontiguousarray(c0)).cuda()
        self.A = self.A0.clone()
        self.b = self.b0.clone()
        self.c = self.c0.clone()
        self.n_features = 2 * (self.m + self.n)
        self.n_outputs = self.n + self.m
        self.lp = lpgb.LP(self.A0, self.b0, self.c0, cuda_stream=self.stream)

    def close(self):
        self.lp.close()

    def draw(self, instance_seed: int):
        """Instance `instance_seed` of the family, drawn on the GPU."""
        key = lpgen.stream_key(instance_seed, lpgen.TAG_NOISE)
        lpgb.family_perturb(self.A0, self.b0, self.c0, key, self.sigma, self.A, self.b, self.c, self.stream)

    def load(self, A, b, c):
        """A host instance (e.g. drawn by lpgen.perturbed_lp for oracle checks)."""
        import torch
        self.A.copy_(torch.from_numpy(np.ascontiguousarray(A)))
        self.b.copy_(torch.from_numpy(np.ascontiguousarray(b)))
        self.c.copy_(torch.from_numpy(np.ascontiguousarray(c)))

    def features(self, out):
        lpgb.family_features(self.A0, self.b0, self.c0, self.A, self.b, self.c, self.sigma, out, self.stream)

    def solve(self, start=None, mode: str = "repair", max_repairs: int | None = None):
        """Solve the current instance.  start = (basis, structural set):
        mode "repair" starts from `basis` (repaired by at most max_repairs
        slack pivots, default m, else the slack basis) with the plain rule;
        "repair_guided" adds the guided rule on the structural set; "crash"
        starts from the slack basis and first enters the structural set in its
        order by ratio-test pivots (lp_set_crash), then the plain rule;
        "guided" starts from the slack basis with the guided rule only.  None
        solves cold."""
        self.lp.update_problem(self.A, self.b, self.c)
        if start is None:
            self.lp.set_priority([])
        else:
            basis, structurals = start
            cap = self.m if max_repairs is None else int(max_repairs)
            if mode == "repair":
                self.lp.set_priority([])
                self.lp.set_basis_repair(basis, cap)
            elif mode == "repair_guided":
                self.lp.set_priority(structurals)
                self.lp.set_basis_repair(basis, cap)
            elif mode == "crash":
                self.lp.set_priority([])
                self.lp.set_crash(list(structurals)[:self.m])
            elif mode == "guided":
                self.lp.set_priority(structurals)
            else:
                raise ValueError(mode)
        res = self.lp.solve()
        return res, self.lp.basis()


def base_hint(family: Family):
    """The base LP's optimal basis and its structural variables: the start
    used to generate training labels."""
    family.lp.update_problem(family.A0, family.b0, family.c0)
    family.lp.set_priority([])
    family.lp.solve()
    basis = family.lp.basis()
    return basis, [int(v) for v in basis if v < family.n]


def generate_labels(family: Family, seeds, hint=None, log_every: int = 0):
    """(features, optimal-basis indicator) pairs for the given instance seeds."""
    import torch
    N = len(seeds)
    X = torch.empty((N, family.n_features), dtype=torch.float32, device="cuda")
    Y = torch.zeros((N, family.n_outputs), dtype=torch.float32, device="cuda")
    pivots = np.zeros(N, np.int64)
    t0 = time.perf_counter()
    for k, s in enumerate(seeds):
        family.draw(int(s))
        family.features(X[k])
        res, basis = family.solve(hint)
        if res.status != lpgb.LP_OPTIMAL:
            raise RuntimeError(f"instance {s}: {res.status_name}")
        Y[k, torch.from_numpy(basis.astype(np.int64)).cuda()] = 1.0
        pivots[k] = res.iterations
        if log_every and (k + 1) % log_every == 0:
            print(f"labels {k + 1}/{N}  {time.perf_counter() - t0:.1f}s  mean pivots {pivots[:k + 1].mean():.0f}",
                  flush=True)
    return X, Y, pivots


def init_params(shapes, seed: int = 0):
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for s in shapes:
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[0])
            out.append(rng.uniform(-lim, lim, size=s).astype(np.float32).ravel())
        else:
            out.append(np.zeros(s, np.float32))
    return np.concatenate(out)


def train(X, Y, hidden: int = 512, epochs: int = 10, batch: int = 256, lr: float = 1e-3, seed: int = 0,
          stream=None, log: bool = False):
    import torch
    N, nf = X.shape
    no = Y.shape[1]
    net = lpgb.MLP(nf, hidden, no, batch, stream)
    net.set_params(init_params(net.shapes(), seed))
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g).cuda()
        tot, cnt = 0.0, 0
        for s in range(0, N - batch + 1, batch):
            idx = perm[s:s + batch]
            xb = X[idx].contiguous()
            yb = Y[idx].contiguous()
            tot += net.train_step(xb, yb, lr)
            cnt += 1
        losses.append(tot / max(1, cnt))
        if log:
            print(f"epoch {ep}: loss {losses[-1]:.4f}", flush=True)
    return net, losses


class Proposer:
    """Inference on the device: features -> logits (lp_mlp_forward) -> proposed
    basis (lp_family_propose); only the m basis entries and the proposed
    structurals come back to the host."""

    def __init__(self, net, m: int, n: int, threshold: float = 0.0):
        import torch
        self.net, self.m, self.n, self.threshold = net, m, n, threshold
        self.logits = torch.empty((1, net.out_dim), dtype=torch.float32, device="cuda")
        self.basis = torch.empty(m, dtype=torch.int32, device="cuda")
        self.work = torch.empty(m + 1, dtype=torch.int32, device="cuda")

    def __call__(self, features):
        self.net.forward(features.reshape(1, -1).contiguous(), self.logits)
        lpgb.family_propose(self.logits, self.m, self.n, self.basis, self.work, self.threshold)
        basis = self.basis.cpu().numpy()
        work = self.work.cpu().numpy()
        k = min(int(work[self.m]), self.m)
        return basis, [int(j) for j in work[:k]]


MODES = ("repair", "repair_guided", "crash", "guided")


def evaluate(family: Family, net, instances, modes=("repair",), max_repairs: int | None = None,
             threshold: float = 0.0):
    """Cold vs warm solves of held-out instances (instance seeds drawn on the
    device, or host (A, b, c) triples): pivots, device seconds (inference
    included for the warm starts), objectives, and how far the proposal is
    from the cold optimum's structural set (false positives / negatives)."""
    import torch
    feat = torch.empty(family.n_features, dtype=torch.float32, device="cuda")
    prop = Proposer(net, family.m, family.n, threshold)
    rows = []
    for inst in instances:
        if isinstance(inst, (int, np.integer)):
            family.draw(int(inst))
        else:
            family.load(*inst)
        cold, basis_cold = family.solve(None)
        z_cold = family.lp.solution()[2]
        opt = {int(v) for v in basis_cold if v < family.n}
        family.features(feat)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        start = prop(feat)
        t_pred = time.perf_counter() - t0
        J = set(start[1])
        row = dict(cold_pivots=cold.iterations, cold_s=cold.seconds, z_cold=z_cold, cold_status=cold.status,
                   cold_reinvert_s=cold.reinvert_seconds, cold_chain_s=cold.chain_seconds,
                   predict_s=t_pred, predicted=len(J), optimal_structurals=len(opt),
                   false_pos=len(J - opt), false_neg=len(opt - J))
        for mode in modes:
            res, _ = family.solve(start, mode=mode, max_repairs=max_repairs)
            row[mode] = dict(pivots=res.iterations, s=res.seconds + t_pred, z=family.lp.solution()[2],
                             status=res.status, repairs=res.warm_repairs, fallback=res.warm_fallback,
                             reinvert_s=res.reinvert_seconds, chain_s=res.chain_seconds)
        rows.append(row)
    return rows


def summarize(rows, modes=("repair",)):
    """Per mode: mean pivots and time-to-optimum against cold, the speedup
    (sum of cold over sum of warm device seconds), fallbacks and the largest
    relative objective gap to the cold solve."""
    cp = np.array([r["cold_pivots"] for r in rows], float)
    cs = np.array([r["cold_s"] for r in rows])
    zc = np.array([r["z_cold"] for r in rows])
    out = dict(instances=len(rows), cold_pivots_mean=float(cp.mean()), cold_time_to_optimum_s=float(cs.mean()),
               predicted_mean=float(np.mean([r["predicted"] for r in rows])),
               optimal_structurals_mean=float(np.mean([r["optimal_structurals"] for r in rows])),
               false_pos_mean=float(np.mean([r["false_pos"] for r in rows])),
               false_neg_mean=float(np.mean([r["false_neg"] for r in rows])),
               predict_s_mean=float(np.mean([r["predict_s"] for r in rows])))
    for mode in modes:
        wp = np.array([r[mode]["pivots"] for r in rows], float)
        ws = np.array([r[mode]["s"] for r in rows])
        zw = np.array([r[mode]["z"] for r in rows])
        out[mode] = dict(pivots_mean=float(wp.mean()), pivot_ratio=float(wp.sum() / cp.sum()),
                         time_to_optimum_s=float(ws.mean()), speedup=float(cs.sum() / ws.sum()),
                         faster_fraction=float(np.mean(ws < cs)),
                         fallbacks=int(sum(r[mode]["fallback"] for r in rows)),
                         repairs_mean=float(np.mean([r[mode]["repairs"] for r in rows])),
                         optimal=bool(all(r[mode]["status"] == lpgb.LP_OPTIMAL for r in rows)),
                         max_rel_objective_gap=float(np.max(np.abs(zw - zc) / np.maximum(1.0, np.abs(zc)))))
    return out


def proposal_sensitivity(family: Family, seeds, swaps=(0, 1, 2, 4, 8, 16), seed: int = 0, kind: str = "swap"):
    """How good a proposal must be: each instance is solved cold, then started
    (mode "repair") from its own optimal basis with k errors: "swap" replaces
    k basic structurals by random nonbasic structurals, "drop" replaces them
    by the slacks of k random tight rows (a proposal that misses structurals),
    "add" replaces k basic slacks by random nonbasic structurals (a proposal
    with extra ones).  Returns, per k, the mean pivots, repair pivots and
    device seconds against cold, and the largest objective gap."""
    rng = np.random.default_rng(seed)
    acc = {k: [] for k in swaps}
    cold_p, cold_s = [], []
    for inst in seeds:
        family.draw(int(inst))
        cold, basis = family.solve(None)
        zc = family.lp.solution()[2]
        cold_p.append(cold.iterations)
        cold_s.append(cold.seconds)
        spos = np.nonzero(basis < family.n)[0]                       # positions of basic structurals
        lpos = np.nonzero(basis >= family.n)[0]                      # positions of basic slacks
        nonb = np.setdiff1d(np.arange(family.n), basis)              # nonbasic structurals
        tight = np.setdiff1d(np.arange(family.n, family.n + family.m), basis)  # nonbasic slacks
        for k in swaps:
            prop = basis.copy()
            if kind == "add":
                kk = min(k, len(lpos), len(nonb))
                at, new = lpos, nonb
            else:
                kk = min(k, len(spos), len(nonb) if kind == "swap" else len(tight))
                at, new = spos, (nonb if kind == "swap" else tight)
            if kk:
                prop[rng.choice(at, kk, replace=False)] = rng.choice(new, kk, replace=False)
            res, _ = family.solve((prop, []), mode="repair")
            acc[k].append((res.iterations, res.warm_repairs, res.seconds, res.warm_fallback,
                           abs(family.lp.solution()[2] - zc) / max(1.0, abs(zc))))
    out = dict(instances=len(cold_p), cold_pivots_mean=float(np.mean(cold_p)), cold_s_mean=float(np.mean(cold_s)))
    for k in swaps:
        a = np.array(acc[k])
        out[f"swap{k}"] = dict(pivots_mean=float(a[:, 0].mean()), repairs_mean=float(a[:, 1].mean()),
                               s_mean=float(a[:, 2].mean()), speedup=float(np.sum(cold_s) / a[:, 2].sum()),
                               fallbacks=int(a[:, 3].sum()), max_rel_objective_gap=float(a[:, 4].max()))
    return out


def main():
    """The configured experiment: 20000 training pairs, 1000 held-out
    instances, base as the dense real workload at m=1024, n=2048 (seed 4)."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--out", default="")
    ap.add_argument("--labels", default="cold", choices=["hint", "cold"],
                    help="label solves start from the slack basis (cold) or the base LP's optimal basis (hint)")
    ap.add_argument("--modes", default="repair", help="comma-separated subset of " + ",".join(MODES))
    ap.add_argument("--max-repairs", type=int, default=None,
                    help="repair pivots before a proposal falls back to the slack basis (default m)")
    ap.add_argument("--thresholds", default="0,1,2,3",
                    help="proposal thresholds on the structural scores, the best one picked on the validation instances")
    ap.add_argument("--validation", type=int, default=200, help="validation instances for the threshold")
    ap.add_argument("--save-params", default="", help="write the trained parameters (float32 .npy) here")
    ap.add_argument("--sensitivity", type=int, default=0,
                    help="only measure starts from the optimal basis with k errors, on this many instances")
    ap.add_argument("--kind", default="swap", choices=["swap", "drop", "add"], help="error kind of --sensitivity")
    args = ap.parse_args()
    modes = tuple(v for v in args.modes.split(",") if v)
    from . import build
    build.build()
    base = lpgen.dense_real_lp(args.m, args.n, 4)
    fam = Family(base)
    if args.sensitivity:
        out = dict(proposal_sensitivity(fam, range(20_000_000, 20_000_000 + args.sensitivity), kind=args.kind),
                   m=args.m, n=args.n, kind=args.kind)
        print(json.dumps(out))
        return
    hint = base_hint(fam) if args.labels == "hint" else None
    t0 = time.perf_counter()
    X, Y, piv = generate_labels(fam, range(1, args.train + 1), hint, log_every=1000)
    t_labels = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, losses = train(X, Y, epochs=args.epochs, log=True)
    t_train = time.perf_counter() - t0
    if args.save_params:
        np.save(args.save_params, net.get_params())
    # the proposal threshold: the best time-to-optimum on validation instances
    # (seeds disjoint from the training and held-out ones)
    val = range(30_000_000, 30_000_000 + args.validation)
    sel = {}
    for t in (float(v) for v in args.thresholds.split(",") if v):
        sv = summarize(evaluate(fam, net, val, ("repair",), args.max_repairs, t), ("repair",))
        sel[t] = sv["repair"]["speedup"]
        print(f"validation threshold {t}: speedup {sel[t]:.3f}, pivot ratio {sv['repair']['pivot_ratio']:.3f}",
              flush=True)
    thr = max(sel, key=sel.get) if sel else 0.0
    rows = evaluate(fam, net, range(10_000_000, 10_000_000 + args.heldout), modes, args.max_repairs, thr)
    out = dict(summarize(rows, modes), train_pairs=args.train, label_seconds=t_labels, train_seconds=t_train,
               label_pivots_mean=float(piv.mean()), losses=losses, m=args.m, n=args.n, labels=args.labels,
               max_repairs=args.max_repairs if args.max_repairs is not None else args.m, epochs=args.epochs,
               threshold=thr, validation_speedups=sel, validation_instances=args.validation)
    print(json.dumps(out))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(out, rows=rows), f, indent=1)


if __name__ == "__main__":
    main()
