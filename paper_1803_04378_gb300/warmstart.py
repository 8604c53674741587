"""Learned warm start for a family of perturbed LPs.

A base LP (A0, b0, c0) defines a family whose instances multiply every entry
by an independent N(1, sigma^2) draw.  A small network (lp_mlp_*: 2(m+n)
features -> 512 -> 512 -> n+m logits) learns, from (instance -> optimal basis)
pairs that the solver itself produces, which variables are basic at the
optimum.  A new instance starts from the basis the network proposes
(lp_set_basis_repair: negative basic values are repaired by dual-style slack
pivots, an unusable proposal falls back to the slack basis), and the predicted
columns are priced first (lp_set_priority, Dantzig's rule restricted to them
while any of them improves).  Every pivot is an ordinary simplex pivot and the
plain method certifies the optimum.

Everything here is orchestration: instances are drawn and featurised on the
GPU (lp_family_*), solved by the CUDA solver, and the network is trained by
the library's own kernels.  Training labels come from solves started from
the base LP's optimal basis, which reach an optimum in a fraction of the cold
pivots.
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

    def solve(self, start=None, mode: str = "repair"):
        """Solve the current instance.  start = (basis, structural set):
        mode "repair" starts from `basis` (repaired if infeasible) with the
        guided rule on the structural set; mode "guided" starts from the slack
        basis and only applies the guided rule.  None solves cold."""
        self.lp.update_problem(self.A, self.b, self.c)
        if start is None:
            self.lp.set_priority([])
        else:
            basis, structurals = start
            self.lp.set_priority(structurals)
            if mode == "repair":
                self.lp.set_basis_repair(basis, self.m)
            elif mode != "guided":
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


def basis_from_scores(z, m: int, n: int):
    """Proposed basis from per-variable scores z (n+m; higher = more likely
    basic): the structurals with z > 0, best first, placed at the positions of
    the rows whose slacks score lowest; every other row keeps its slack."""
    zs = np.asarray(z[:n])
    order = np.argsort(-zs, kind="stable")
    J = [int(j) for j in order if zs[j] > 0.0][:m]
    rows = np.argsort(np.asarray(z[n:n + m]), kind="stable")[:len(J)]
    basis = np.arange(n, n + m, dtype=np.int32)
    for j, r in zip(J, rows):
        basis[r] = j
    return basis, J


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


def predicted_start(net, features, m: int, n: int):
    """The network's proposal for one instance: (basis, structural set)."""
    import torch
    logits = torch.empty((1, net.out_dim), dtype=torch.float32, device="cuda")
    net.forward(features.reshape(1, -1).contiguous(), logits)
    torch.cuda.synchronize()
    return basis_from_scores(logits[0].cpu().numpy(), m, n)


def evaluate(family: Family, net, instances, guided: bool = False):
    """Cold vs warm solves of host instances: pivots, device seconds, objectives
    (guided: also the slack-basis start with the guided rule only)."""
    import torch
    feat = torch.empty(family.n_features, dtype=torch.float32, device="cuda")
    rows = []
    for (A, b, c) in instances:
        family.load(A, b, c)
        cold, _ = family.solve(None)
        z_cold = family.lp.solution()[2]
        family.features(feat)
        t0 = time.perf_counter()
        start = predicted_start(net, feat, family.m, family.n)
        t_pred = time.perf_counter() - t0
        warm, _ = family.solve(start)
        z_warm = family.lp.solution()[2]
        row = dict(cold_pivots=cold.iterations, warm_pivots=warm.iterations,
                   cold_s=cold.seconds, warm_s=warm.seconds + t_pred, predict_s=t_pred,
                   z_cold=z_cold, z_warm=z_warm, predicted=len(start[1]),
                   repairs=warm.warm_repairs, fallback=warm.warm_fallback,
                   status=(cold.status, warm.status))
        if guided:
            gd, _ = family.solve(start, mode="guided")
            row.update(guided_pivots=gd.iterations, guided_s=gd.seconds + t_pred,
                       z_guided=family.lp.solution()[2], guided_status=gd.status)
        rows.append(row)
    return rows


def summarize(rows):
    cp = np.array([r["cold_pivots"] for r in rows], float)
    wp = np.array([r["warm_pivots"] for r in rows], float)
    cs = np.array([r["cold_s"] for r in rows])
    wsec = np.array([r["warm_s"] for r in rows])
    zc = np.array([r["z_cold"] for r in rows])
    zw = np.array([r["z_warm"] for r in rows])
    fb = np.array([r.get("fallback", 0) for r in rows])
    rp = np.array([r.get("repairs", 0) for r in rows])
    out = dict(instances=len(rows), cold_pivots_mean=float(cp.mean()), warm_pivots_mean=float(wp.mean()),
               fallbacks=int(fb.sum()), repairs_mean=float(rp.mean()),
               pivot_ratio=float(wp.sum() / cp.sum()), cold_time_to_optimum_s=float(cs.mean()),
               warm_time_to_optimum_s=float(wsec.mean()), speedup=float(cs.sum() / wsec.sum()),
               max_rel_objective_gap=float(np.max(np.abs(zw - zc) / np.maximum(1.0, np.abs(zc)))))
    if rows and "guided_pivots" in rows[0]:
        gp = np.array([r["guided_pivots"] for r in rows], float)
        gs = np.array([r["guided_s"] for r in rows])
        zg = np.array([r["z_guided"] for r in rows])
        out.update(guided_pivots_mean=float(gp.mean()), guided_pivot_ratio=float(gp.sum() / cp.sum()),
                   guided_time_to_optimum_s=float(gs.mean()), guided_speedup=float(cs.sum() / gs.sum()),
                   guided_max_rel_objective_gap=float(np.max(np.abs(zg - zc) / np.maximum(1.0, np.abs(zc)))))
    return out


def main():
    """Full experiment: 20000 training pairs, 1000 held-out instances, base
    as the dense real workload at m=1024, n=2048 (seed 4)."""
    import argparse
    import json

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--out", default="")
    ap.add_argument("--labels", default="hint", choices=["hint", "cold"],
                    help="label solves start from the base LP's optimal basis (hint) or the slack basis")
    ap.add_argument("--guided", action="store_true",
                    help="also evaluate the slack-basis start with the guided rule only")
    args = ap.parse_args()
    from . import build
    build.build()
    base = lpgen.dense_real_lp(args.m, args.n, 4)
    fam = Family(base)
    hint = base_hint(fam) if args.labels == "hint" else None
    t0 = time.perf_counter()
    X, Y, piv = generate_labels(fam, range(1, args.train + 1), hint, log_every=1000)
    t_labels = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, losses = train(X, Y, epochs=args.epochs, log=True)
    t_train = time.perf_counter() - t0
    held = [lpgen.perturbed_lp(base, 10_000_000 + k) for k in range(args.heldout)]
    rows = evaluate(fam, net, held, guided=args.guided)
    out = dict(summarize(rows), train_pairs=args.train, label_seconds=t_labels, train_seconds=t_train,
               label_pivots_mean=float(piv.mean()), losses=losses, m=args.m, n=args.n, labels=args.labels)
    print(json.dumps(out))
    if args.out:
        json.dump(out, open(args.out, "w"), indent=1)
    del torch


if __name__ == "__main__":
    main()
