"""Training and evaluation of the learned (levels, p) selector.

The selector (include/fmm.h, ``fmm_select``) is a small network that reads occupancy
statistics of a particle system and predicts, for a candidate (levels, p), the relative L2
error and the run time of the mixed-precision method; it then picks the cheapest candidate
predicted to meet a requested accuracy, or the fixed fallback (8, 20).

Its training tuples are generated by the method itself: for each synthetic system, every
candidate of the grid is run through ``fmm_potential`` (in the precision given, by default the
BF16x2 tensor-core form the benchmark quotes), timed with CUDA events, and measured against the
library's FP64 direct sum (``fmm_direct_targets``) on sampled targets.  The network is then
fitted by the library's own forward / backward / Adam kernels.

``evaluate`` compares, on held-out systems, the learned pick with the fixed fallback, with a
rule that uses no network (levels = round(log4(N / 16)), p = the smallest of the grid that meets
the target on a uniform calibration system), and with the best candidate an exhaustive search of
the grid finds (its regret).

Workload of the tuples: N log-uniform in [2^16, 2^20]; families uniform, Gaussian mixture
(K in [4, 64], sigma log-uniform in [0.02, 0.5], out-of-box draws redrawn) and annulus
(r in [1, 2] about (2.5, 2.5)); q ~ U[-1, 1].

    python -m paper_2009_00767_gb300.selector train --out selector.bin --systems 96
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding, inputs

FALLBACK = (8, 20)
P_GRID = (8, 12, 16, 20, 24, 28)   # the p candidates of fmm_select
DEFAULT_PRECISION = "bf16x2"
TENSOR_CORE = ("tf32", "3xtf32", "bf16", "bf16x2", "bf16x3")   # these take p + 1 <= 32 coefficients
LOG10_SCALE = 8.0           # the network predicts log10(error) / 8
ERR_FLOOR = 1e-8            # errors below this are labelled at the floor


def candidates(n, precision=DEFAULT_PRECISION):
    l0 = int(round(math.log(n / 16.0) / math.log(4.0)))
    pmax = 31 if precision in TENSOR_CORE else 40
    out = []
    for lev in range(l0 - 2, l0 + 3):
        if 2 <= lev <= 11:
            for p in P_GRID:
                if p <= pmax:
                    out.append((lev, p))
    return out


def system(seed, n_lo=1 << 16, n_hi=1 << 20):
    """One synthetic system of the training / evaluation family."""
    u = inputs.u01(seed, 41, 4)
    n = int(math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * u[0]))
    fam = int(u[1] * 3)
    if fam == 0:
        xy, q = inputs.uniform(n, seed)
        name = "uniform"
    elif fam == 1:
        k = int(4 + 60 * u[2])
        xy, q = inputs.gmm(n, seed, k=k, sigma_lo=0.02, sigma_hi=0.5)
        name = f"gmm{k}"
    else:
        xy, q = inputs.annulus(n, seed)
        name = "annulus"
    return name, xy, q


def _time_plan(torch, plan, xy_d, q_d, phi, reps=3):
    binding.fmm_potential(plan.handle, xy_d, q_d, phi)   # warm-up
    plan.sync()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        binding.fmm_potential(plan.handle, xy_d, q_d, phi)
        b.record()
        plan.sync()
        ms.append(a.elapsed_time(b))
        if ms[-1] > 200.0:
            break
    return float(np.median(ms))


def reference_targets(torch, xy_d, q_d, n, seed, s=256):
    idx = np.unique((inputs.u01(seed, 77, s) * n).astype(np.int64))
    idx_d = torch.from_numpy(idx).to(xy_d.device)
    ref = torch.empty(idx.shape[0], dtype=torch.float64, device=xy_d.device)
    binding.fmm_direct_targets(xy_d, q_d, idx_d, ref)
    torch.cuda.synchronize()
    return idx_d, ref


def run_candidate(torch, xy_d, q_d, idx_d, ref, lev, p, precision=DEFAULT_PRECISION):
    n = int(q_d.shape[0])
    phi = torch.empty(n, dtype=torch.float64, device=xy_d.device)
    with binding.Plan(n, lev, p, 5.0, precision) as plan:
        ms = _time_plan(torch, plan, xy_d, q_d, phi)
    err = float(torch.linalg.norm(phi[idx_d] - ref) / torch.linalg.norm(ref))
    return err, ms


def label(err, ms):
    return [math.log10(max(err, ERR_FLOOR)) / LOG10_SCALE, math.log(max(ms, 1e-3))]


def generate(sel, seeds, log=print, precision=DEFAULT_PRECISION):
    """Tuples (features ++ candidate, [log10 err / 8, log ms]) for the systems of ``seeds``."""
    import torch
    X, T, meta = [], [], []
    for sd in seeds:
        name, xy, q = system(sd)
        xy_d = torch.from_numpy(xy).to("cuda")
        q_d = torch.from_numpy(q).to("cuda")
        feat = sel.features(xy_d)
        idx_d, ref = reference_targets(torch, xy_d, q_d, q.shape[0], sd)
        t0 = time.time()
        for lev, p in candidates(q.shape[0], precision):
            err, ms = run_candidate(torch, xy_d, q_d, idx_d, ref, lev, p, precision)
            X.append(np.concatenate([feat, [lev / 12.0, p / 32.0]]))
            T.append(label(err, ms))
            meta.append({"seed": sd, "family": name, "n": int(q.shape[0]), "levels": lev, "p": p, "err": err, "ms": ms})
        log(f"system {sd}: {name} N={q.shape[0]} {len(candidates(q.shape[0], precision))} candidates in "
            f"{time.time() - t0:.1f}s")
    return np.asarray(X, dtype=np.float32), np.asarray(T, dtype=np.float32), meta


def best_feasible(meta_rows, target):
    ok = [r for r in meta_rows if r["err"] <= target]
    return min(ok, key=lambda r: r["ms"]) if ok else None


def heuristic_levels(n):
    """The depth that puts about 16 particles in a finest square, clamped to [2, 11]."""
    return min(11, max(2, int(round(math.log(n / 16.0) / math.log(4.0)))))


def calibrate_p(target=1e-6, precision=DEFAULT_PRECISION, n=1 << 18, seed=880001):
    """The rule's p: the smallest p of the grid whose error on a uniform system of n particles (at
    the rule's depth) meets the target, judged by the FP64 direct sum."""
    import torch
    xy, q = inputs.uniform(n, seed)
    xy_d = torch.from_numpy(xy).to("cuda")
    q_d = torch.from_numpy(q).to("cuda")
    idx_d, ref = reference_targets(torch, xy_d, q_d, n, seed)
    for p in P_GRID:
        err, _ = run_candidate(torch, xy_d, q_d, idx_d, ref, heuristic_levels(n), p, precision)
        if err <= target:
            return p
    return P_GRID[-1]


def evaluate(sel, seeds, target=1e-6, margin=0.3, precision=DEFAULT_PRECISION, exhaustive=False, p_rule=None):
    """Learned pick vs the fixed fallback on held-out systems, both measured against the FP64 direct
    sum; with ``exhaustive`` also the rule without a network (p_rule: its calibrated p) and the best
    feasible candidate of the whole grid (the pick's regret = ms_pick / ms_best - 1)."""
    import torch
    if exhaustive and p_rule is None:
        p_rule = calibrate_p(target, precision)
    rows = []
    for sd in seeds:
        name, xy, q = system(sd)
        n = int(q.shape[0])
        xy_d = torch.from_numpy(xy).to("cuda")
        q_d = torch.from_numpy(q).to("cuda")
        lev, p, fb = sel.select(xy_d, target, margin)
        idx_d, ref = reference_targets(torch, xy_d, q_d, n, sd)
        err_l, ms_l = run_candidate(torch, xy_d, q_d, idx_d, ref, lev, p, precision)
        err_f, ms_f = run_candidate(torch, xy_d, q_d, idx_d, ref, *FALLBACK, precision)
        row = {"seed": sd, "family": name, "n": n, "pick": [lev, p], "fallback_used": fb,
               "err_pick": err_l, "ms_pick": ms_l, "err_fallback": err_f, "ms_fallback": ms_f}
        if exhaustive:
            grid = []
            for cl, cp in candidates(n, precision):
                e, m = (err_l, ms_l) if (cl, cp) == (lev, p) else run_candidate(torch, xy_d, q_d, idx_d, ref, cl,
                                                                               cp, precision)
                grid.append({"levels": cl, "p": cp, "err": e, "ms": m})
            best = best_feasible(grid, target)
            hl = heuristic_levels(n)
            err_h, ms_h = run_candidate(torch, xy_d, q_d, idx_d, ref, hl, p_rule, precision)
            row.update({"rule": [hl, p_rule], "err_rule": err_h, "ms_rule": ms_h,
                        "best": [best["levels"], best["p"]] if best else None,
                        "ms_best": best["ms"] if best else None,
                        "regret": (ms_l / best["ms"] - 1.0) if best else None})
        rows.append(row)
    return rows


def summary(rows, target=1e-6):
    """Totals over held-out rows: time and the count meeting the target for each way of choosing."""
    out = {"systems": len(rows)}
    for key in ("pick", "fallback", "rule"):
        if f"ms_{key}" in rows[0]:
            out[key] = {"ms_total": sum(r[f"ms_{key}"] for r in rows),
                        "met": sum(r[f"err_{key}"] <= target for r in rows)}
    if rows and rows[0].get("ms_best") is not None:
        out["best"] = {"ms_total": sum(r["ms_best"] for r in rows if r["ms_best"] is not None)}
        reg = [r["regret"] for r in rows if r["regret"] is not None]
        out["regret"] = {"mean": float(np.mean(reg)), "max": float(np.max(reg)), "median": float(np.median(reg))}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--out", required=True)
    tr.add_argument("--systems", type=int, default=96)
    tr.add_argument("--seed0", type=int, default=700000)
    tr.add_argument("--epochs", type=int, default=6000)
    tr.add_argument("--hidden", type=int, default=64)
    tr.add_argument("--dataset", default=None, help="save the generated tuples (.npz)")
    tr.add_argument("--eval-systems", type=int, default=24)
    tr.add_argument("--report", default=None)
    tr.add_argument("--precision", default=DEFAULT_PRECISION)
    a = ap.parse_args(argv)
    build_lib()
    sel = binding.Selector(hidden=a.hidden, seed=1)
    X, T, meta = generate(sel, range(a.seed0, a.seed0 + a.systems), precision=a.precision)
    if a.dataset:
        np.savez(a.dataset, X=X, T=T, meta=json.dumps(meta))
    losses = []
    for chunk in range(a.epochs // 500):
        losses.append(sel.train(X, T, 500, lr=1e-3 if chunk < 8 else 3e-4))
        print(f"epoch {(chunk + 1) * 500}: loss {losses[-1]:.5f}")
    sel.save(a.out)
    ev = evaluate(sel, range(a.seed0 + 10_000, a.seed0 + 10_000 + a.eval_systems), precision=a.precision,
                  exhaustive=True)
    rep = {"train_tuples": int(X.shape[0]), "precision": a.precision, "losses": losses, "eval": ev,
           "summary": summary(ev)}
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    print("held-out:", json.dumps(summary(ev)))


def build_lib():
    from . import build
    build.build()


if __name__ == "__main__":
    main()
