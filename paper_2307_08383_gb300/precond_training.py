"""Training and evaluation of the learned block-Jacobi correction.

Instances are reduced camera systems this library forms (FP64 assembly) from
seeded aerial scenes of 2,000-8,000 cameras with 200 points per camera: for
each scene the RCS of LM iteration 0 (lambda0) and of LM iteration 1 (lambda
after one step of Nielsen's rule).  Scene seeds 0-99 give the 200 training
instances, 100-103 the validation instances, 200-209 the 20 held-out ones.

Training runs Adam on the network's loss (GPU forward and backward kernels,
include/ba.h) over the training instances.  Among the initial weights (a
zero output layer: plain block-Jacobi) and the weights after each epoch, for
each learning rate tried, it keeps those with the fewest PCG iterations of
the mixed-precision solve to 1e-8 summed over the validation instances - so
the kept network never does worse than block-Jacobi there.

Evaluation: iterations and time to ||b - S x|| / ||b|| <= 1e-8 (the true FP64
residual) for FP64 block-Jacobi PCG, mixed-precision block-Jacobi PCG (FP32
inner PCG on the demoted S, FP64 refinement) and mixed precision with the
learned correction.

    python -m paper_2307_08383_gb300.precond_training --train 100 --heldout 10 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _instances_of_scene(seed: int, n_cams=None):
    """(row_ptr, col, val, b, lam) of the FP64 RCS at LM iterations 0 and 1."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import scenes
    import paper_2307_08383_gb300 as B
    s = scenes.preconditioner_scene(seed, n_cams=n_cams)
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, stream=None, precision=B.BA_FP64,
                  pcg_rel_tol=0.1)
    out = []
    lam0, _, _ = g.lm_state()
    g.linearize()
    g.form_rcs(lam0)
    out.append((*g.rcs(), lam0))
    g.lm_step()
    lam1, _, _ = g.lm_state()
    g.linearize()
    g.form_rcs(lam1)
    out.append((*g.rcs(), lam1))
    g.close()
    return seed, out


def make_instances(seeds, workers=8, n_cams=None):
    """RCS instances of the given scene seeds, built in a spawn pool."""
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(workers) as pool:
        for seed, inst in pool.imap_unordered(_worker, [(s, n_cams) for s in seeds]):
            res[seed] = inst
    return [x for s in sorted(res) for x in res[s]]


def _worker(args):
    return _instances_of_scene(*args)


def _problem(B, inst, **kw):
    row_ptr, col, val, b, _ = inst
    return B.Problem.from_rcs(row_ptr, col, val, b, **kw)


def _mixed(B, tol=1e-8, inner=1e-4):
    return dict(precision=B.BA_FP64, solve_precision=B.BA_FP32, inner_rel_tol=inner, pcg_rel_tol=tol,
                pcg_max_iters=50000)


def solve_iters(B, probs, net):
    """Total PCG iterations of the solves of probs with net (None: block-Jacobi)."""
    total = 0
    for g in probs:
        B.ba_set_precond_net(g, net)
        info, conv = g.solve_rcs()
        total += info["pcg_iters"] if conv and not info["used_fallback"] else 10 ** 7
        B.ba_set_precond_net(g, None)
    return total


def train(B, train_inst, val_inst, epochs=20, lrs=(1e-3,), kp=4, seed=0, log=print):
    """Adam over train_inst for each learning rate; returns the net with the
    kept weights (fewest validation iterations, block-Jacobi included)."""
    tr = [_problem(B, x, precision=B.BA_FP32) for x in train_inst]
    va = [_problem(B, x, **_mixed(B)) for x in val_inst]
    net = B.PrecondNet(seed=seed)
    bj = solve_iters(B, va, None)
    best = (bj, None, -1, net.params())
    hist = [{"lr": None, "epoch": -1, "val_iters": bj}]
    log(f"block-Jacobi validation iterations {bj}")
    for lr in lrs:
        net = B.PrecondNet(seed=seed)
        rng = np.random.default_rng(seed)
        step = 0
        for ep in range(epochs):
            losses = []
            for k in rng.permutation(len(tr)):
                losses.append(net.train_step(tr[k], kp=kp, seed=1000003 * ep + step, lr=lr))
                step += 1
            it = solve_iters(B, va, net)
            hist.append({"lr": lr, "epoch": ep, "loss": float(np.mean(losses)), "val_iters": it})
            log(f"lr {lr:g} epoch {ep}: loss {np.mean(losses):.5f} validation iterations {it} (block-Jacobi {bj})")
            if it < best[0]:
                best = (it, lr, ep, net.params())
        net.close()
    for g in tr + va:
        g.close()
    net = B.PrecondNet(seed=seed)
    net.set_params(best[3])
    return net, best[3], {"kept_lr": best[1], "kept_epoch": best[2], "val_iters": best[0],
                          "val_iters_block_jacobi": bj, "history": hist}


def _timed_solve(B, g):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, conv = g.solve_rcs()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, info, conv


def evaluate(B, net, instances, tol=1e-8, inner=1e-4, repeats=3):
    """Per instance: (iterations, seconds, true residual) of the three solvers."""
    rows = []
    for inst in instances:
        r = {"n": len(inst[0]) - 1, "lambda": inst[4]}
        for name, kw, use_net in (("fp64_block_jacobi", dict(precision=B.BA_FP64, pcg_rel_tol=tol,
                                                             pcg_max_iters=50000), False),
                                  ("mixed_block_jacobi", _mixed(B, tol, inner), False),
                                  ("mixed_learned", _mixed(B, tol, inner), True)):
            g = _problem(B, inst, **kw)
            if use_net:
                B.ba_set_precond_net(g, net)
            _timed_solve(B, g)  # warm-up (kernel attributes, workspaces)
            best = None
            for _ in range(repeats):
                dt, info, conv = _timed_solve(B, g)
                if best is None or dt < best[0]:
                    best = (dt, info, conv)
            dt, info, conv = best
            r[name] = {"seconds": dt, "pcg_iters": info["pcg_iters"], "refine_steps": info["refine_steps"],
                       "true_rel_resid": info["rcs_rel_resid"], "converged": bool(conv),
                       "used_fallback": info["used_fallback"]}
            B.ba_set_precond_net(g, None)
            g.close()
        rows.append(r)
    return rows


def summarize(rows):
    def med(key, field):
        return statistics.median(r[key][field] for r in rows)
    out = {}
    for key in ("fp64_block_jacobi", "mixed_block_jacobi", "mixed_learned"):
        out[key] = {"median_seconds": med(key, "seconds"), "median_pcg_iters": med(key, "pcg_iters"),
                    "all_converged": all(r[key]["converged"] for r in rows),
                    "max_true_rel_resid": max(r[key]["true_rel_resid"] for r in rows)}
    out["speedup_mixed_learned_vs_fp64_block_jacobi"] = (out["fp64_block_jacobi"]["median_seconds"]
                                                         / out["mixed_learned"]["median_seconds"])
    out["iteration_ratio_learned_vs_block_jacobi"] = (out["mixed_learned"]["median_pcg_iters"]
                                                      / out["mixed_block_jacobi"]["median_pcg_iters"])
    return out


def save_params(path, params, meta):
    np.savez(path, params=np.asarray(params, dtype=np.float32), meta=json.dumps(meta))


def load_params(path):
    d = np.load(path, allow_pickle=False)
    return d["params"], json.loads(str(d["meta"]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=100, help="training scenes (2 instances each)")
    ap.add_argument("--val", type=int, default=4, help="validation scenes (2 instances each)")
    ap.add_argument("--heldout", type=int, default=10, help="held-out scenes (2 instances each)")
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--lrs", default="1e-3,3e-3")
    ap.add_argument("--kp", type=int, default=4)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--n-cams", type=int, default=None, help="fix the camera count (default U[2000, 8000])")
    ap.add_argument("--out", default="precond_weights.npz")
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    t0 = time.time()
    train_inst = make_instances(range(args.train), args.workers, args.n_cams)
    val_inst = make_instances(range(100, 100 + args.val), args.workers, args.n_cams)
    held = make_instances(range(200, 200 + args.heldout), args.workers, args.n_cams)
    t_gen = time.time() - t0
    print(f"instances: {len(train_inst)} training, {len(val_inst)} validation, {len(held)} held-out "
          f"in {t_gen:.0f} s", flush=True)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import paper_2307_08383_gb300 as B
    lrs = [float(x) for x in args.lrs.split(",")]
    t1 = time.time()
    net, params, tinfo = train(B, train_inst, val_inst, epochs=args.epochs, lrs=lrs, kp=args.kp,
                               log=lambda m: print(m, flush=True))
    t_train = time.time() - t1
    rows = evaluate(B, net, held)
    summ = summarize(rows)
    meta = {"train_instances": len(train_inst), "val_instances": len(val_inst), "heldout_instances": len(held),
            "epochs": args.epochs, "lrs": lrs, "kp": args.kp, "instance_seconds": t_gen,
            "train_seconds": t_train, **tinfo, "heldout": summ}
    save_params(args.out, params, meta)
    if args.report:
        with open(args.report, "w") as f:
            json.dump({"meta": meta, "rows": rows}, f, indent=1)
    print(json.dumps(summ))


if __name__ == "__main__":
    main()
