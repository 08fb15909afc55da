"""Training and evaluation of the learned warm start.

Pairs: for a seeded synthetic cube (synth.make_cube), the dirty cube and the
state Algorithm 1 reaches after a fixed number of passes from X = U = V = 0
(by default 500): the cube X and the J+1 planes of the wavelet dual U.  The
network (net.WarmStartNet with J + 2 output maps) is trained on such pairs
with its own CUDA kernels.  Evaluation: on held-out seeds, the passes and the
time Algorithm 1 needs to reach a relative objective error of 1e-4 (against
F*, the objective after a long run) from the zero state and from the
network's (X, U), with V = 0.

Why U: from the state after 500 passes, the method needs about 500 fewer
passes to reach 1e-4 than from zero; from that X alone, with U = V = 0, it
needs as many as from zero.  The slow part of the iteration is the wavelet
dual, chiefly its finest plane.

Usage (one GPU):
    python -m paper_1602_08847_gb300.warmstart --train-seeds 1000:3000 \
        --eval-seeds 5000:5200 --epochs 2 --out <weights.npy>
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np
import torch

from . import synth
from .muffin import Muffin
from .net import WarmStartNet, n_params, warm_start

MU_S, MU_L = 0.25, 3.0


def cube_stream(cfg: str, seeds, workers: int):
    """(seed, dirty, psf) float32 arrays, generated by a spawn pool in seed order."""
    seeds = list(seeds)
    if workers <= 1:
        for s in seeds:
            yield synth.cube_arrays((cfg, s))
        return
    with mp.get_context("spawn").Pool(workers) as pool:
        yield from pool.imap(synth.cube_arrays, [(cfg, s) for s in seeds], chunksize=2)


def problem(dirty: torch.Tensor, psf: torch.Tensor, nscales: int, fine_levels: int = -1) -> Muffin:
    return Muffin(dirty, psf, nscales=nscales, gen=1, mu_s=MU_S, mu_l=MU_L, fine_levels=fine_levels)


def make_pairs(cfg: str, seeds, iters: int, workers: int, fine_levels: int = -1, input_passes: int = 0):
    """Lists of device tensors for the given seeds: network inputs (the dirty
    cube, or the cube after ``input_passes`` passes), target cubes X (float32)
    and target duals U (bfloat16 [L][J+1][N][N]) after ``iters`` passes."""
    nscales = synth.CONFIGS[cfg].nscales
    dirty, target_x, target_u = [], [], []
    for _, y, h in cube_stream(cfg, seeds, workers):
        yd = torch.from_numpy(y).cuda()
        m = problem(yd, torch.from_numpy(h).cuda(), nscales, fine_levels)
        if input_passes > 0:
            m.iterate(input_passes)
            yd = m.get_cube()
        m.iterate(iters - input_passes)
        x, u, _, _ = m.get_state()
        target_x.append(x)
        target_u.append(u.to(torch.bfloat16))
        dirty.append(yd)
        m.close()
        del u
    torch.cuda.synchronize()
    return dirty, target_x, target_u


def train(net: WarmStartNet, dirty, target_x, target_u, epochs: int, lr: float, lr_final: float, seed: int = 0,
          log_every: int = 100) -> list[float]:
    """Adam over the pairs in a seeded random order, learning rate cosine-decayed
    from lr to lr_final; returns the mean loss of every log_every steps.

    Every log_every steps (and at the end) the network's bounded tensor-core
    waits are checked: a wait that gave up raises MuffinError(TIMEOUT) and
    stops the training (the device already dropped the updates after it)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(dirty)
    total = epochs * n
    loss = torch.zeros(total, dtype=torch.float64, device="cuda")
    step = 0
    for _ in range(epochs):
        for i in rng.permutation(n):
            r = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * step / max(total - 1, 1)))
            net.train_step(dirty[i], target_x[i], target_u[i] if net.n_out > 1 else None, r, loss[step:step + 1])
            step += 1
            if step % log_every == 0:
                net.check()
    net.check()
    curve = loss.cpu().numpy()
    return [float(curve[k:k + log_every].mean()) for k in range(0, total, log_every)]


def passes_to_tolerance(m: Muffin, fstar: float, tol: float, check_every: int, max_passes: int):
    """Iterate until |F - F*| <= tol |F*|; returns (passes or None, GPU ms in passes)."""
    it, ms = 0, 0.0
    f, _ = m.objective()
    if abs(f - fstar) <= tol * abs(fstar):
        return 0, 0.0
    while it < max_passes:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        m.iterate(check_every)
        e1.record()
        f, _ = m.objective()          # synchronises
        ms += e0.elapsed_time(e1)
        it += check_every
        if abs(f - fstar) <= tol * abs(fstar):
            return it, ms
    return None, ms


def prediction_error(net: WarmStartNet, yd: torch.Tensor, hd: torch.Tensor, nscales: int, iters: int,
                     fine_levels: int = -1, input_passes: int = 0) -> dict:
    """RMS error of the network's cube (relative) and of each plane of its U
    against the state Algorithm 1 reaches after ``iters`` passes."""
    m = problem(yd, hd, nscales, fine_levels)
    inp = yd
    if input_passes > 0:
        m.iterate(input_passes)
        inp = m.get_cube()
    m.iterate(iters - input_passes)
    x, u, _, _ = m.get_state()
    m.close()
    px, pu = net.predict(inp)
    out = {"x_rel": float((px - x).norm() / x.norm())}
    if pu is not None:
        out["u_rms"] = [float((pu[:, j] - u[:, j]).pow(2).mean().sqrt()) for j in range(u.shape[1])]
        out["u_ref_rms"] = [float(u[:, j].pow(2).mean().sqrt()) for j in range(u.shape[1])]
    return out


def evaluate_one(net: WarmStartNet | None, y: np.ndarray, h: np.ndarray, nscales: int, fstar_passes: int = 2000,
                 tol: float = 1e-4, check_every: int = 10, fine_levels: int = -1, diagnose_iters: int = 0,
                 input_passes: int = 0) -> dict:
    yd, hd = torch.from_numpy(y).cuda(), torch.from_numpy(h).cuda()
    m = problem(yd, hd, nscales, fine_levels)
    m.iterate(fstar_passes)
    fstar, _ = m.objective()
    m.close()
    out = {"f_star": fstar}
    if net is not None and diagnose_iters > 0:
        out["prediction"] = prediction_error(net, yd, hd, nscales, diagnose_iters, fine_levels, input_passes)
    arms = [("zero", None)] + ([("net", net)] if net is not None else [])
    for name, nn in arms:
        m = problem(yd, hd, nscales, fine_levels)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec = {}
        pre = 0
        if nn is not None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if input_passes > 0:
                m.iterate(input_passes)
                dec = warm_start(m, nn, m.get_cube(), keep_state=True)
            else:
                dec = warm_start(m, nn, yd)
            e1.record()
            torch.cuda.synchronize()
            rec.update(dec)
            rec["start_ms"] = e0.elapsed_time(e1)
            pre = input_passes
        passes, ms = passes_to_tolerance(m, fstar, tol, check_every, 10 * fstar_passes)
        if passes is not None:
            passes += pre
        torch.cuda.synchronize()
        rec.update({"passes": passes, "pass_ms": ms, "wall_ms": 1e3 * (time.perf_counter() - t0)})
        out[name] = rec
        m.close()
    return out


def summarise(results: list[dict]) -> dict:
    s = {"n": len(results)}
    for arm in ("zero", "net"):
        if arm not in results[0]:
            continue
        p = np.array([r[arm]["passes"] if r[arm]["passes"] is not None else np.nan for r in results], float)
        w = np.array([r[arm]["wall_ms"] for r in results], float)
        g = np.array([r[arm]["pass_ms"] + r[arm].get("start_ms", 0.0) for r in results], float)
        s[arm] = {"passes_median": float(np.nanmedian(p)), "passes_mean": float(np.nanmean(p)),
                  "reached": int(np.sum(~np.isnan(p))),
                  "gpu_ms_median": float(np.median(g)), "gpu_ms_mean": float(np.mean(g)),
                  "wall_ms_median": float(np.median(w)), "wall_ms_mean": float(np.mean(w))}
        if arm == "net":
            s[arm]["used"] = int(sum(r["net"]["used"] for r in results))
    if "prediction" in results[0]:
        s["prediction"] = {"x_rel_mean": float(np.mean([r["prediction"]["x_rel"] for r in results]))}
        if "u_rms" in results[0]["prediction"]:
            s["prediction"]["u_rms_mean"] = np.mean([r["prediction"]["u_rms"] for r in results], axis=0).tolist()
            s["prediction"]["u_ref_rms_mean"] = np.mean([r["prediction"]["u_ref_rms"] for r in results],
                                                        axis=0).tolist()
    return s


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_256x256x64.npy")


def load_committed(path: str = WEIGHTS):
    """(WarmStartNet for 64 x 256 x 256 cubes, training record) from the
    weights shipped with the package, or (None, {}) when there are none."""
    if not os.path.exists(path):
        return None, {}
    meta = {}
    rec = os.path.splitext(path)[0] + ".json"
    if os.path.exists(rec):
        with open(rec) as f:
            meta = json.load(f)
    theta = torch.from_numpy(np.load(path).astype(np.float32)).cuda()
    n_out = {n_params(k): k for k in range(1, 9)}[theta.numel()]
    shape = tuple(meta.get("shape", (64, 256, 256)))
    return WarmStartNet(shape, theta=theta, n_out=n_out), meta


def _seeds(spec: str):
    a, b = spec.split(":")
    return range(int(a), int(b))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="256x256x64")
    ap.add_argument("--train-seeds", default="1000:3000")
    ap.add_argument("--eval-seeds", default="5000:5200")
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=2e-5)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--fine-levels", type=int, default=2)
    ap.add_argument("--x-weight", type=float, default=1000.0, help="loss weight of the cube map (U maps: 1)")
    ap.add_argument("--u-weights", default="4,1,1,1,1", help="comma-separated loss weights of the U planes")
    ap.add_argument("--cube-only", action="store_true", help="predict X alone (one output map)")
    ap.add_argument("--diagnose", action="store_true", help="also report the prediction error on the eval seeds")
    ap.add_argument("--input-passes", type=int, default=50,
                    help="network input: the cube after this many plain passes (0: the dirty cube)")
    ap.add_argument("--weights", default=None, help="skip training: evaluate these weights (.npy)")
    ap.add_argument("--out", default=None, help="where to write the trained weights (.npy) and a .json record")
    args = ap.parse_args()

    cfg = synth.CONFIGS[args.config]
    shape = (cfg.nchan, cfg.n, cfg.n)
    n_out = 1 if args.cube_only else cfg.nscales + 2
    lam = [args.x_weight] + [1.0] * (n_out - 1)
    if args.u_weights and n_out > 1:
        uw = [float(v) for v in args.u_weights.split(",")]
        if len(uw) != n_out - 1:
            raise SystemExit(f"--u-weights needs {n_out - 1} values")
        lam = [args.x_weight] + uw
    record = {"config": args.config, "shape": shape, "n_out": n_out, "out_weight": lam, "iters": args.iters,
              "epochs": args.epochs,
              "train_seeds": args.train_seeds, "eval_seeds": args.eval_seeds, "lr": args.lr,
              "lr_final": args.lr_final, "init_seed": args.init_seed, "mu_s": MU_S, "mu_l": MU_L,
              "input_passes": args.input_passes}
    if args.weights:
        theta = torch.from_numpy(np.load(args.weights).astype(np.float32)).cuda()
    else:
        t0 = time.perf_counter()
        dirty, target_x, target_u = make_pairs(args.config, _seeds(args.train_seeds), args.iters, args.workers,
                                               args.fine_levels, args.input_passes)
        record["pairs_s"] = time.perf_counter() - t0
        net = WarmStartNet(shape, training=True, theta=torch.from_numpy(synth.net_init(args.init_seed, n_out)).cuda(),
                           n_out=n_out, out_weight=lam)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        record["loss_curve"] = train(net, dirty, target_x, target_u, args.epochs, args.lr, args.lr_final,
                                     seed=args.init_seed)
        torch.cuda.synchronize()
        record["train_s"] = time.perf_counter() - t0
        record["train_steps"] = args.epochs * len(dirty)
        theta = net.get_params()
        net.close()
        del dirty, target_x, target_u
        torch.cuda.empty_cache()
        if args.out:
            np.save(args.out, theta.cpu().numpy())
    n_out = {n_params(k): k for k in range(1, 9)}[theta.numel()]
    net = WarmStartNet(shape, theta=theta, n_out=n_out)
    results = []
    for _, y, h in cube_stream(args.config, _seeds(args.eval_seeds), args.workers):
        results.append(evaluate_one(net, y, h, cfg.nscales, fine_levels=args.fine_levels,
                                    diagnose_iters=args.iters if args.diagnose else 0,
                                    input_passes=args.input_passes))
    record["eval"] = summarise(results)
    record["per_seed"] = results
    if args.out:
        with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
            json.dump(record, f, indent=1)
    print(json.dumps({k: v for k, v in record.items() if k != "per_seed"}))


if __name__ == "__main__":
    main()
