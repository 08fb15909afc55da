"""Throughput of one MUFFIN primal-dual pass (Algorithm 1) over a whole cube.

Default workload: the 512 x 512 x 256 cube (200 sources, 10% point-like,
128 antennas, IUWT 5 scales, generation 1, mu_s = 0.25, mu_lambda = 3, step
sizes from the power method and Condat's rule), FP32 iterates.  A step is one
pass of Algorithm 1 over the cube; the metric is voxel-iterations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl muffin|reference]

Under torchrun each rank solves its own cube (seed + rank): weak scaling, no
collective on the data path; the step time is the max over ranks.
--impl reference times the FP64 oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iter/s"
WORKLOAD = "512x512x256 cube, 200 sources (10% point), 128 antennas, IUWT J=5 gen1, mu_s=0.25, mu_l=3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="muffin", choices=["muffin", "reference"])
    ap.add_argument("--config", default="512x512x256")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ttt", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-union", action="store_true")
    ap.add_argument("--ttt-seeds", type=int, default=0,
                    help="also rerun the warm-start evaluation live on this many held-out seeds (5000 ...)")
    ap.add_argument("--fine-levels", type=int, default=-1,
                    help="wavelet split (levels on halo tiles); -1: chosen by timing at set-up")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle timing (host cores)
# One timing process: builds a channel slice of the workload, runs one untimed
# pass, reports "ready", waits for "go" on stdin (so that the processes of the
# all-core mode time their passes together), times `steps` passes, then times
# the spectral step (the oracle's dense L x L transform and its adjoint) on a
# pixel sample at the slice's L and at the workload's full L, which lets the
# per-voxel cost be carried over to the full channel count.
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import muffin_oracle as mo
from paper_1602_08847_gb300 import synth
cfg = synth.CONFIGS[{cfg!r}]
full_L = cfg.nchan
sl = synth.CubeConfig(**{{**cfg.as_dict(), "nchan": {chan0} + {nchan}}})
cube = synth.make_cube(sl)
y, psf = cube.dirty[{chan0}:], cube.psf[{chan0}:]
p = mo.make_problem(y, psf, cfg.nscales, gen=1, mu_s=0.25, mu_l=3.0, tau=1e-3)
s = mo.zero_state(p)
s = mo.iterate(p, s, 1)
print("ready", flush=True)
sys.stdin.readline()
times = []
t_start = time.perf_counter()
for _ in range({steps}):
    t0 = time.perf_counter(); s = mo.iterate(p, s, 1); times.append(time.perf_counter() - t0)
t_end = time.perf_counter()
def spec_cost(L, npix=4096, reps=3):
    v = np.random.Generator(np.random.PCG64(1)).standard_normal((L, npix))
    t0 = time.perf_counter()
    for _ in range(reps):
        mo.spectral_adjoint(v); mo.spectral_analysis(v)
    return (time.perf_counter() - t0) / reps / (L * npix)
print(json.dumps({{"times": times, "wall": t_end - t_start, "voxels": {nchan} * cfg.n * cfg.n,
                  "spec_slice": spec_cost({nchan}), "spec_full": spec_cost(full_L)}}))
"""

SINGLE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_time(cfg_name: str, nchan: int, steps: int, procs: int = 1) -> dict:
    """The FP64 oracle, single-threaded, in `procs` concurrent processes, each on
    its own nchan-channel slice of the workload (channels k*nchan ...), timed
    together.  value: voxel-iterations per second of all processes; full_L_value:
    the same with the slice's spectral cost per voxel replaced by the full
    channel count's (the oracle's spectral step is a dense L x L product)."""
    env = dict(os.environ, **SINGLE_THREAD)
    ps = []
    for k in range(procs):
        code = ORACLE_SNIPPET.format(root=ROOT, cfg=cfg_name, nchan=nchan, steps=steps, chan0=k * nchan)
        ps.append(subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                                   stderr=subprocess.PIPE, text=True, env=env))
    try:
        for pr in ps:
            ln = pr.stdout.readline()
            if ln.strip() != "ready":
                raise RuntimeError("oracle process failed: " + pr.stderr.read()[-2000:])
        for pr in ps:
            pr.stdin.write("go\n")
            pr.stdin.flush()
        outs = []
        for pr in ps:
            out, err = pr.communicate(timeout=3600)
            if pr.returncode != 0:
                raise RuntimeError(err[-2000:])
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for pr in ps:
            if pr.poll() is None:
                pr.kill()
    wall = max(o["wall"] for o in outs)
    vox = sum(o["voxels"] for o in outs) * steps
    per_vox = wall / (vox / procs)                   # seconds per voxel-iteration of one process
    full = per_vox + max(o["spec_full"] - o["spec_slice"] for o in outs)
    return {"value": vox / wall, "seconds": wall, "steps": steps, "voxels": outs[0]["voxels"], "procs": procs,
            "full_L_value": procs / full}


def reference_arm(args, rank: int) -> None:
    if rank != 0:
        return
    from paper_1602_08847_gb300 import synth
    cfg = synth.CONFIGS[args.config]
    nchan = 4
    res = oracle_time(args.config, nchan, max(args.steps, 1))
    sample = (f"{cfg.n}x{cfg.n}x{nchan} slice of the workload (same N, J, sources, antennas; first {nchan} "
              f"channels), {res['steps']} passes after 1 untimed, numpy FP64, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": res["value"], "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "host_cpus": os.cpu_count(), "extrapolated": False,
                             "full_L_value": res["full_L_value"],
                             "full_L_note": f"per-voxel cost with the spectral step at L = {cfg.nchan} "
                                            "(timed on a pixel sample) in place of the slice's"},
            "e2e": {"value": res["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(cfg_name: str) -> dict:
    """The oracle on the host cores: one thread, and every core (one single-threaded
    process per core, each on its own 16-channel slice).  The headline value is
    the single-thread rate carried over to the full channel count."""
    from paper_1602_08847_gb300 import synth
    cfg = synth.CONFIGS[cfg_name]
    nchan, steps = 16, 3
    cores = os.cpu_count() or 1
    one = oracle_time(cfg_name, nchan, steps, 1)
    procs = max(1, min(cores, cfg.nchan // nchan))
    allc = oracle_time(cfg_name, nchan, steps, procs)
    return {"value": one["full_L_value"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(), "host_cpus": cores, "extrapolated": True,
            "sample": (f"{cfg.n}x{cfg.n}x{nchan} slice of the workload (first {nchan} channels), {steps} passes "
                       f"after 1 untimed, numpy FP64, 1 thread; per-voxel cost carried over to L = {cfg.nchan} by "
                       f"timing the oracle's spectral step at L = {cfg.nchan} and L = {nchan} on 4096 pixels"),
            "single": {"value": one["value"], "full_L_value": one["full_L_value"], "threads": 1,
                       "seconds": one["seconds"]},
            "all_core": {"value": allc["value"], "full_L_value": allc["full_L_value"], "processes": procs,
                         "threads_per_process": 1, "seconds": allc["seconds"],
                         "sample": f"{procs} concurrent processes, each on its own {nchan}-channel slice "
                                   f"(channels {nchan} k .. {nchan} k + {nchan - 1}), timed together"}}


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    from paper_1602_08847_gb300 import replicas
    rank, world, local = replicas.world()
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import numpy as np
    import torch
    from paper_1602_08847_gb300 import synth
    from paper_1602_08847_gb300.muffin import Muffin, solve

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return replicas.max_over_ranks(v, dist, "cuda")

    cfg = synth.CONFIGS[args.config]
    cube = synth.make_cube(cfg, seed=replicas.rank_seed(cfg.seed, rank))
    L, n = cfg.nchan, cfg.n
    voxels = L * n * n
    kw = dict(nscales=cfg.nscales, gen=1, mu_s=0.25, mu_l=3.0, fine_levels=args.fine_levels)
    m = Muffin(torch.from_numpy(cube.dirty).cuda(), torch.from_numpy(cube.psf).cuda(), **kw)
    stream = torch.cuda.current_stream()

    m.iterate(args.warmup)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        m.iterate(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms / args.steps
    value = replicas.aggregate_throughput(voxels * args.steps, world, ms / 1e3)
    launches = m.kernels_per_iteration() * args.steps
    fine_levels, cluster = m.tiling()
    fine_threads, coarse_threads = m.block_threads()

    # per-stage device times over a second timed region (events between stages on the launching stream)
    names = [s for s in __import__("paper_1602_08847_gb300.muffin", fromlist=["stage_names"]).stage_names()]
    stage_ms = m.iterate_timed(args.steps)
    stage_bytes = m.stage_bytes()
    k = int(np.argmax(stage_ms))
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    ach = stage_bytes[k] * args.steps / (stage_ms[k] / 1e3) / 1e9
    J = cfg.nscales
    step_bytes = (8 * J + 30) * voxels
    roofline = {"bound": "hbm", "kernel": names[k], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_src, "traffic": None,
                "stage_ms_per_step": {nm: t / args.steps for nm, t in zip(names, stage_ms)},
                "stage_gbs": {nm: (b * args.steps / (t / 1e3) / 1e9 if t > 0 else 0.0)
                              for nm, b, t in zip(names, stage_bytes, stage_ms)},
                "step": {"algorithmic_bytes": step_bytes, "bytes_per_voxel": 8 * J + 30,
                         "achieved": step_bytes / (ms_step / 1e3) / 1e9,
                         "frac": step_bytes / (ms_step / 1e3) / 1e9 / peak}}
    traffic_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_file):
        with open(traffic_file) as f:
            tr = json.load(f)
        if tr.get("kernel") == names[k] and tr.get("workload") == args.config:
            roofline["traffic"] = tr.get("bytes_per_launch")
    m.close()
    del m

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "voxels_per_gpu": voxels, "nscales": J, "iuwt_gen": 1,
                       "l2": "inputs larger than L2 (state ~2.4 GB per cube)", "parallelism": f"replicas{world}",
                       "graph": True, "iuwt_fine_levels": fine_levels, "iuwt_cluster": cluster,
                       "iuwt_block_threads": [fine_threads, coarse_threads]},
            "roofline": roofline, "gpu_launches": launches, "clocks": clk.summary()}

    # end to end through the public call: pinned host cubes in, X back to host
    if not args.no_e2e:
        hd = torch.from_numpy(cube.dirty).pin_memory()
        hp = torch.from_numpy(cube.psf).pin_memory()
        solve(hd, hp, 1, **kw)          # warm the allocator and the kernels
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        x = solve(hd, hp, args.steps, **kw)
        torch.cuda.synchronize()
        t = max_over_ranks(time.perf_counter() - t0)
        line["e2e"] = {"value": voxels * world * args.steps / t, "unit": METRIC,
                       "h2d_bytes_per_step": (hd.numel() + hp.numel()) * 4 / args.steps,
                       "d2h_bytes_per_step": x.numel() * 4 / args.steps,
                       "what": f"muffin.solve(): H2D of y and PSF, set-up (FP64 spectra, power method), "
                               f"{args.steps} passes, D2H of X; one call"}

    # four uneven cubes advanced together: one graph launch per pass (muffin_batch) vs one by one
    # the comparison dictionary of Sec. 4: the same pass with W_s = union of eight Daubechies bases
    if not args.no_union and rank == 0:
        cu = synth.make_cube("256x256x64")
        mu = Muffin(torch.from_numpy(cu.dirty).cuda(), torch.from_numpy(cu.psf).cuda(), nscales=4,
                    mu_s=0.25, mu_l=3.0, dictionary="union")
        mi = Muffin(torch.from_numpy(cu.dirty).cuda(), torch.from_numpy(cu.psf).cuda(), nscales=4,
                    mu_s=0.25, mu_l=3.0)
        res = {}
        for name, m_ in (("union", mu), ("iuwt", mi)):
            m_.iterate(10)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            m_.iterate(50)
            s1.record()
            torch.cuda.synchronize()
            res[name] = s0.elapsed_time(s1) / 50
        vox_b = cu.cfg.nchan * cu.cfg.n * cu.cfg.n
        line["union_dictionary"] = {"workload": "256x256x64, J=4, W_s = union of 8 Daubechies bases (db1-db8)",
                                    "ms_per_step": res["union"], "value": vox_b / (res["union"] * 1e-3),
                                    "unit": METRIC, "iuwt_ms_per_step": res["iuwt"],
                                    "kernels_per_step": mu.kernels_per_iteration()}
        mu.close()
        mi.close()

    if not args.no_batch and rank == 0:
        from paper_1602_08847_gb300.muffin import Batch
        ms = []
        vox_c = 0
        for name in ("128x128x16", "256x256x32", "512x512x64", "1024x1024x8"):
            cc = synth.make_cube(name)
            ms.append(Muffin(torch.from_numpy(cc.dirty).cuda(), torch.from_numpy(cc.psf).cuda(),
                             nscales=cc.cfg.nscales, gen=1, mu_s=0.25, mu_l=3.0))
            vox_c += cc.cfg.nchan * cc.cfg.n * cc.cfg.n
        b = Batch(ms)
        b.iterate(5)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        b.iterate(args.steps)
        s1.record()
        torch.cuda.synchronize()
        t_batch = s0.elapsed_time(s1) / args.steps
        for m_ in ms:
            m_.iterate(2)
        torch.cuda.synchronize()
        s0.record()
        for _ in range(args.steps):
            for m_ in ms:
                m_.iterate(1)
        s1.record()
        torch.cuda.synchronize()
        t_seq = s0.elapsed_time(s1) / args.steps
        # the same cubes, one persistent launch per pass
        t_pers = None
        try:
            b.set_mode("persistent")
            b.iterate(5)
            b.check()
            s0.record()
            b.iterate(args.steps)
            s1.record()
            torch.cuda.synchronize()
            b.check()
            t_pers = s0.elapsed_time(s1) / args.steps
        except Exception as exc:  # noqa: BLE001
            t_pers = "failed: " + str(exc)[:200]
        line["batched"] = {"workload": "128^2x16 + 256^2x32 + 512^2x64 + 1024^2x8, 40 sources, 60 antennas, J=4, "
                                       "seeds 11-14, splits chosen per cube by the set-up autotuner",
                           "voxels": vox_c, "ms_per_step": t_batch, "value": vox_c / (t_batch / 1e3),
                           "unit": METRIC, "one_by_one_ms_per_step": t_seq,
                           "persistent_ms_per_step": t_pers,
                           "tilings": [m_.tiling() for m_ in ms]}
        b.close()
        for m_ in ms:
            m_.close()
        del ms
        torch.cuda.empty_cache()

    # time to 1e-4 relative objective on the 256x256x64 cube (F* from 2000 passes), from the zero
    # state and from the learned warm start (the committed network, if present)
    if not args.no_ttt and rank == 0:
        from paper_1602_08847_gb300 import warmstart as ws
        cb = synth.make_cube("256x256x64")
        net, meta = ws.load_committed()
        r = ws.evaluate_one(net, cb.dirty, cb.psf, 4, input_passes=meta.get("input_passes", 0) if net else 0)
        ttt = {"workload": "256x256x64, 40 sources, 60 antennas, J=4 (seed 2, not a training seed)",
               "f_star": r["f_star"], "f_star_passes": 2000, "check_every": 10, "zero": r["zero"]}
        if net is not None:
            ttt["warm"] = r["net"]
            ttt["warm"]["input_passes"] = meta.get("input_passes", 0)
            ttt["warm_over_zero_gpu_ms"] = (r["net"]["pass_ms"] + r["net"]["start_ms"]) / r["zero"]["pass_ms"]
            if meta.get("eval"):
                ttt["held_out_record"] = {"seeds": meta.get("eval_seeds"), "summary": meta["eval"],
                                          "what": "evaluation in the committed training record "
                                                  "(paper_1602_08847_gb300/weights/warmstart_256x256x64.json)",
                                          "command": meta.get("command")}
            if args.ttt_seeds > 0:
                live = []
                for seed in range(5000, 5000 + args.ttt_seeds):
                    _, y_s, h_s = synth.cube_arrays(("256x256x64", seed))
                    live.append(ws.evaluate_one(net, y_s, h_s, 4, input_passes=meta.get("input_passes", 0)))
                ttt["held_out_live"] = {"seeds": f"5000:{5000 + args.ttt_seeds}", "summary": ws.summarise(live)}
            net.close()
        line["time_to_rel_obj_1e-4"] = ttt

    if rank == 0 and not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline(args.config)
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "unit": METRIC, "cores": 1, "kind": "oracle",
                                    "sample": "failed: " + str(exc)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
