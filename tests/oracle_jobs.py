"""Long FP64 oracle runs of the precision tests, started in worker processes at
the beginning of a GPU test session so that they overlap the other GPU tests.

The oracle runs whole (Algorithm 1, 100 passes from zero) on every case; where
a case sets mu_lambda = 0 the channels of the cube evolve independently
(Sec. 4, first step; pinned in test_oracle.py by
test_zero_spectral_weight_separates_channels), so the oracle runs on channel
slices, in parallel.  Step sizes come from closed-form norms and Condat's rule
(the oracle's power method would take minutes at these sizes), computed once
here and passed to both sides.

Workers are started with the "spawn" method and import only numpy, the oracle
and the seeded input generator (no torch, no CUDA).
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from oracle import muffin_oracle as mo
from paper_1602_08847_gb300 import synth

N_PASSES = 100
MU_S, MU_L = 0.25, 3.0

_cubes: dict = {}
_cases: dict = {}
_pool = None


def cube(name_or_cfg):
    """Seeded synthetic cube, generated once per process."""
    key = name_or_cfg if isinstance(name_or_cfg, str) else name_or_cfg.name
    if key not in _cubes:
        _cubes[key] = synth.make_cube(name_or_cfg)
    return _cubes[key]


def closed_form_steps(c, J: int, gen: int, mu_s: float, mu_l: float, dictionary: str = "iuwt"):
    """(tau, sigma): beta = 1.01 max_l |hhat_l|^2, ||W_s||^2 = 1.01 x its closed form
    (the IUWT's transfer-function maximum, 1 for the union of orthonormal bases)."""
    hh = mo.psf_multiplier(c.psf)
    beta = 1.01 * float(np.max(np.abs(hh) ** 2))
    ws2 = 1.01 * (1.0 if dictionary == "union" else mo.iuwt_norm2_closed_form(c.cfg.n, J, gen))
    tau, sigma, _, _ = mo.condat_steps(beta, mo.dual_norm2(mu_s, mu_l, ws2), 1.0)
    return tau, sigma


def _oracle_run(y, psf, J, gen, mu_s, mu_l, tau, sigma, n_iter, dictionary):
    """Worker: Algorithm 1 in FP64 from zero; (X, objective at X)."""
    p = mo.make_problem(y, psf, J, gen=gen, mu_s=mu_s, mu_l=mu_l, tau=tau, sigma=sigma, dictionary=dictionary)
    s = mo.iterate(p, mo.zero_state(p), n_iter)
    return s.X, mo.objective(p, s.X)


CUBE_64x64x256 = synth.CubeConfig("64x64x256", n=64, nchan=256, n_src=40, n_ant=60, nscales=3, seed=4)
BATCH = ("128x128x16", "256x256x32", "512x512x64", "1024x1024x8")


# Two cases take the oracle many minutes: the full 256 x 256 x 64 cube with
# every term (all channels coupled, so one process: about 7 minutes for 100
# passes on one host core) and the union of bases on it (the oracle's DWT
# matrices: about 15 minutes of host time in 8 slices).  They run when
# MUFFIN_PRECISION_FULL is set; the other cases always run.
FULL = bool(os.environ.get("MUFFIN_PRECISION_FULL"))


def _plan():
    """case -> dict(cube, J, gen, mu_l, dictionary, groups): groups are channel lists, one job each."""
    plan = {
        "64x64x256": dict(cube=CUBE_64x64x256, J=3, mu_l=MU_L, dictionary="iuwt", groups=[None]),
        "512x512x256_mu_l0": dict(cube="512x512x256", J=5, mu_l=0.0, dictionary="iuwt", groups=[[0], [128], [255]]),
    }
    for name in BATCH:
        L = synth.CONFIGS[name].nchan
        plan["batch_" + name] = dict(cube=name, J=4, mu_l=0.0, dictionary="iuwt", groups=[[0], [L - 1]])
    if FULL:
        plan["256x256x64"] = dict(cube="256x256x64", J=4, mu_l=MU_L, dictionary="iuwt", groups=[None])
        plan["union_256x256x64_mu_l0"] = dict(cube="256x256x64", J=4, mu_l=0.0, dictionary="union",
                                              groups=[list(range(8 * k, 8 * k + 8)) for k in range(8)])
    return plan


def start():
    """Submit every oracle job (largest first); idempotent."""
    global _pool
    if _pool is not None:
        return
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"           # one thread per worker: the workers share the host's cores
    try:
        # half the host's cores: the GPU tests of this process run their own oracle checks meanwhile
        _pool = cf.ProcessPoolExecutor(max_workers=max(2, min(8, (os.cpu_count() or 4) // 2)),
                                       mp_context=mp.get_context("spawn"))
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    jobs = []
    for case, c in _plan().items():
        cb = cube(c["cube"])
        tau, sigma = closed_form_steps(cb, c["J"], 1, MU_S, c["mu_l"], c["dictionary"])
        futs = []
        for g in c["groups"]:
            y = cb.dirty if g is None else cb.dirty[g]
            psf = cb.psf if g is None else cb.psf[g]
            cost = y.size * (8 if c["dictionary"] == "union" else 1) * (1 if c["mu_l"] == 0 else 2)
            futs.append([cost, (y, psf, c["J"], 1, MU_S, c["mu_l"], tau, sigma, N_PASSES, c["dictionary"]), None])
            jobs.append(futs[-1])
        _cases[case] = dict(c, tau=tau, sigma=sigma, jobs=futs)
    for j in sorted(jobs, key=lambda j: -j[0]):
        j[2] = _pool.submit(_oracle_run, *j[1])


def case(name: str):
    """(plan entry with tau, sigma, and per group (channels, X, objective)) of a case; waits for its jobs."""
    start()
    c = _cases[name]
    out = []
    for g, j in zip(c["groups"], c["jobs"]):
        X, obj = j[2].result()
        out.append((g, X, obj))
    return c, out


def log(record: dict) -> None:
    """Append a measured error to the file named by MUFFIN_PRECISION_LOG, if set."""
    path = os.environ.get("MUFFIN_PRECISION_LOG")
    if path:
        import json
        with open(path, "a") as f:
            f.write(json.dumps(record) + "\n")
