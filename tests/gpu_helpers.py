"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from oracle import muffin_oracle as mo
from paper_1602_08847_gb300 import synth


def small_cube(n, L, J, seed, n_src=6, n_ant=16):
    return synth.make_cube(synth.CubeConfig("t", n=n, nchan=L, n_src=n_src, n_ant=n_ant, nscales=J, seed=seed))


def problem(cube, J, gen, mu_s, mu_l, tau=None, sigma=1.0, rho=1.0, w=None, dictionary="iuwt"):
    p = mo.make_problem(cube.dirty, cube.psf, J, gen=gen, mu_s=mu_s, mu_l=mu_l, sigma=sigma, rho=rho, w=w,
                        tau=tau, dictionary=dictionary)
    return p


def gpu_solver(cube, p, fine_levels=-1, power_iters=0):
    from paper_1602_08847_gb300.muffin import Muffin
    return Muffin(torch.from_numpy(cube.dirty).cuda(), torch.from_numpy(cube.psf).cuda(), nscales=p.J, gen=p.gen,
                  mu_s=p.mu_s, mu_l=p.mu_l, tau=p.tau, sigma=p.sigma, rho=p.rho,
                  weights=None if np.all(p.w == 1.0) else list(p.w), fine_levels=fine_levels,
                  power_iters=power_iters, dictionary=p.dictionary)


def to64(t):
    return t.detach().cpu().numpy().astype(np.float64)


def max_rel(a, b):
    """max |a - b| over max |b| (elementwise error on the scale of the reference)."""
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (scale if scale > 0 else 1.0)


def random_state(p, seed):
    L, n, _ = p.shape
    x, u, v = synth.random_state((L, n, n), mo.ws_planes(p) - 1, seed, scale=float(np.abs(p.y).max()))
    return x, u, v


def one_pass_both(cube, p, seed, fine_levels=-1, n_pass=1):
    """n_pass passes of Algorithm 1 from the same random state on both sides.

    With n_pass >= 2 the second pass reads the adjoints S = W_s^T U and
    T = W_lambda^T V that the kernels of the first pass wrote (the first pass
    reads the ones set_state computed)."""
    x, u, v = random_state(p, seed)
    m = gpu_solver(cube, p, fine_levels)
    m.set_state(torch.from_numpy(x).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), 0)
    m.iterate(n_pass)
    gx, gu, gv, _ = m.get_state()
    torch.cuda.synchronize()
    m.close()
    s = mo.iterate(p, mo.State(x.astype(np.float64), u.astype(np.float64), v.astype(np.float64)), n_pass)
    return (to64(gx), to64(gu), to64(gv)), s
