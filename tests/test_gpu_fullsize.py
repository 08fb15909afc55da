"""One pass of Algorithm 1 at the full sizes the benchmark uses, checked on
sampled outputs that the FP64 oracle can compute one channel or one pixel at
a time (the whole cube would take the oracle minutes).

512 x 512 x 256 (J = 5) and 256 x 256 x 64 (J = 4), graph-launched passes as
bench.py times them.  Random non-trivial states (X >= 0, |U|, |V| <= 1).
"""
import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
from paper_1602_08847_gb300 import synth
from gpu_helpers import max_rel
import oracle_jobs as oj

pytestmark = pytest.mark.gpu
TOL1 = 2e-5


def _setup(name):
    cube = oj.cube(name)      # generated once per session (shared with the precision tests)
    cfg = cube.cfg
    L, n, J = cfg.nchan, cfg.n, cfg.nscales
    hh = mo.psf_multiplier(cube.psf)
    # step sizes from closed-form norms (the oracle's own power method would take minutes here)
    beta = 1.01 * float(np.max(np.abs(hh) ** 2))
    l2 = mo.dual_norm2(0.25, 3.0, 1.01 * mo.iuwt_norm2_closed_form(n, J, 1))
    tau, sigma, rho, _ = mo.condat_steps(beta, l2, 1.0)
    return cube, hh, tau, sigma


def _gpu_pass(cube, tau, sigma, x, u, v):
    from paper_1602_08847_gb300.muffin import Muffin
    cfg = cube.cfg
    m = Muffin(torch.from_numpy(cube.dirty).cuda(), torch.from_numpy(cube.psf).cuda(), nscales=cfg.nscales, gen=1,
               mu_s=0.25, mu_l=3.0, tau=tau, sigma=sigma, rho=1.0)
    m.set_state(torch.from_numpy(x).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), 0)
    m.iterate(1)
    gx, gu, gv, _ = m.get_state()
    out = (gx.cpu().numpy(), gu.cpu().numpy(), gv.cpu().numpy())
    m.close()
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("name,chans", [("512x512x256", [0, 77, 255]), ("256x256x64", [0, 31, 63])])
def test_full_size_pass_on_sampled_channels(lib, name, chans):
    """X and every plane of U of sampled channels after one pass from a random state."""
    cube, hh, tau, sigma = _setup(name)
    L, n, J = cube.cfg.nchan, cube.cfg.n, cube.cfg.nscales
    x, u, v = synth.random_state((L, n, n), J, seed=17, scale=float(np.abs(cube.dirty).max()))
    gx, gu, _ = _gpu_pass(cube, tau, sigma, x, u, v)
    C = mo.dct_matrix(L)
    for l in chans:
        xl = x[l].astype(np.float64)
        grad = mo.apply_Ht(mo.apply_H(xl[None], hh[l:l + 1]) - cube.dirty[l:l + 1].astype(np.float64), hh[l:l + 1])[0]
        S = mo.iuwt_adjoint(u[l].astype(np.float64), J, 1)
        T = np.tensordot(C[:, l], v.astype(np.float64), axes=(0, 0))       # column l of V W_lambda^T
        xt = mo.positive(xl - tau * (grad + 0.25 * S + 3.0 * T))
        ut = mo.sat(u[l].astype(np.float64) + sigma * 0.25 * mo.iuwt_analysis(2 * xt - xl, J, 1))
        assert max_rel(gx[l].astype(np.float64), xt) < TOL1, l
        for j in range(J + 1):
            assert max_rel(gu[l, j].astype(np.float64), ut[j]) < TOL1, (l, j)


@pytest.mark.parametrize("name", ["512x512x256", "256x256x64"])
def test_full_size_pass_on_sampled_pixels(lib, name):
    """V (the spectral dual) at sampled pixels after one pass, with U = 0 so that
    the spatial adjoint vanishes and every channel's X~ at a pixel follows from
    its gradient alone."""
    cube, hh, tau, sigma = _setup(name)
    L, n, J = cube.cfg.nchan, cube.cfg.n, cube.cfg.nscales
    x, _, v = synth.random_state((L, n, n), J, seed=18, scale=float(np.abs(cube.dirty).max()))
    u = np.zeros((L, J + 1, n, n), dtype=np.float32)
    _, gu, gv = _gpu_pass(cube, tau, sigma, x, u, v)
    rng = np.random.Generator(np.random.PCG64(5))
    pix = [(int(a), int(b)) for a, b in rng.integers(0, n, (6, 2))]
    x64 = x.astype(np.float64)
    grad = mo.gradient(x64, cube.dirty.astype(np.float64), hh, np.ones(L))
    v64 = v.astype(np.float64)
    T = mo.spectral_adjoint(v64[:, [p[0] for p in pix], [p[1] for p in pix]][:, :, None])[:, :, 0]
    for k, (py, px) in enumerate(pix):
        xs = x64[:, py, px]
        xt = mo.positive(xs - tau * (grad[:, py, px] + 3.0 * T[:, k]))
        vt = mo.sat(v64[:, py, px] + sigma * 3.0 * (mo.dct_matrix(L) @ (2 * xt - xs)))
        assert max_rel(gv[:, py, px].astype(np.float64), vt) < TOL1, (py, px)
