"""FP64 error of the FP32 CUDA path after 100 passes from zero at the sizes
the benchmark runs: relative L2 error of the cube X <= 1e-4 and relative
objective error <= 1e-6 against the FP64 oracle run for the same passes with
the same step sizes (Algorithm 1; Eqs. 5-14).

Cases:
* 256 x 256 x 64, J = 4, all terms (mu_s = 0.25, mu_lambda = 3): in full
  (when MUFFIN_PRECISION_FULL is set: its oracle runs about 7 minutes).
* 512 x 512 x 256, J = 5, mu_lambda = 0 (channels separate, Sec. 4 first
  step): the GPU runs the whole cube, the oracle channels 0, 128 and 255.
  Measures the drift of the N = 512 FFTs and the J = 5 stencils.
* 64 x 64 x 256, J = 3, all terms: the spectral step's drift at L = 256.
* 256 x 256 x 64 with W_s the union of eight Daubechies bases, mu_lambda = 0:
  in full (the oracle in eight channel slices; when MUFFIN_PRECISION_FULL is
  set).
* the four uneven cubes of the batch (128^2 x 16, 256^2 x 32, 512^2 x 64,
  1024^2 x 8), advanced together in one batch, mu_lambda = 0: the first and
  last channel of each.

The oracle runs are started at the beginning of the session (tests/oracle_jobs.py).
Where only some channels are compared, the objective compared is the oracle's
objective of those channels (their own terms of Eqs. 5-6) at the GPU's and at
the oracle's X.
"""
import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
import oracle_jobs as oj

pytestmark = pytest.mark.gpu
TOL_X, TOL_OBJ = 1e-4, 1e-6


def _solver(cb, c, dictionary="iuwt"):
    from paper_1602_08847_gb300.muffin import Muffin
    return Muffin(torch.from_numpy(cb.dirty).cuda(), torch.from_numpy(cb.psf).cuda(), nscales=c["J"], gen=1,
                  mu_s=oj.MU_S, mu_l=c["mu_l"], tau=c["tau"], sigma=c["sigma"], rho=1.0, dictionary=dictionary)


def _channel_errors(name, cb, c, groups, gx):
    worst_x, worst_o = 0.0, 0.0
    for g, X, obj in groups:
        p = mo.make_problem(cb.dirty[g], cb.psf[g], c["J"], gen=1, mu_s=oj.MU_S, mu_l=c["mu_l"], tau=c["tau"],
                            sigma=c["sigma"], dictionary=c["dictionary"])
        xg = gx[g].astype(np.float64)
        rel = np.linalg.norm(xg - X) / np.linalg.norm(X)
        robj = abs(mo.objective(p, xg) - obj) / abs(obj)
        worst_x, worst_o = max(worst_x, rel), max(worst_o, robj)
    oj.log({"case": name, "passes": oj.N_PASSES, "rel_l2_x": worst_x, "rel_objective": worst_o,
            "channels": [g for g, _, _ in groups]})
    assert worst_x <= TOL_X, worst_x
    assert worst_o <= TOL_OBJ, worst_o


@pytest.mark.parametrize("name", ["256x256x64", "64x64x256"])
def test_100_passes_full_cube(lib, name):
    if name == "256x256x64" and not oj.FULL:
        pytest.skip("the FP64 oracle takes about 7 minutes here: set MUFFIN_PRECISION_FULL=1")
    c, groups = oj.case(name)
    cb = oj.cube(c["cube"])
    m = _solver(cb, c)
    m.iterate(oj.N_PASSES)
    gx = m.get_cube().cpu().numpy().astype(np.float64)
    gobj, _ = m.objective()
    m.close()
    (_, X, obj), = groups
    rel = np.linalg.norm(gx - X) / np.linalg.norm(X)
    robj = abs(gobj - obj) / abs(obj)
    oj.log({"case": name, "passes": oj.N_PASSES, "rel_l2_x": rel, "rel_objective": robj})
    assert rel <= TOL_X, rel
    assert robj <= TOL_OBJ, (gobj, obj)


@pytest.mark.parametrize("name,dictionary", [("512x512x256_mu_l0", "iuwt"), ("union_256x256x64_mu_l0", "union")])
def test_100_passes_channels_separate(lib, name, dictionary):
    if dictionary == "union" and not oj.FULL:
        pytest.skip("the FP64 oracle of the union takes about 15 minutes of host time: set MUFFIN_PRECISION_FULL=1")
    c, groups = oj.case(name)
    cb = oj.cube(c["cube"])
    m = _solver(cb, c, dictionary)
    m.iterate(oj.N_PASSES)
    gx = m.get_cube().cpu().numpy()
    m.close()
    torch.cuda.empty_cache()
    _channel_errors(name, cb, c, groups, gx)


def test_100_passes_batched_uneven_cubes(lib):
    from paper_1602_08847_gb300.muffin import Batch
    cases = [oj.case("batch_" + n) for n in oj.BATCH]
    cubes = [oj.cube(n) for n in oj.BATCH]
    ms = [_solver(cb, c) for cb, (c, _) in zip(cubes, cases)]
    b = Batch(ms)
    b.iterate(oj.N_PASSES)
    xs = [m.get_cube().cpu().numpy() for m in ms]
    b.close()
    for m in ms:
        m.close()
    torch.cuda.empty_cache()
    for n, cb, (c, groups), gx in zip(oj.BATCH, cubes, cases, xs):
        _channel_errors("batch_" + n, cb, c, groups, gx)
