"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances: FP32 iterates against FP64.  One pass from a random state:
max |gpu - oracle| <= 2e-5 of the largest magnitude of each array (FP32 FFTs of
up to 2^20 points and 5-level stencils accumulate a few ulp per stage).  After
100 passes from zero: relative L2 error of X <= 1e-4 and relative objective
error <= 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
from gpu_helpers import small_cube, problem, gpu_solver, to64, max_rel, one_pass_both

pytestmark = pytest.mark.gpu
TOL1 = 2e-5


@pytest.mark.parametrize("n,L", [(16, 3), (32, 5), (64, 4), (128, 3), (256, 2), (512, 2), (1024, 1)])
def test_gradient_step_all_sizes(lib, n, L):
    """mu_s = mu_lambda = 0: one pass is X <- (X - tau grad)_+ (FFT path only)."""
    cube = small_cube(n, L, 1, seed=n + L)
    p = problem(cube, 1, 1, 0.0, 0.0)
    (gx, gu, gv), s = one_pass_both(cube, p, seed=3)
    assert max_rel(gx, s.X) < TOL1
    assert gx.min() >= 0.0
    assert np.array_equal(gv, s.V) and np.array_equal(gu, s.U)   # mu = 0: duals untouched


@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("n,L,J,j1", [
    (16, 2, 3, -1), (64, 3, 3, 0), (64, 3, 3, 1), (64, 3, 3, 2), (64, 3, 3, 3), (64, 2, 5, 3),
    (128, 2, 4, 0), (128, 2, 4, 1), (128, 2, 4, 2), (256, 1, 3, 2), (256, 2, 4, -1), (256, 1, 2, -1),
    (512, 1, 5, -1), (1024, 1, 4, -1),
    (256, 2, 4, 1), (512, 1, 5, 2), (512, 1, 4, 2), (1024, 1, 4, 3),
    (64, 3, 0, -1), (256, 2, 0, -1),
])
def test_spatial_pass_matches_oracle(lib, gen, n, L, J, j1):
    """mu_lambda = 0: X and every wavelet plane of U after two passes (the
    second reads the spatial adjoint the first pass's kernels wrote), for every
    tiling split (fine halo tiles / class-permuted coarse sub-images)."""
    cube = small_cube(n, L, max(J, 1), seed=10 + n + J)
    p = problem(cube, J, gen, 0.4, 0.0, tau=None, sigma=2.0)
    (gx, gu, gv), s = one_pass_both(cube, p, seed=5, fine_levels=j1, n_pass=2)
    assert max_rel(gx, s.X) < TOL1
    for j in range(J + 1):
        assert max_rel(gu[:, j], s.U[:, j]) < TOL1, f"plane {j}"
    assert np.abs(gu).max() <= 1.0


@pytest.mark.parametrize("L", [1, 3, 8, 15, 16, 32, 64, 100, 128, 256])
def test_spectral_pass_matches_oracle(lib, L):
    """mu_s = 0: X and V after two passes (dense DCT for L not a power of two or
    below 16, Makhoul FFT-DCT otherwise; the second pass reads the T that the
    first pass's spectral kernel wrote)."""
    cube = small_cube(16, L, 1, seed=40 + L)
    p = problem(cube, 1, 1, 0.0, 0.7, sigma=3.0)
    (gx, gu, gv), s = one_pass_both(cube, p, seed=7, n_pass=2)
    assert max_rel(gx, s.X) < TOL1
    assert max_rel(gv, s.V) < TOL1


@pytest.mark.parametrize("gen", [1, 2])
def test_full_pass_relaxed_weighted(lib, gen):
    """All terms at once with rho != 1 and per-channel weights 1/sigma_l^2."""
    cube = small_cube(64, 6, 3, seed=77)
    w = np.linspace(0.5, 2.0, 6)
    # a step well inside Condat's bound so that rho = 1.3 < delta
    p = problem(cube, 3, gen, 0.3, 1.5, sigma=1.5, rho=1.3, w=w, tau=1e-3)
    (gx, gu, gv), s = one_pass_both(cube, p, seed=9, n_pass=2)
    assert max_rel(gx, s.X) < TOL1
    assert max_rel(gu, s.U) < TOL1
    assert max_rel(gv, s.V) < TOL1


@pytest.mark.parametrize("gen", [1, 2])
def test_100_passes_64x64x8(lib, gen):
    """The 64 x 64 x 8 workload (5 sources, 20 antennas, J = 3, 100 passes from
    zero): rel L2 of X <= 1e-4 and relative objective <= 1e-6 against FP64."""
    from paper_1602_08847_gb300 import synth
    cube = synth.make_cube("64x64x8")
    p = problem(cube, 3, gen, 0.25, 3.0)
    m = gpu_solver(cube, p)
    m.iterate(100)
    gx = to64(m.get_cube())
    gobj, _ = m.objective()
    m.close()
    s = mo.iterate(p, mo.zero_state(p), 100)
    rel = np.linalg.norm(gx - s.X) / np.linalg.norm(s.X)
    obj = mo.objective(p, s.X)
    assert rel <= 1e-4, rel
    assert abs(gobj - obj) / abs(obj) <= 1e-6, (gobj, obj)


@pytest.mark.parametrize("gen", [1, 2])
def test_objective_evaluator(lib, gen):
    """muffin_objective at a given X equals Eqs. 5-6 evaluated in FP64."""
    cube = small_cube(128, 5, 3, seed=21)
    p = problem(cube, 3, gen, 0.3, 0.9, w=np.array([1.0, 0.5, 2.0, 1.5, 0.75]))
    x = np.abs(np.random.Generator(np.random.PCG64(4)).standard_normal((5, 128, 128))).astype(np.float32)
    m = gpu_solver(cube, p)
    m.set_cube(torch.from_numpy(x).cuda())
    tot, terms = m.objective()
    m.close()
    ref = mo.objective_terms(p, x.astype(np.float64))
    for a, b in zip(terms, ref):
        assert abs(a - b) <= 1e-6 * abs(b), (terms, ref)
    assert abs(tot - sum(ref)) <= 1e-6 * abs(sum(ref))


def test_step_sizes_from_power_method(lib):
    cube = small_cube(64, 4, 3, seed=31)
    p = problem(cube, 3, 1, 0.25, 3.0, w=np.array([1.0, 2.0, 0.5, 1.0]))
    m = gpu_solver(cube, p, power_iters=60)
    st = m.step_sizes()
    m.close()
    closed = max(p.w[l] * np.max(np.abs(p.hhat[l]) ** 2) for l in range(4))
    assert abs(st["beta_closed"] - closed) <= 1e-9 * closed
    assert closed * 0.995 <= st["beta"] <= closed * 1.0101
    wn = mo.iuwt_norm2_closed_form(64, 3, 1)
    assert wn * 0.99 <= st["ws_norm2"] <= wn * 1.0101


def test_auto_steps_meet_condat(lib):
    from paper_1602_08847_gb300.muffin import Muffin
    cube = small_cube(64, 4, 2, seed=32)
    m = Muffin(torch.from_numpy(cube.dirty).cuda(), torch.from_numpy(cube.psf).cuda(), nscales=2, mu_s=0.25,
               mu_l=3.0)
    st = m.step_sizes()
    m.close()
    assert 1.0 / st["tau"] - st["sigma"] * st["l_norm2"] > st["beta"] / 2
    delta = 2.0 - 0.5 * st["beta"] / (1.0 / st["tau"] - st["sigma"] * st["l_norm2"])
    assert 0 < st["rho"] < delta


def test_checkpoint_resume_is_bitwise(lib):
    cube = small_cube(256, 4, 4, seed=33)
    p = problem(cube, 4, 1, 0.25, 3.0)
    a = gpu_solver(cube, p)
    a.iterate(50)
    x, u, v, it = a.get_state()
    a.iterate(50)
    x_ref = a.get_cube().clone()
    split = a.tiling()[0]
    a.close()
    b = gpu_solver(cube, p, fine_levels=split)   # same tiling: the split is chosen by timing otherwise
    b.set_state(x, u, v, it)
    b.iterate(50)
    x_b = b.get_cube()
    _, _, _, it_b = b.get_state()
    b.close()
    assert torch.equal(x_ref, x_b) and it_b == 100


def test_two_step_calibration(lib):
    """Sec. 4: mu_lambda = 0 first (channels separate), then mu_lambda > 0 from that X."""
    cube = small_cube(64, 8, 3, seed=34)
    p0 = problem(cube, 3, 1, 0.25, 0.0, tau=2e-3)
    p1 = problem(cube, 3, 1, 0.25, 3.0, tau=2e-3)
    m = gpu_solver(cube, p0)
    m.iterate(30)
    m.set_mu(0.25, 3.0)
    m.iterate(30)
    gx = to64(m.get_cube())
    m.close()
    s = mo.iterate(p0, mo.zero_state(p0), 30)
    s = mo.iterate(p1, s, 30)
    assert np.linalg.norm(gx - s.X) / np.linalg.norm(s.X) < 1e-4


def test_autotuned_split_is_valid_and_reported(lib):
    cube = small_cube(256, 4, 4, seed=36)
    p = problem(cube, 4, 1, 0.25, 3.0)
    m = gpu_solver(cube, p)
    j1, cs = m.tiling()
    m.iterate(3)
    gx = to64(m.get_cube())
    m.close()
    assert 0 <= j1 <= 3 and cs in (0, 1, 2, 4, 8)
    s = mo.iterate(p, mo.zero_state(p), 3)
    assert np.linalg.norm(gx - s.X) / np.linalg.norm(s.X) < 1e-5


def test_errors_are_reported(lib):
    from paper_1602_08847_gb300.muffin import Muffin, MuffinError
    cube = small_cube(64, 2, 2, seed=35)
    with pytest.raises(MuffinError, match="ARG"):
        Muffin(torch.from_numpy(cube.dirty).cuda(), None, nscales=7)
    m = Muffin(torch.from_numpy(cube.dirty).cuda(), None, nscales=2)
    with pytest.raises(MuffinError, match="STATE"):
        m.iterate(1)
    bad = cube.psf.copy()
    bad[0, 3, 3] = np.nan
    with pytest.raises(MuffinError, match="NONFINITE"):
        m.set_psf(torch.from_numpy(bad).cuda())
    m.close()
    dirty = cube.dirty.copy()
    dirty[1, 0, 0] = np.inf
    with pytest.raises(MuffinError, match="NONFINITE"):
        Muffin(torch.from_numpy(dirty).cuda(), None, nscales=2)
