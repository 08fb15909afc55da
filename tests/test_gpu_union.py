"""W_s as the union of eight Daubechies bases (the comparison dictionary of
Sec. 4): the CUDA path against the FP64 oracle, element by element."""
import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
from gpu_helpers import small_cube, problem, gpu_solver, to64, max_rel, one_pass_both

pytestmark = pytest.mark.gpu
TOL1 = 2e-5


@pytest.mark.parametrize("n,L,J", [(16, 3, 1), (16, 2, 3), (32, 4, 2), (64, 8, 3), (128, 3, 5), (256, 2, 4)])
def test_union_spatial_pass_matches_oracle(lib, n, L, J):
    """mu_lambda = 0: X and all eight planes of U after one pass from a random
    state (levels shorter than the longest filter included)."""
    cube = small_cube(n, L, J, seed=70 + n + J)
    p = problem(cube, J, 1, 0.4, 0.0, sigma=2.0, dictionary="union")
    (gx, gu, gv), s = one_pass_both(cube, p, seed=8)
    assert max_rel(gx, s.X) < TOL1
    for b in range(8):
        assert max_rel(gu[:, b], s.U[:, b]) < TOL1, f"basis {b + 1}"
    assert np.abs(gu).max() <= 1.0


@pytest.mark.parametrize("n,J", [(512, 2), (1024, 1)])
def test_union_spatial_pass_large_planes(lib, n, J):
    """Planes of 512 and 1024 pixels, where the fused analysis works on
    narrower column slabs (16 and 8 columns); step sizes given, so the oracle
    skips its power methods."""
    cube = small_cube(n, 1, J, seed=90 + J)
    p = problem(cube, J, 1, 0.4, 0.0, tau=1e-3, sigma=2.0, dictionary="union")
    (gx, gu, gv), s = one_pass_both(cube, p, seed=9)
    assert max_rel(gx, s.X) < TOL1
    for b in range(8):
        assert max_rel(gu[:, b], s.U[:, b]) < TOL1, f"basis {b + 1}"


def test_union_full_pass_relaxed_weighted(lib):
    cube = small_cube(64, 6, 3, seed=77)
    p = problem(cube, 3, 1, 0.3, 0.8, sigma=1.5, rho=1.3, tau=1e-3, w=np.array([1.0, 2.0, 0.5, 1.5, 1.0, 0.8]),
                dictionary="union")
    (gx, gu, gv), s = one_pass_both(cube, p, seed=9)
    assert max_rel(gx, s.X) < TOL1
    assert max_rel(gu, s.U) < TOL1
    assert max_rel(gv, s.V) < TOL1


def test_union_100_passes_64x64x8(lib):
    """The 64 x 64 x 8 workload with the union dictionary, 100 passes from zero:
    rel L2 of X <= 1e-4 and relative objective <= 1e-6 against FP64."""
    from paper_1602_08847_gb300 import synth
    cube = synth.make_cube("64x64x8")
    p = problem(cube, 3, 1, 0.25, 3.0, dictionary="union")
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


def test_union_objective_and_norm(lib):
    cube = small_cube(64, 4, 3, seed=78)
    p = problem(cube, 3, 1, 0.3, 0.9, dictionary="union")
    x = np.abs(np.random.Generator(np.random.PCG64(5)).standard_normal((4, 64, 64))).astype(np.float32)
    m = gpu_solver(cube, p, power_iters=30)
    m.set_cube(torch.from_numpy(x).cuda())
    tot, terms = m.objective()
    st = m.step_sizes()
    m.close()
    ref = mo.objective_terms(p, x.astype(np.float64))
    for a, b in zip(terms, ref):
        assert abs(a - b) <= 1e-6 * abs(b), (terms, ref)
    # a tight frame: ||W_s||^2 = 1, reported with the 1.01 margin
    assert abs(st["ws_norm2"] - 1.01) < 1e-4


def test_union_checkpoint_resume_is_bitwise(lib):
    cube = small_cube(128, 4, 4, seed=79)
    p = problem(cube, 4, 1, 0.25, 3.0, dictionary="union")
    a = gpu_solver(cube, p)
    a.iterate(20)
    x, u, v, it = a.get_state()
    assert u.shape == (4, 8, 128, 128)
    a.iterate(20)
    x_ref = a.get_cube().clone()
    a.close()
    b = gpu_solver(cube, p)
    b.set_state(x, u, v, it)
    b.iterate(20)
    assert torch.equal(x_ref, b.get_cube())
    b.close()


def test_union_needs_a_level(lib):
    from paper_1602_08847_gb300.muffin import make_params, muffin_check_params
    code, msg = muffin_check_params(make_params(64, 2, 0, dictionary="union"))
    assert code != 0 and "J >= 1" in msg
