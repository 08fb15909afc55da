"""Batches of uneven cubes in one graph launch per pass (muffin_batch_*)."""
import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
from gpu_helpers import small_cube, problem, gpu_solver, to64

pytestmark = pytest.mark.gpu


def _cubes():
    specs = [(64, 8, 3, 1), (128, 4, 4, 2), (32, 3, 2, 1), (256, 2, 4, 1)]
    out = []
    for i, (n, L, J, gen) in enumerate(specs):
        cube = small_cube(n, L, J, seed=60 + i)
        out.append((cube, problem(cube, J, gen, 0.25, 1.5)))
    return out


def test_batch_equals_cubes_run_one_by_one(lib):
    """Each cube of a batch gets exactly the passes it would get alone."""
    from paper_1602_08847_gb300.muffin import Batch
    cubes = _cubes()
    solo = []
    for cube, p in cubes:
        m = gpu_solver(cube, p)
        split = m.tiling()[0]
        m.iterate(7)
        solo.append((m.get_cube().clone(), split))
        m.close()
    batch_ms = [gpu_solver(cube, p, fine_levels=split) for (cube, p), (_, split) in zip(cubes, solo)]
    b = Batch(batch_ms)
    b.iterate(3)
    b.iterate(4)
    torch.cuda.synchronize()
    for m, (x_solo, _) in zip(batch_ms, solo):
        assert torch.equal(m.get_cube(), x_solo)
        assert m.get_state()[3] == 7
    b.close()
    for m in batch_ms:
        m.close()


def test_batch_matches_oracle_and_follows_context_changes(lib):
    """A context changed after the batch was built (two-step calibration) is
    recaptured; every cube still matches the FP64 oracle."""
    from paper_1602_08847_gb300.muffin import Batch
    cubes = _cubes()[:2]
    ms = [gpu_solver(cube, p) for cube, p in cubes]
    b = Batch(ms)
    b.iterate(5)
    ms[0].set_mu(0.25, 0.0)
    b.iterate(5)
    torch.cuda.synchronize()
    xs = [to64(m.get_cube()) for m in ms]
    b.close()
    for m in ms:
        m.close()
    (c0, p0), (c1, p1) = cubes
    s0 = mo.iterate(p0, mo.zero_state(p0), 5)
    p0b = mo.Problem(y=p0.y, hhat=p0.hhat, J=p0.J, gen=p0.gen, mu_s=0.25, mu_l=0.0, tau=p0.tau, sigma=p0.sigma,
                     rho=p0.rho)
    s0 = mo.iterate(p0b, s0, 5)
    s1 = mo.iterate(p1, mo.zero_state(p1), 10)
    assert np.linalg.norm(xs[0] - s0.X) / np.linalg.norm(s0.X) < 1e-5
    assert np.linalg.norm(xs[1] - s1.X) / np.linalg.norm(s1.X) < 1e-5


def test_batch_rejects_bad_arguments(lib):
    from paper_1602_08847_gb300.muffin import Batch, MuffinError, Muffin
    cube, p = _cubes()[0]
    m = Muffin(torch.from_numpy(cube.dirty).cuda(), None, nscales=3)
    with pytest.raises(MuffinError, match="STATE"):
        Batch([m])
    m.close()
    m2 = gpu_solver(cube, p)
    with pytest.raises(MuffinError, match="twice"):
        Batch([m2, m2])
    m2.close()


def _persistent_cubes():
    """Uneven cubes the persistent kernel takes: every FFT size it serves, coarse
    sub-images of 32, 64 and 128 (resident and streamed dual planes), the
    Makhoul and the dense spectral step."""
    specs = [(128, 16, 4, 2), (256, 4, 4, 2), (512, 2, 5, 3), (1024, 3, 4, 3)]
    out = []
    for i, (n, L, J, j1) in enumerate(specs):
        cube = small_cube(n, L, J, seed=70 + i)
        out.append((cube, problem(cube, J, 1, 0.25, 1.5), j1))
    return out


def test_persistent_batch_equals_graph_batch_and_oracle(lib):
    """One persistent launch per pass (mode 1) gives what the graph branches
    (mode 0) give, and matches the FP64 oracle."""
    from paper_1602_08847_gb300.muffin import Batch
    cubes = _persistent_cubes()
    states = {}
    for mode in ("graph", "persistent"):
        ms = [gpu_solver(cube, p, fine_levels=j1) for cube, p, j1 in cubes]
        b = Batch(ms)
        b.set_mode(mode)
        assert b.mode == mode
        b.iterate(3)
        b.iterate(3)
        b.check()
        states[mode] = [tuple(t.clone() for t in m.get_state()[:3]) for m in ms]
        b.close()
        for m in ms:
            m.close()
    for (xg, ug, vg), (xp, up, vp) in zip(states["graph"], states["persistent"]):
        for a, c in ((xg, xp), (ug, up), (vg, vp)):
            scale = float(a.abs().max()) or 1.0
            assert float((a - c).abs().max()) <= 1e-6 * scale
    for (cube, p, _), (x, _, _) in zip(cubes, states["persistent"]):
        s = mo.iterate(p, mo.zero_state(p), 6)
        assert np.linalg.norm(to64(x) - s.X) / np.linalg.norm(s.X) < 1e-5


def test_persistent_batch_barrier_gives_up_and_reports(lib):
    """Failure detection without a GPU fault: with the barrier's poll bound at 0
    every block that does not arrive last gives up at once, the blocks skip
    the remaining stages and the launch ends; check() reports TIMEOUT.  With
    the bound restored the batch runs again."""
    from paper_1602_08847_gb300.muffin import Batch, MuffinError
    cubes = _persistent_cubes()[:2]
    ms = [gpu_solver(cube, p, fine_levels=j1) for cube, p, j1 in cubes]
    b = Batch(ms)
    b.set_mode("persistent")
    b.set_wait_limit(0)
    b.iterate(1)
    with pytest.raises(MuffinError, match="TIMEOUT"):
        b.check()
    b.set_wait_limit(None)
    b.iterate(2)
    b.check()
    b.close()
    for m in ms:
        m.close()


def test_persistent_batch_rejects_unsupported_cubes(lib):
    from paper_1602_08847_gb300.muffin import Batch, MuffinError
    cube = small_cube(64, 2, 2, seed=79)
    m = gpu_solver(cube, problem(cube, 2, 2, 0.25, 1.5))       # generation 2: no persistent path
    b = Batch([m])
    with pytest.raises(MuffinError, match="ARG"):
        b.set_mode("persistent")
    assert b.mode == "graph"
    b.close()
    m.close()
