"""The pass schedule (channel groups, graph branches) changes when kernels run,
not what they compute: every plan gives bitwise the same state, and the state
matches the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import muffin_oracle as mo
from gpu_helpers import small_cube, problem, gpu_solver, to64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,J,j1", [(128, 16, 4, 3), (64, 13, 3, 2), (256, 32, 4, 2)])
def test_pass_plans_are_bitwise_identical(lib, n, L, J, j1):
    cube = small_cube(n, L, J, seed=80 + L)
    p = problem(cube, J, 1, 0.3, 1.2, tau=None, sigma=1.5)
    ref = None
    for plan in [(0, 1), (4, 2), (3, 3), (1, 1), (5, 3), (L, 2)]:
        m = gpu_solver(cube, p, fine_levels=j1)
        m.set_plan(*plan)
        g, b = m.plan()
        assert 1 <= g <= L and 1 <= b <= 3
        m.iterate(6)
        x, u, v, _ = m.get_state()
        torch.cuda.synchronize()
        m.close()
        if ref is None:
            ref = (x, u, v)
        else:
            assert torch.equal(ref[0], x) and torch.equal(ref[1], u) and torch.equal(ref[2], v), plan
    s = mo.iterate(p, mo.zero_state(p), 6)
    assert np.linalg.norm(to64(ref[0]) - s.X) / np.linalg.norm(s.X) < 1e-5


def test_plan_argument_errors(lib):
    from paper_1602_08847_gb300.muffin import MuffinError
    cube = small_cube(64, 4, 2, seed=90)
    m = gpu_solver(cube, problem(cube, 2, 1, 0.25, 3.0))
    with pytest.raises(MuffinError, match="ARG"):
        m.set_plan(-1, 1)
    with pytest.raises(MuffinError, match="ARG"):
        m.set_plan(2, 4)
    m.close()
