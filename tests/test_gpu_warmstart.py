"""What the trained warm-start network gains over the plain method.

The network shipped with the package was trained on 2000 synthetic
256x256x64 cubes (seeds 1000-2999) by the project's own kernels.  Here, on
held-out cubes, Algorithm 1 must reach a relative objective error of 1e-4
(against F*, the objective after 2000 passes from zero) in fewer passes and
less GPU time from the network's state than from the zero state, and the
objective test that guards the prediction must keep it.
"""
import os

import pytest
import torch

from paper_1602_08847_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def committed(lib):
    from paper_1602_08847_gb300 import warmstart as ws
    if not os.path.exists(ws.WEIGHTS):
        pytest.fail("the trained warm-start weights are missing from the package")
    net, meta = ws.load_committed()
    yield ws, net, meta
    net.close()


@pytest.mark.parametrize("seed", [5198, 5199])
def test_warm_start_reaches_tolerance_sooner(committed, seed):
    ws, net, meta = committed
    _, y, h = synth.cube_arrays(("256x256x64", seed))
    r = ws.evaluate_one(net, y, h, 4, input_passes=meta["input_passes"])
    zero, warm = r["zero"], r["net"]
    assert zero["passes"] is not None and warm["passes"] is not None
    assert warm["used"]
    assert warm["passes"] < zero["passes"], (warm["passes"], zero["passes"])
    assert warm["pass_ms"] + warm["start_ms"] < zero["pass_ms"], (warm, zero)


def test_rejected_prediction_leaves_the_state_alone(committed):
    """The objective test: a network whose cube is worse than the current one
    is not used, and the state it found is restored."""
    ws, net, meta = committed
    from paper_1602_08847_gb300.net import WarmStartNet, warm_start
    _, y, h = synth.cube_arrays(("256x256x64", 5197))
    yd, hd = torch.from_numpy(y).cuda(), torch.from_numpy(h).cuda()
    m = ws.problem(yd, hd, 4)
    m.iterate(30)
    x0, u0, v0, it0 = m.get_state()
    bad = WarmStartNet(net.shape, theta=torch.zeros(net.n_params, device="cuda"), n_out=net.n_out)
    bad_theta = torch.zeros(net.n_params, device="cuda")
    bad_theta[-net.n_out] = 10.0      # bias of the cube map: a flat bright cube
    bad.set_params(bad_theta)
    dec = warm_start(m, bad, m.get_cube(), keep_state=True)
    assert not dec["used"]
    x1, u1, v1, it1 = m.get_state()
    assert it1 == it0
    assert torch.equal(x0, x1) and torch.equal(u0, u1) and torch.equal(v0, v1)
    m.close()
    bad.close()


def test_held_out_evaluation(committed):
    """The evaluation of the training record, rerun on held-out seeds 5000 ..
    5000 + n - 1 (n = MUFFIN_WARMSTART_SEEDS; about 1.5 s of GPU time per cube,
    so it runs only when asked): every cube reaches the tolerance from both
    starts, and the network's start takes less GPU time on the median cube."""
    n = int(os.environ.get("MUFFIN_WARMSTART_SEEDS", "0"))
    if n <= 0:
        pytest.skip("set MUFFIN_WARMSTART_SEEDS (e.g. 200) to rerun the held-out evaluation")
    ws, net, meta = committed
    results = []
    for seed in range(5000, 5000 + n):
        _, y, h = synth.cube_arrays(("256x256x64", seed))
        results.append(ws.evaluate_one(net, y, h, 4, input_passes=meta["input_passes"]))
    s = ws.summarise(results)
    print(s)
    assert s["zero"]["reached"] == n and s["net"]["reached"] == n
    assert s["net"]["gpu_ms_median"] < s["zero"]["gpu_ms_median"], s
