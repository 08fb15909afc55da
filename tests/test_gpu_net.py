"""Warm-start network kernels against the FP64 network oracle.

Inputs and weights are drawn on the bfloat16 grid, so both sides start from
the same numbers.  A single layer's output then differs from the oracle only by
float32 accumulation and the final rounding to bfloat16 (half an ulp, 2^-9
relative); weight gradients are float32 sums of exact products.  Through the
six layers the bfloat16 roundings of the feature maps add up; the bound used
there is stated at the test.
"""
import numpy as np
import pytest
import torch

from oracle import warmstart_net as wn
from paper_1602_08847_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(2, 8, 16), (3, 9, 20), (5, 17, 35)]   # one tile; ragged tails along every axis


@pytest.fixture(scope="module")
def netmod(lib):
    from paper_1602_08847_gb300 import net
    return net


def bf(shape, seed, lo=-1.0, hi=1.0):
    return synth.bf16_round(synth.random_field(shape, seed, lo, hi).astype(np.float32)).astype(np.float64)


def to_map(a):
    """oracle [C][Z][Y][X] -> device bfloat16 [Z][Y][X][C]."""
    return torch.from_numpy(np.ascontiguousarray(a.transpose(1, 2, 3, 0)).astype(np.float32)).cuda().to(torch.bfloat16)


def from_map(t):
    return t.float().cpu().numpy().astype(np.float64).transpose(3, 0, 1, 2)


def close_bf16(gpu, ref, scale):
    """Within one bfloat16 ulp of the exact value, plus float32 accumulation."""
    err = np.abs(gpu - ref)
    return np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-5 * scale), float(np.max(err))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("relu", [True, False])
def test_layer_forward(netmod, shape, relu):
    a = np.maximum(bf((32,) + shape, 1), 0.0)
    w = bf((32, 32, 3, 3, 3), 2, -0.1, 0.1)
    b = bf((32,), 3, -0.2, 0.2)
    ref = wn.conv3d(a, w, b)
    if relu:
        ref = np.maximum(ref, 0.0)
    z = netmod.conv3d_forward(to_map(a), torch.from_numpy(w.astype(np.float32)).cuda(),
                              torch.from_numpy(b.astype(np.float32)).cuda(), relu)
    ok, err = close_bf16(from_map(z), ref, np.max(np.abs(ref)))
    assert ok, err


@pytest.mark.parametrize("shape", SHAPES)
def test_layer_backward_data(netmod, shape):
    dz = bf((32,) + shape, 4)
    w = bf((32, 32, 3, 3, 3), 5, -0.1, 0.1)
    mask = np.maximum(bf((32,) + shape, 6), 0.0)        # a ReLU output: about half zeros
    da, _, _ = wn.conv3d_backward(np.zeros_like(dz), w, dz)
    ref = da * (mask > 0)
    got = netmod.conv3d_backward_data(to_map(dz), torch.from_numpy(w.astype(np.float32)).cuda(), to_map(mask))
    ok, err = close_bf16(from_map(got), ref, np.max(np.abs(ref)))
    assert ok, err
    # without a mask: the plain adjoint
    got = netmod.conv3d_backward_data(to_map(dz), torch.from_numpy(w.astype(np.float32)).cuda(), None)
    ok, err = close_bf16(from_map(got), da, np.max(np.abs(da)))
    assert ok, err


@pytest.mark.parametrize("shape", SHAPES + [(8, 40, 64)])
def test_layer_backward_weights(netmod, shape):
    a = np.maximum(bf((32,) + shape, 7), 0.0)
    dz = bf((32,) + shape, 8)
    _, dw, db = wn.conv3d_backward(a, np.zeros((32, 32, 3, 3, 3)), dz)
    _, dw_abs, db_abs = wn.conv3d_backward(np.abs(a), np.zeros((32, 32, 3, 3, 3)), np.abs(dz))
    gdw, gdb = netmod.conv3d_backward_weights(to_map(a), to_map(dz))
    gdw = gdw.cpu().numpy().astype(np.float64)
    gdb = gdb.cpu().numpy().astype(np.float64)
    # float32 sums of exact products: error below n * 2^-24 of the sum of magnitudes
    n = np.prod(shape)
    assert np.all(np.abs(gdw - dw) <= n * 2.0 ** -24 * dw_abs + 1e-30)
    assert np.all(np.abs(gdb - db) <= n * 2.0 ** -24 * db_abs + 1e-30)


def net_inputs(shape, seed):
    """bfloat16-exact dirty cube with max |y| = 1 (so y / s is exact), a target."""
    y = bf(shape, seed, -0.3, 1.0)
    y.flat[np.argmax(np.abs(y))] = 1.0
    t = np.maximum(synth.random_field(shape, seed + 1, -0.5, 1.0), 0.0)
    return y, t


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bf16(a):
    return synth.bf16_round(a).astype(np.float64)


def gradient_at_bf16_points(theta, y, t, arch, t_aux=None, lam=None):
    """The oracle's gradient with the feature maps and the back-propagated
    map gradients rounded to bfloat16 where the kernels store them (weights
    rounded too; sums exact).  Its distance to the exact gradient measures how
    far bfloat16 storage alone moves the result on this input."""
    layers = wn.unpack(theta, arch)
    s = wn.input_scale(y)
    a = bf16(np.asarray(y)[None] / s)
    acts = [a]
    for k, ((w, b), (_, _, relu)) in enumerate(zip(layers, arch)):
        z = wn.conv3d(a, bf16(w), b)
        a = bf16(np.maximum(z, 0.0)) if relu else z
        acts.append(a)
    z = acts[-1]
    K = z.shape[0]
    target = np.empty_like(z)
    target[0] = t / s
    if K > 1:
        target[1:] = t_aux
    lam = np.ones(K) if lam is None else np.asarray(lam)
    dz = (2.0 / z[0].size) * lam[:, None, None, None] * (z - target)
    grads = [None] * len(layers)
    for k in range(len(layers) - 1, -1, -1):
        da, dw, db = wn.conv3d_backward(acts[k], bf16(layers[k][0]), dz)
        grads[k] = (dw, db)
        if k > 0:
            dz = bf16(da * (acts[k] > 0.0))
    return wn.pack(grads)


def check_gradient(g, theta, y, t, arch, t_aux=None, lam=None):
    """Per layer: the GPU gradient lies within twice the bfloat16-storage
    envelope of the exact gradient, plus 1 %."""
    _, g_ref = wn.gradient(theta, y, t, arch, t_aux, lam)
    g_bf = gradient_at_bf16_points(theta, y, t, arch, t_aux, lam)
    off = 0
    for ci, co, _ in arch:
        nw = co * ci * 27
        for part in (slice(off, off + nw), slice(off + nw, off + nw + co)):
            envelope = rel(g_bf[part], g_ref[part])
            assert rel(g[part], g_ref[part]) <= 2 * envelope + 1e-2, (ci, co, rel(g[part], g_ref[part]), envelope)
            cos = np.dot(g[part], g_ref[part]) / np.linalg.norm(g[part]) / np.linalg.norm(g_ref[part])
            assert cos > 0.995
        off += nw + co


@pytest.mark.parametrize("shape", [(4, 12, 20), (3, 16, 16)])
def test_network_prediction(netmod, shape):
    theta = synth.net_init(7).astype(np.float64)
    y, _ = net_inputs(shape, 11)
    ref, _, _ = wn.forward(theta, y)
    ref = np.maximum(ref, 0.0)
    n = netmod.WarmStartNet(shape, theta=torch.from_numpy(theta.astype(np.float32)).cuda())
    got, aux = n.predict(torch.from_numpy(y.astype(np.float32)).cuda())
    assert aux is None
    got = got.cpu().numpy().astype(np.float64)
    # five bfloat16 feature maps, each rounded to 2^-9 relative: well inside 2 %
    assert rel(got, ref) < 2e-2, rel(got, ref)
    assert np.all(got >= 0)


def test_network_loss_and_gradient(netmod):
    shape = (4, 12, 20)
    theta = synth.net_init(8).astype(np.float64)
    theta[-1] = 0.05
    y, t = net_inputs(shape, 12)
    loss_ref, g_ref = wn.gradient(theta, y, t)
    n = netmod.WarmStartNet(shape, training=True, theta=torch.from_numpy(theta.astype(np.float32)).cuda())
    loss, g = n.loss_grad(torch.from_numpy(y.astype(np.float32)).cuda(), torch.from_numpy(t.astype(np.float32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    check_gradient(g, theta, y, t, wn.ARCH)


def test_network_with_dual_outputs(netmod):
    """Six output maps (the cube and five planes of U): prediction, loss and
    gradient with per-map weights and bfloat16 field targets."""
    shape, K = (3, 10, 18), 6
    arch = wn.arch(K)
    rng = np.random.Generator(np.random.PCG64(21))
    theta = synth.bf16_round(rng.normal(0.0, 0.05, wn.n_params(arch)).astype(np.float32)).astype(np.float64)
    theta[:wn.n_params(wn.ARCH) - 865] = synth.net_init(11)[:wn.n_params(wn.ARCH) - 865]
    y, t = net_inputs(shape, 15)
    t_aux = bf((K - 1,) + shape, 16)
    lam = np.array([50.0, 1.0, 2.0, 0.5, 1.0, 3.0])
    # prediction: cube and clamped fields
    ref_x, acts, s = wn.forward(theta, y, arch)
    n = netmod.WarmStartNet(shape, theta=torch.from_numpy(theta.astype(np.float32)).cuda(), n_out=K)
    x, aux = n.predict(torch.from_numpy(y.astype(np.float32)).cuda())
    ref_aux = np.clip(acts[-1][1:], -1, 1).transpose(1, 0, 2, 3)       # [nz][K-1][ny][nx]
    assert rel(x.cpu().numpy().astype(np.float64), np.maximum(ref_x, 0)) < 2e-2
    assert rel(aux.cpu().numpy().astype(np.float64), ref_aux) < 2e-2
    # loss and gradient
    loss_ref, g_ref = wn.gradient(theta, y, t, arch, t_aux, lam)
    n = netmod.WarmStartNet(shape, training=True, theta=torch.from_numpy(theta.astype(np.float32)).cuda(), n_out=K,
                            out_weight=lam)
    ta = torch.from_numpy(np.ascontiguousarray(t_aux.transpose(1, 0, 2, 3)).astype(np.float32)).cuda()
    loss, g = n.loss_grad(torch.from_numpy(y.astype(np.float32)).cuda(), torch.from_numpy(t.astype(np.float32)).cuda(),
                          ta.to(torch.bfloat16))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    check_gradient(g, theta, y, t, arch, t_aux, lam)


def test_first_adam_step_moves_by_lr_times_sign(netmod):
    shape = (2, 8, 16)
    theta = synth.net_init(9).astype(np.float32)
    y, t = net_inputs(shape, 13)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    n = netmod.WarmStartNet(shape, training=True, theta=dev(theta))
    _, g = n.loss_grad(dev(y), dev(t))
    n.train_step(dev(y), dev(t), None, 1e-3)
    step = (n.get_params().cpu().numpy() - theta).astype(np.float64)
    g = g.cpu().numpy().astype(np.float64)
    big = np.abs(g) > 1e-5
    assert np.allclose(step[big], -1e-3 * np.sign(g[big]), rtol=1e-3, atol=2e-7)


def test_training_lowers_the_loss(netmod):
    shape = (4, 16, 16)
    y, _ = net_inputs(shape, 14)
    t = 0.8 * np.maximum(y, 0.0)                       # learnable from y
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    n = netmod.WarmStartNet(shape, training=True, theta=dev(synth.net_init(10)))
    yd, td = dev(y), dev(t)
    first, _ = n.loss_grad(yd, td)
    for _ in range(60):
        n.train_step(yd, td, None, 2e-3)
    last, _ = n.loss_grad(yd, td)
    assert last < 0.5 * first, (first, last)


def test_network_argument_errors(netmod):
    with pytest.raises(ValueError):
        netmod.WarmStartNet((0, 8, 8))
    with pytest.raises(ValueError):
        netmod.WarmStartNet((2, 8, 8), n_out=9)
    n = netmod.WarmStartNet((2, 8, 8))
    with pytest.raises(ValueError):
        n.predict(torch.zeros((2, 8, 9), device="cuda"))
    m = netmod.WarmStartNet((2, 8, 8), training=True, n_out=3)
    with pytest.raises(ValueError):                      # the fields' target is missing
        m.loss_grad(torch.zeros((2, 8, 8), device="cuda"), torch.zeros((2, 8, 8), device="cuda"))
    with pytest.raises(Exception):
        n.loss_grad(torch.zeros((2, 8, 8), device="cuda"), torch.zeros((2, 8, 8), device="cuda"))


def test_wait_give_up_is_reported_and_context_survives(netmod):
    """Failure detection of the bounded tensor-core waits, without a GPU fault:
    with the poll bound at 0 every pipeline wait gives up at once; each thread
    block drains its copy and MMAs in flight (full bound), frees its tensor
    memory and returns.  The prediction reports MUFFIN_ERR_TIMEOUT, the Adam
    step queued after a timed-out gradient is dropped on the device and
    reported by check(); with the bound restored the same context gives the
    prediction of an untouched run, bit for bit, and trains again."""
    from paper_1602_08847_gb300.muffin import MuffinError
    shape, K = (6, 40, 24), 3
    theta = torch.from_numpy(synth.net_init(21, K).astype(np.float32)).cuda()
    y = torch.from_numpy(synth.random_field(shape, 22, -0.3, 1.0).astype(np.float32)).cuda()
    ref = netmod.WarmStartNet(shape, theta=theta, n_out=K)
    x_ref, aux_ref = ref.predict(y)
    ref.close()
    n = netmod.WarmStartNet(shape, theta=theta, n_out=K)
    tr = netmod.WarmStartNet(shape, training=True, theta=theta, n_out=K)
    tx = torch.relu(y)
    ta = torch.zeros((shape[0], K - 1, shape[1], shape[2]), dtype=torch.bfloat16, device="cuda")
    try:
        netmod.set_wait_limit(0)
        with pytest.raises(MuffinError, match="TIMEOUT"):
            n.predict(y)
        before = tr.get_params().clone()
        tr.train_step(y, tx, ta, 1e-2)
        with pytest.raises(MuffinError, match="TIMEOUT"):
            tr.check()
        assert torch.equal(tr.get_params(), before)      # the update was dropped
    finally:
        netmod.set_wait_limit(None)
    x, aux = n.predict(y)
    assert torch.equal(x, x_ref) and torch.equal(aux, aux_ref)
    tr.train_step(y, tx, ta, 1e-2)
    tr.check()
    assert not torch.equal(tr.get_params(), before)
    n.close()
    tr.close()
    assert netmod.wait_timeouts() == 0


def test_no_tensor_core_wait_gave_up(netmod):
    """Every bounded wait of the tcgen05 layers above ended by completion."""
    assert netmod.wait_timeouts() == 0
