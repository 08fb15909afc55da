"""Pins of the warm-start network oracle (oracle/warmstart_net.py).

Each check compares the oracle with something other than itself: a library
routine that computes the same correlation, nested loops on a tiny input, the
adjoint identity between two separately written code paths, central finite
differences of the loss, and closed forms of Adam.
"""
import numpy as np
import pytest
import scipy.ndimage

from oracle import warmstart_net as wn

SMALL = ((1, 3, True), (3, 2, True), (2, 1, False))


def rnd(shape, seed, lo=-1.0, hi=1.0):
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, shape)


def test_single_channel_layer_is_scipy_correlate_with_zero_padding():
    a = rnd((1, 5, 6, 7), 1)
    w = rnd((1, 1, 3, 3, 3), 2)            # not symmetric: a flipped kernel fails
    b = np.array([0.3])
    z = wn.conv3d(a, w, b)[0]
    ref = scipy.ndimage.correlate(a[0], w[0, 0], mode="constant", cval=0.0) + 0.3
    assert np.max(np.abs(z - ref)) < 1e-13


def test_multichannel_layer_equals_nested_loops():
    ci, co, Z, Y, X = 2, 3, 3, 4, 5
    a = rnd((ci, Z, Y, X), 3)
    w = rnd((co, ci, 3, 3, 3), 4)
    b = rnd((co,), 5)
    z = wn.conv3d(a, w, b)
    ref = np.zeros((co, Z, Y, X))
    for o in range(co):
        for p in range(Z):
            for q in range(Y):
                for r in range(X):
                    acc = b[o]
                    for i in range(ci):
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    zz, yy, xx = p + dz - 1, q + dy - 1, r + dx - 1
                                    if 0 <= zz < Z and 0 <= yy < Y and 0 <= xx < X:
                                        acc += w[o, i, dz, dy, dx] * a[i, zz, yy, xx]
                    ref[o, p, q, r] = acc
    assert np.max(np.abs(z - ref)) < 1e-13


def test_layer_backward_is_the_adjoint_of_the_forward():
    """<conv(a), dz> = <a, da> (linear in a) and <conv_w(a), dz> = <w, dw> (linear in w)."""
    ci, co, shape = 3, 4, (4, 5, 3)
    a = rnd((ci,) + shape, 6)
    w = rnd((co, ci, 3, 3, 3), 7)
    dz = rnd((co,) + shape, 8)
    zero = np.zeros(co)
    da, dw, db = wn.conv3d_backward(a, w, dz)
    lhs = np.sum(wn.conv3d(a, w, zero) * dz)
    assert abs(lhs - np.sum(a * da)) < 1e-11 * abs(lhs)
    assert abs(lhs - np.sum(w * dw)) < 1e-11 * abs(lhs)
    # the bias enters every voxel once
    ones = np.ones(co)
    assert np.allclose(np.sum(wn.conv3d(np.zeros_like(a), w, ones) * dz), db.sum(), rtol=1e-13)


def _fd_check(arch, shape, seed, n_sample=None, h=1e-5):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.normal(0.0, 0.4, wn.n_params(arch))
    y = rng.uniform(-0.5, 1.0, shape)
    t = rng.uniform(0.0, 1.0, shape)
    K = arch[-1][1]
    t_aux = rng.uniform(-1.0, 1.0, (K - 1,) + shape) if K > 1 else None
    lam = rng.uniform(0.5, 3.0, K)
    _, g = wn.gradient(theta, y, t, arch, t_aux, lam)
    idx = np.arange(theta.size) if n_sample is None else rng.choice(theta.size, n_sample, replace=False)
    fd = np.empty(idx.size)
    for n, i in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[n] = (wn.loss(tp, y, t, arch, t_aux, lam) - wn.loss(tm, y, t, arch, t_aux, lam)) / (2 * h)
    return g[idx], fd


def test_gradient_matches_central_differences_small_net():
    g, fd = _fd_check(SMALL, (3, 4, 4), 9)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)


def test_gradient_matches_central_differences_several_outputs():
    """Three output maps (the cube and two further fields), weighted loss."""
    small3 = SMALL[:-1] + ((2, 3, False),)
    g, fd = _fd_check(small3, (3, 4, 4), 19)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)


def test_loss_weights_and_targets_enter_as_defined():
    """lam = (0, 1) and a zero network: loss = mean of the aux target squared."""
    K = 2
    theta = np.zeros(wn.n_params(wn.arch(K)))
    y = rnd((2, 3, 4), 20)
    t_aux = rnd((1, 2, 3, 4), 21)
    val = wn.loss(theta, y, rnd((2, 3, 4), 22), wn.arch(K), t_aux, (0.0, 1.0))
    assert np.isclose(val, np.mean(t_aux[0] ** 2), rtol=1e-14)


def test_gradient_matches_central_differences_full_net():
    """The six-layer architecture on a 2x3x3 cube, 60 sampled parameters
    (every layer's weights and biases are among them)."""
    g, fd = _fd_check(wn.ARCH, (2, 3, 3), 10, n_sample=60)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)


def test_gradient_of_every_layer_is_nonzero_and_loss_is_mean_square():
    rng = np.random.Generator(np.random.PCG64(11))
    theta = rng.normal(0.0, 0.3, wn.n_params())
    y = rng.uniform(0.0, 1.0, (2, 4, 4))
    t = rng.uniform(0.0, 1.0, (2, 4, 4))
    pred, _, s = wn.forward(theta, y)
    assert np.isclose(wn.loss(theta, y, t), np.mean((pred / s - t / s) ** 2), rtol=1e-14)
    _, g = wn.gradient(theta, y, t)
    off = 0
    for ci, co, _ in wn.ARCH:
        assert np.any(g[off:off + co * ci * 27] != 0)
        off += co * ci * 27 + co


def test_zero_weights_give_the_last_bias_times_the_scale():
    theta = np.zeros(wn.n_params())
    theta[-1] = 0.25
    y = rnd((3, 4, 5), 12)
    pred, _, s = wn.forward(theta, y)
    assert s == np.max(np.abs(y))
    assert np.allclose(pred, 0.25 * s, rtol=0, atol=1e-15)


def test_prediction_is_scale_equivariant():
    """The input is normalised by max |y|, so net(c y) = c net(y) for c > 0."""
    rng = np.random.Generator(np.random.PCG64(13))
    theta = rng.normal(0.0, 0.3, wn.n_params(SMALL))
    y = rng.uniform(-0.2, 1.0, (3, 4, 4))
    p1, _, _ = wn.forward(theta, y, SMALL)
    p2, _, _ = wn.forward(theta, 7.5 * y, SMALL)
    assert np.allclose(p2, 7.5 * p1, rtol=1e-13, atol=0)


def test_adam_first_step_moves_each_parameter_by_lr():
    """Kingma and Ba, Sec. 2.1: with bias correction the first step is lr * g / (|g| + eps)."""
    g = np.array([3.0, -0.02, 1e-3, -50.0])
    theta, m, v = wn.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(theta, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_with_a_constant_gradient_takes_equal_steps():
    g = np.array([0.5, -2.0])
    theta, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 31):
        theta, m, v = wn.adam_step(theta, g, m, v, t, lr=1e-3)
    assert np.allclose(theta, -30e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)


@pytest.mark.parametrize("plant", ["no_relu_mask", "flipped_kernel", "swapped_features"])
def test_planted_mistakes_are_caught(plant, monkeypatch):
    if plant == "no_relu_mask":
        orig = wn.gradient

        def wrong(theta, y, t, arch=wn.ARCH, t_aux=None, lam=None):
            layers = wn.unpack(theta, arch)
            _, acts, s = wn.forward(theta, y, arch)
            r = acts[-1][0] - t / s
            dz = (2.0 / r.size) * lam[0] * r[None]
            grads = [None] * len(layers)
            for k in range(len(layers) - 1, -1, -1):
                da, dw, db = wn.conv3d_backward(acts[k], layers[k][0], dz)
                grads[k] = (dw, db)
                dz = da
            return float(np.mean(r * r)), wn.pack(grads)

        monkeypatch.setattr(wn, "gradient", wrong)
        g, fd = _fd_check(SMALL, (3, 4, 4), 9)
        assert np.linalg.norm(g - fd) > 1e-3 * np.linalg.norm(fd)
        monkeypatch.setattr(wn, "gradient", orig)
    elif plant == "flipped_kernel":
        orig = wn.conv3d
        monkeypatch.setattr(wn, "conv3d", lambda a, w, b: orig(a, w[:, :, ::-1, ::-1, ::-1], b))
        with pytest.raises(AssertionError):
            test_single_channel_layer_is_scipy_correlate_with_zero_padding()
    else:
        orig = wn.conv3d
        monkeypatch.setattr(wn, "conv3d",
                            lambda a, w, b: orig(a, np.ascontiguousarray(w.reshape(w.shape[1], w.shape[0], 3, 3, 3)
                                                                         .transpose(1, 0, 2, 3, 4)), b)
                            if w.shape[0] == w.shape[1] else orig(a, w, b))
        ci = co = 2
        a = rnd((ci, 3, 3, 3), 14)
        w = rnd((co, ci, 3, 3, 3), 15)
        z = wn.conv3d(a, w, np.zeros(co))
        ref = sum(w[0, i, 1, 1, 1] * a[i, 1, 1, 1] for i in range(ci))
        ref += sum(w[0, i, dz, dy, dx] * a[i, dz, dy, dx]
                   for i in range(ci) for dz in range(3) for dy in range(3) for dx in range(3)) - \
            sum(w[0, i, 1, 1, 1] * a[i, 1, 1, 1] for i in range(ci))
        assert abs(z[0, 1, 1, 1] - ref) > 1e-6
