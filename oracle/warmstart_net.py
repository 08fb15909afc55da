"""FP64 CPU oracle of the warm-start network (forward, loss, gradients, Adam).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` and ``__graft_entry__.smoke()`` may
import this module; the CUDA library shares no code with it.

The paper has no network.  Its warm start is the two-step schedule of Sec. 4,
where the second run of Algorithm 1 starts from the cube the first run
produced.  Here a small 3D convolutional network predicts such a starting cube
from the dirty cube, and Algorithm 1 continues from the prediction.  What this
module computes has plain definitions, written out below:

* layer k: zero-padded 3x3x3 cross-correlation over (channel, row, column) of
  the cube, plus a bias, then ReLU (not after the last layer):
  ``z[co, p] = b[co] + sum_ci sum_{d in {-1,0,1}^3} w[co, ci, d + 1] a[ci, p + d]``
  with ``a[ci, q] = 0`` for q outside the cube;
* six layers: 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> K feature maps;
* input normalisation: ``a0 = y / s`` with ``s = max |y|`` over the whole
  dirty cube; output map 0 predicts the cube, ``s * z6[0]``; output maps
  1 .. K-1 predict K-1 further fields of the state of Algorithm 1 (the planes
  of the wavelet dual U), ``z6[k]`` as they are;
* loss: ``(1/V) sum_p [lam_0 (z6[0] - t_x / s)^2
  + sum_{k>=1} lam_k (z6[k] - t_aux[k-1])^2]`` over the V voxels, for a
  target cube t_x, target fields t_aux and channel weights lam;
* gradients by the chain rule; the ReLU derivative is 1 where the layer's
  output is > 0 and 0 elsewhere;
* Adam (Kingma and Ba, "Adam: a method for stochastic optimization", ICLR
  2015, Algorithm 1) with bias-corrected moments.

Cubes here are ``[C][Z][Y][X]`` float64 with Z the spectral channel axis of the
sky cube and C the feature axis.  Weights are ``[co][ci][3][3][3]``.  A packed
parameter vector concatenates, layer by layer, the weights in that order and
then the biases.
"""
from __future__ import annotations

import numpy as np

# (input features, output features, ReLU after the layer)
def arch(n_out: int = 1):
    return ((1, 32, True), (32, 32, True), (32, 32, True), (32, 32, True), (32, 32, True), (32, n_out, False))


ARCH = arch(1)


def n_params(arch=ARCH) -> int:
    return sum(co * ci * 27 + co for ci, co, _ in arch)


def unpack(theta: np.ndarray, arch=ARCH) -> list[tuple[np.ndarray, np.ndarray]]:
    """Packed vector -> [(w [co][ci][3][3][3], b [co]), ...]."""
    theta = np.asarray(theta, dtype=np.float64)
    out, off = [], 0
    for ci, co, _ in arch:
        w = theta[off:off + co * ci * 27].reshape(co, ci, 3, 3, 3)
        off += co * ci * 27
        b = theta[off:off + co]
        off += co
        out.append((w, b))
    assert off == theta.size, "parameter vector does not match the architecture"
    return out


def pack(layers: list[tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


# --------------------------------------------------------------------------
# one layer
# --------------------------------------------------------------------------

def conv3d(a: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3x3 cross-correlation plus bias: a [ci][Z][Y][X] -> [co][Z][Y][X]."""
    ci, Z, Y, X = a.shape
    co = w.shape[0]
    ap = np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1)))
    z = np.empty((co, Z, Y, X))
    z[:] = b[:, None, None, None]
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                z += np.tensordot(w[:, :, kz, ky, kx], ap[:, kz:kz + Z, ky:ky + Y, kx:kx + X], axes=(1, 0))
    return z


def conv3d_backward(a: np.ndarray, w: np.ndarray, dz: np.ndarray):
    """Gradients of sum(dz * conv3d(a, w, b)) with respect to a, w and b."""
    ci, Z, Y, X = a.shape
    ap = np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dap = np.zeros_like(ap)
    dw = np.empty_like(w)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                win = (slice(None), slice(kz, kz + Z), slice(ky, ky + Y), slice(kx, kx + X))
                dap[win] += np.tensordot(w[:, :, kz, ky, kx], dz, axes=(0, 0))
                dw[:, :, kz, ky, kx] = np.tensordot(dz, ap[win], axes=([1, 2, 3], [1, 2, 3]))
    da = dap[:, 1:-1, 1:-1, 1:-1]
    db = dz.sum(axis=(1, 2, 3))
    return da, dw, db


# --------------------------------------------------------------------------
# the network
# --------------------------------------------------------------------------

def input_scale(y: np.ndarray) -> float:
    s = float(np.max(np.abs(y)))
    return s if s > 0 else 1.0


def forward(theta: np.ndarray, y: np.ndarray, arch=ARCH):
    """Dirty cube y [L][N][N] -> (cube prediction s z6[0] [L][N][N], activations, scale s).

    activations[0] is the normalised input, activations[k] the output of layer
    k (after its ReLU when it has one); activations[6] holds all K output maps."""
    s = input_scale(y)
    a = np.asarray(y, dtype=np.float64)[None] / s
    acts = [a]
    for (w, b), (_, _, relu) in zip(unpack(theta, arch), arch):
        z = conv3d(a, w, b)
        a = np.maximum(z, 0.0) if relu else z
        acts.append(a)
    return s * a[0], acts, s


def _residual(acts, s, t, t_aux, lam):
    """Weighted residual maps r[k] = z6[k] - target[k] and the weights [K]."""
    z = acts[-1]
    K = z.shape[0]
    target = np.empty_like(z)
    target[0] = np.asarray(t, dtype=np.float64) / s
    if K > 1:
        target[1:] = np.asarray(t_aux, dtype=np.float64)
    lam = np.ones(K) if lam is None else np.asarray(lam, dtype=np.float64)
    return z - target, lam


def loss(theta: np.ndarray, y: np.ndarray, t: np.ndarray, arch=ARCH, t_aux=None, lam=None) -> float:
    _, acts, s = forward(theta, y, arch)
    r, lam = _residual(acts, s, t, t_aux, lam)
    return float(np.sum(lam[:, None, None, None] * r * r) / r[0].size)


def gradient(theta: np.ndarray, y: np.ndarray, t: np.ndarray, arch=ARCH, t_aux=None, lam=None):
    """(loss, packed gradient of the loss with respect to theta)."""
    layers = unpack(theta, arch)
    _, acts, s = forward(theta, y, arch)
    r, lam = _residual(acts, s, t, t_aux, lam)
    value = float(np.sum(lam[:, None, None, None] * r * r) / r[0].size)
    dz = (2.0 / r[0].size) * lam[:, None, None, None] * r
    grads = [None] * len(layers)
    for k in range(len(layers) - 1, -1, -1):
        w, _ = layers[k]
        da, dw, db = conv3d_backward(acts[k], w, dz)
        grads[k] = (dw, db)
        if k > 0:
            dz = da * (acts[k] > 0.0)     # ReLU of layer k (output acts[k])
    return value, pack(grads)


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------

def adam_step(theta, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t >= 1; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
