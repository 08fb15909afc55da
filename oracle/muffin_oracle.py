"""FP64 CPU oracle of the MUFFIN primal-dual method (Deguignet et al., Sec. 2-3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library never
calls it and shares no code with it; the two meet only through the seeded
inputs of ``paper_1602_08847_gb300.synth``.

Everything here is plain numpy in float64, written for a reader to check by eye
against the paper.  Arrays are channel-major: a cube ``X`` is ``[L][N][N]``
(column ``x_l`` of the paper is ``X[l]``; row ``x^n`` of the paper, the spectrum
of pixel n, is ``X[:, py, px]``).  Wavelet coefficients ``U`` are
``[L][J+1][N][N]``: ``U[l, j]`` for the detail planes j < J and ``U[l, J]`` for
the coarse plane.

Readings of the paper taken here (each also listed in the design notes):

* H_l (Eq. 4) is circular convolution on the N x N grid by the PSF of channel
  l, whose peak is given at pixel (N/2, N/2).  Its Fourier multiplier is
  ``fft2(ifftshift(psf))``.
* the dagger in Algorithm 1 and Eqs. 8-9 is the adjoint; ``i^d_l`` in the
  gradient line of Algorithm 1 is the dirty image ``y_l`` of Eq. 8.
* the weights 1/sigma_l^2 of Eq. 5 enter as ``w_l`` (default 1, which is
  Algorithm 1 as printed).
* W_s is the isotropic undecimated wavelet transform with the B3-spline
  filter [1, 4, 6, 4, 1]/16 at dilations 2^j, periodic boundary, J detail
  planes plus the coarse plane, every plane penalised.  Generation 1:
  w_j = c_j - c_{j+1}; generation 2 (the one used in Sec. 4):
  w_j = c_j - H_j c_{j+1}.
* W_lambda is the orthonormal DCT-II along the channel axis; its adjoint is
  its inverse.
* sat clips to [-1, 1] (Eq. 7); (.)_+ clips below at 0.
* the initial state is X = U = V = 0.
* step sizes follow Condat's condition 1/tau - sigma ||L||^2 > beta / 2 with
  rho < delta = 2 - beta / 2 (1/tau - sigma ||L||^2)^-1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# B3-spline scaling filter of the starlet (isotropic undecimated) transform.
B3 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


# --------------------------------------------------------------------------
# H_l: convolution by the PSF (Eq. 4), its adjoint and its norm
# --------------------------------------------------------------------------

def psf_multiplier(psf: np.ndarray) -> np.ndarray:
    """Fourier multiplier of H_l: the DFT of the PSF moved so its peak is at 0."""
    psf = np.asarray(psf, dtype=np.float64)
    return np.fft.fft2(np.fft.ifftshift(psf, axes=(-2, -1)), axes=(-2, -1))


def apply_H(x: np.ndarray, hhat: np.ndarray) -> np.ndarray:
    """H_l x_l for every channel: circular convolution via the DFT."""
    return np.real(np.fft.ifft2(hhat * np.fft.fft2(x, axes=(-2, -1)), axes=(-2, -1)))


def apply_Ht(x: np.ndarray, hhat: np.ndarray) -> np.ndarray:
    """H_l^T x_l: circular correlation, multiplier conj(hhat)."""
    return np.real(np.fft.ifft2(np.conj(hhat) * np.fft.fft2(x, axes=(-2, -1)), axes=(-2, -1)))


def convolve_direct(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Circular convolution by a centred PSF written as the plain double sum.

    (H x)[p] = sum_q psf_c[(p - q) mod N] x[q], with psf_c the PSF whose peak was
    moved from (N/2, N/2) to (0, 0).  O(N^4): for tiny grids only.
    """
    n = x.shape[-1]
    pc = np.fft.ifftshift(np.asarray(psf, dtype=np.float64))
    out = np.zeros((n, n))
    for py in range(n):
        for px in range(n):
            acc = 0.0
            for qy in range(n):
                for qx in range(n):
                    acc += pc[(py - qy) % n, (px - qx) % n] * x[qy, qx]
            out[py, px] = acc
    return out


def gradient(x: np.ndarray, y: np.ndarray, hhat: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient of the data term of Eq. 5: w_l H_l^T (H_l x_l - y_l) (Eq. 8)."""
    return w[:, None, None] * apply_Ht(apply_H(x, hhat) - y, hhat)


# --------------------------------------------------------------------------
# W_s: isotropic undecimated wavelet transform (a trous, B3 spline)
# --------------------------------------------------------------------------

def smooth(c: np.ndarray, j: int) -> np.ndarray:
    """H_j c: separable B3 filter with holes at dilation 2^j, periodic boundary.

    out[y, x] = sum_a sum_b h[a] h[b] c[(y + (a-2) d) mod N, (x + (b-2) d) mod N],
    d = 2^j.  The filter is symmetric, so this is its own adjoint.
    """
    d = 2 ** j
    rows = np.zeros_like(c)
    for k in range(5):
        rows += B3[k] * np.roll(c, -(k - 2) * d, axis=-1)
    out = np.zeros_like(c)
    for k in range(5):
        out += B3[k] * np.roll(rows, -(k - 2) * d, axis=-2)
    return out


def iuwt_analysis(x: np.ndarray, J: int, gen: int = 1) -> np.ndarray:
    """W_s x: J detail planes then the coarse plane, stacked on axis -3."""
    planes = []
    c = np.asarray(x, dtype=np.float64)
    for j in range(J):
        c_next = smooth(c, j)
        if gen == 1:
            planes.append(c - c_next)
        else:
            planes.append(c - smooth(c_next, j))
        c = c_next
    planes.append(c)
    return np.stack(planes, axis=-3)


def iuwt_synthesis(u: np.ndarray, J: int, gen: int = 1) -> np.ndarray:
    """The perfect-reconstruction inverse of iuwt_analysis (not its adjoint).

    Generation 1: x = sum of the detail planes plus the coarse plane.
    Generation 2: c_j = H_j c_{j+1} + w_j, from the coarse plane down to c_0.
    """
    if gen == 1:
        return np.sum(u, axis=-3)
    c = u[..., J, :, :]
    for j in range(J - 1, -1, -1):
        c = smooth(c, j) + u[..., j, :, :]
    return c


def iuwt_adjoint(u: np.ndarray, J: int, gen: int = 1) -> np.ndarray:
    """W_s^T u, the exact adjoint of iuwt_analysis (Eq. 9, Sec. 4).

    Every H_j is symmetric and all of them commute (circulant filters), so with
    A_j = H_{j-1}...H_0 the analysis is w_j = G_j A_j x with G_j = I - H_j
    (generation 1) or I - H_j^2 (generation 2), and c_J = A_J x.  Its adjoint
    is sum_j A_j G_j u_j + A_J u_J, evaluated from the coarse end:
    r = u_J, then r <- G_j u_j + H_j r for j = J-1 .. 0.
    """
    r = np.asarray(u[..., J, :, :], dtype=np.float64)
    for j in range(J - 1, -1, -1):
        uj = u[..., j, :, :]
        if gen == 1:
            g = uj - smooth(uj, j)
        else:
            g = uj - smooth(smooth(uj, j), j)
        r = g + smooth(r, j)
    return r


def iuwt_norm2_closed_form(n: int, J: int, gen: int = 1) -> float:
    """||W_s||^2 from the transfer functions on the N x N DFT grid.

    All filters are circulant and real-symmetric, so W_s^T W_s is diagonal in
    the DFT basis with eigenvalue sum_j |g_j(w)|^2 + |a_J(w)|^2.  The 1-D B3
    response at dilation d is (6 + 8 cos(d t) + 2 cos(2 d t)) / 16.
    """
    t = 2.0 * np.pi * np.arange(n) / n

    def b3(d):
        r = (6.0 + 8.0 * np.cos(d * t) + 2.0 * np.cos(2.0 * d * t)) / 16.0
        return r[:, None] * r[None, :]

    a = np.ones((n, n))
    total = np.zeros((n, n))
    for j in range(J):
        h = b3(2 ** j)
        g = (1.0 - h) if gen == 1 else (1.0 - h * h)
        total += (g * a) ** 2
        a = a * h
    total += a ** 2
    return float(total.max())


# --------------------------------------------------------------------------
# W_lambda: orthonormal cosine transform along the channel axis
# --------------------------------------------------------------------------

def dct_matrix(L: int) -> np.ndarray:
    """Orthonormal DCT-II matrix C[k, l] = c_k cos(pi (2l + 1) k / (2L))."""
    k = np.arange(L)[:, None]
    l = np.arange(L)[None, :]
    c = np.cos(np.pi * (2 * l + 1) * k / (2.0 * L))
    scale = np.full((L, 1), np.sqrt(2.0 / L))
    scale[0, 0] = np.sqrt(1.0 / L)
    return scale * c


def spectral_analysis(x: np.ndarray) -> np.ndarray:
    """x^n W_lambda for every pixel n: the DCT of each pixel's spectrum."""
    C = dct_matrix(x.shape[0])
    return np.tensordot(C, x, axes=(1, 0))


def spectral_adjoint(v: np.ndarray) -> np.ndarray:
    """v^n W_lambda^T for every pixel: the transpose (= inverse) DCT."""
    C = dct_matrix(v.shape[0])
    return np.tensordot(C.T, v, axes=(1, 0))


# --------------------------------------------------------------------------
# proximal maps (Eq. 7 and the positive-orthant projection)
# --------------------------------------------------------------------------

def sat(u: np.ndarray) -> np.ndarray:
    """Eq. 7: -1 below -1, 1 above 1, identity in between."""
    return np.where(u < -1.0, -1.0, np.where(u > 1.0, 1.0, u))


def positive(x: np.ndarray) -> np.ndarray:
    """Projection on the positive orthant."""
    return np.where(x > 0.0, x, 0.0)


# --------------------------------------------------------------------------
# the problem and Algorithm 1
# --------------------------------------------------------------------------

@dataclass
class Problem:
    """Data and parameters of Eqs. 5-6 plus the step sizes of Algorithm 1."""

    y: np.ndarray            # [L][N][N] dirty cube
    hhat: np.ndarray         # [L][N][N] complex multipliers of H_l
    J: int
    gen: int = 1
    mu_s: float = 0.25
    mu_l: float = 3.0
    tau: float = 1e-3
    sigma: float = 1.0
    rho: float = 1.0
    w: np.ndarray = None     # [L] channel weights 1/sigma_l^2

    def __post_init__(self):
        self.y = np.asarray(self.y, dtype=np.float64)
        if self.w is None:
            self.w = np.ones(self.y.shape[0])
        self.w = np.asarray(self.w, dtype=np.float64)

    @property
    def shape(self):
        return self.y.shape


@dataclass
class State:
    X: np.ndarray
    U: np.ndarray
    V: np.ndarray
    it: int = 0

    def copy(self) -> "State":
        return State(self.X.copy(), self.U.copy(), self.V.copy(), self.it)


def zero_state(p: Problem) -> State:
    L, n, _ = p.shape
    return State(np.zeros((L, n, n)), np.zeros((L, p.J + 1, n, n)), np.zeros((L, n, n)))


def iterate(p: Problem, s: State, n_iter: int = 1) -> State:
    """n_iter passes of Algorithm 1, one statement per line of the algorithm."""
    X, U, V = s.X, s.U, s.V
    for _ in range(n_iter):
        grad = gradient(X, p.y, p.hhat, p.w)
        spatial = p.mu_s * iuwt_adjoint(U, p.J, p.gen)
        spectral = p.mu_l * spectral_adjoint(V)
        Xt = positive(X - p.tau * (grad + spatial + spectral))
        Ut = sat(U + p.sigma * p.mu_s * iuwt_analysis(2.0 * Xt - X, p.J, p.gen))
        Vt = sat(V + p.sigma * p.mu_l * spectral_analysis(2.0 * Xt - X))
        X = p.rho * Xt + (1.0 - p.rho) * X
        U = p.rho * Ut + (1.0 - p.rho) * U
        V = p.rho * Vt + (1.0 - p.rho) * V
    return State(X, U, V, s.it + n_iter)


def objective_terms(p: Problem, X: np.ndarray) -> tuple[float, float, float]:
    """(data term of Eq. 5, spatial term, spectral term of Eq. 6) at X.

    The positivity indicator of Eq. 6 is left out: it is 0 for the iterates of
    Algorithm 1, which are non-negative by construction.
    """
    r = p.y - apply_H(X, p.hhat)
    data = 0.5 * float(np.sum(p.w[:, None, None] * r * r))
    spatial = p.mu_s * float(np.sum(np.abs(iuwt_analysis(X, p.J, p.gen))))
    spectral = p.mu_l * float(np.sum(np.abs(spectral_analysis(X))))
    return data, spatial, spectral


def objective(p: Problem, X: np.ndarray) -> float:
    return float(sum(objective_terms(p, X)))


def snr_db(X: np.ndarray, X_true: np.ndarray) -> float:
    """Reconstruction SNR of Sec. 4: 10 log10(||X*||^2 / ||X - X*||^2)."""
    return 10.0 * np.log10(np.sum(X_true ** 2) / np.sum((X - X_true) ** 2))


# --------------------------------------------------------------------------
# step sizes: operator norms by power iteration and Condat's condition
# --------------------------------------------------------------------------

def power_iteration(apply, x0: np.ndarray, n_iter: int) -> float:
    """Largest eigenvalue of a symmetric PSD operator by the power method."""
    x = x0 / np.linalg.norm(x0)
    lam = 0.0
    for _ in range(n_iter):
        y = apply(x)
        lam = float(np.vdot(x, y))
        x = y / np.linalg.norm(y)
    return lam


def data_lipschitz(hhat: np.ndarray, w: np.ndarray, n_iter: int = 50, seed: int = 7) -> float:
    """beta = max_l w_l ||H_l^T H_l||: power method run on each channel."""
    rng = np.random.Generator(np.random.PCG64(seed))
    best = 0.0
    for l in range(hhat.shape[0]):
        x0 = rng.standard_normal(hhat.shape[1:])
        lam = power_iteration(lambda v: apply_Ht(apply_H(v, hhat[l]), hhat[l]), x0, n_iter)
        best = max(best, w[l] * lam)
    return best


def iuwt_norm2(n: int, J: int, gen: int = 1, n_iter: int = 100, seed: int = 7) -> float:
    """||W_s||^2 = largest eigenvalue of W_s^T W_s by the power method."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = rng.standard_normal((n, n))
    return power_iteration(lambda v: iuwt_adjoint(iuwt_analysis(v, J, gen), J, gen), x0, n_iter)


def dual_norm2(mu_s: float, mu_l: float, ws_norm2: float) -> float:
    """||L||^2 for L = [mu_s W_s ; mu_lambda W_lambda] with W_lambda orthonormal."""
    return mu_s * mu_s * ws_norm2 + mu_l * mu_l


def condat_steps(beta: float, l_norm2: float, sigma: float = 1.0, safety: float = 0.99,
                 rho: float = 1.0) -> tuple[float, float, float, float]:
    """(tau, sigma, rho, delta) meeting 1/tau - sigma ||L||^2 > beta/2 and rho < delta."""
    tau = safety / (0.5 * beta + sigma * l_norm2)
    delta = 2.0 - 0.5 * beta / (1.0 / tau - sigma * l_norm2)
    if not (0.0 < rho < delta):
        raise ValueError(f"rho={rho} outside (0, {delta})")
    return tau, sigma, rho, delta


def make_problem(y, psf, J, gen=1, mu_s=0.25, mu_l=3.0, sigma=1.0, rho=1.0, w=None,
                 tau=None, margin=1.01, power_iters=50) -> Problem:
    """Problem with step sizes from power-iteration norms (x margin) and Condat."""
    y = np.asarray(y, dtype=np.float64)
    hhat = psf_multiplier(psf)
    w = np.ones(y.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    if tau is None:
        beta = margin * data_lipschitz(hhat, w, power_iters)
        wn = margin * iuwt_norm2(y.shape[-1], J, gen)
        tau, sigma, rho, _ = condat_steps(beta, dual_norm2(mu_s, mu_l, wn), sigma, rho=rho)
    return Problem(y=y, hhat=hhat, J=J, gen=gen, mu_s=mu_s, mu_l=mu_l, tau=tau,
                   sigma=sigma, rho=rho, w=w)
