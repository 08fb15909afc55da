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

import functools
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
# W_s as a union of eight orthonormal Daubechies wavelet bases (Sec. 4)
# --------------------------------------------------------------------------
# The comparison dictionary of Sec. 4 (the one of MUFFIN v1): W_s x is the
# concatenation of the 2D periodic discrete wavelet transforms of x in the
# Daubechies bases with 1 .. 8 vanishing moments, J levels each, scaled by
# 1/sqrt(8) so that W_s^T W_s = I (a tight frame; the scale is a reading).
# Daubechies filters are built from their definition: the lowpass filter
# H(z) = sqrt(2) ((1 + z^-1)/2)^p Q(z) with |Q(e^iw)|^2 = P(sin^2(w/2)),
# P(y) = sum_{k<p} C(p-1+k, k) y^k, and Q keeping the zeros inside the unit
# circle (the minimum-phase choice), normalised to Q(1) = 1.

DB_BASES = 8


def daubechies_lowpass(p: int) -> np.ndarray:
    """h[0 .. 2p-1] of the Daubechies filter with p vanishing moments, H(z) = sum_t h[t] z^-t."""
    return _daubechies_lowpass(p).copy()


@functools.lru_cache(maxsize=None)
def _daubechies_lowpass(p: int) -> np.ndarray:
    from math import comb
    q = np.array([1.0 + 0j])
    if p > 1:
        P = [comb(p - 1 + k, k) for k in range(p)]          # ascending powers of y
        for yk in np.roots(P[::-1]):
            a = 1.0 - 2.0 * yk                               # y = (2 - z - 1/z)/4  <=>  z^2 - 2a z + 1 = 0
            r = np.sqrt(a * a - 1.0 + 0j)
            zk = a + r if abs(a + r) < 1.0 else a - r
            q = np.convolve(q, np.array([1.0, -zk])) / (1.0 - zk)
    binom = np.array([comb(p, t) for t in range(p + 1)], dtype=np.float64) / 2.0 ** p
    return np.sqrt(2.0) * np.real(np.convolve(binom, q))


def daubechies_highpass(h: np.ndarray) -> np.ndarray:
    """g[t] = (-1)^t h[2p-1-t]: the orthogonal mirror filter."""
    t = np.arange(h.size)
    return (-1.0) ** t * h[::-1]


def dwt_step(x: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """One periodic analysis step along an axis of even length M:
    lo[k] = sum_t h[t] x[(2k+t) mod M], hi[k] = sum_t g[t] x[(2k+t) mod M],
    returned as [lo | hi] along that axis."""
    g = daubechies_highpass(h)
    M = x.shape[axis]
    k = np.arange(M // 2)
    lo = sum(h[t] * np.take(x, (2 * k + t) % M, axis=axis) for t in range(h.size))
    hi = sum(g[t] * np.take(x, (2 * k + t) % M, axis=axis) for t in range(h.size))
    return np.concatenate([lo, hi], axis=axis)


def dwt_step_adjoint(c: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """Adjoint of dwt_step: x[(2k+t) mod M] += h[t] lo[k] + g[t] hi[k]."""
    g = daubechies_highpass(h)
    M = c.shape[axis]
    lo = np.take(c, np.arange(M // 2), axis=axis)
    hi = np.take(c, np.arange(M // 2, M), axis=axis)
    x = np.zeros_like(c)
    xm = np.moveaxis(x, axis, 0)
    lom, him = np.moveaxis(lo, axis, 0), np.moveaxis(hi, axis, 0)
    k = np.arange(M // 2)
    for t in range(h.size):
        xm[(2 * k + t) % M] += h[t] * lom + g[t] * him     # the M/2 targets are distinct for a fixed t
    return x


@functools.lru_cache(maxsize=None)
def _step_matrices(hkey: bytes, M: int):
    """(A, B): the matrices of dwt_step and dwt_step_adjoint on length-M vectors,
    column i the image of unit vector i (so the iteration runs as matmuls)."""
    h = np.frombuffer(hkey, dtype=np.float64)
    eye = np.eye(M)
    return dwt_step(eye, h, axis=0), dwt_step_adjoint(eye, h, axis=0)


def dwt2(x: np.ndarray, h: np.ndarray, J: int) -> np.ndarray:
    """J-level periodic 2D DWT of [..][N][N] images in the Mallat layout: level j
    transforms the top-left (N/2^j)^2 square (rows, then columns) by dwt_step."""
    c = np.array(x, dtype=np.float64, copy=True)
    M = c.shape[-1]
    for _ in range(J):
        A, _ = _step_matrices(np.asarray(h, dtype=np.float64).tobytes(), M)
        sq = c[..., :M, :M] @ A.T                     # dwt_step along rows
        c[..., :M, :M] = np.einsum("ij,...jk->...ik", A, sq)   # dwt_step along columns
        M //= 2
    return c


def dwt2_adjoint(c: np.ndarray, h: np.ndarray, J: int) -> np.ndarray:
    """Adjoint of dwt2: the levels in reverse order, each by dwt_step_adjoint along
    columns, then along rows."""
    x = np.array(c, dtype=np.float64, copy=True)
    N = x.shape[-1]
    for j in reversed(range(J)):
        M = N >> j
        _, B = _step_matrices(np.asarray(h, dtype=np.float64).tobytes(), M)
        sq = np.einsum("ij,...jk->...ik", B, x[..., :M, :M])
        x[..., :M, :M] = sq @ B.T
    return x


def union_analysis(x: np.ndarray, J: int) -> np.ndarray:
    """W_s x for the union of bases: [L][N][N] -> [L][8][N][N]."""
    s = 1.0 / np.sqrt(DB_BASES)
    return np.stack([s * dwt2(x, daubechies_lowpass(p), J) for p in range(1, DB_BASES + 1)], axis=1)


def union_adjoint(u: np.ndarray, J: int) -> np.ndarray:
    """W_s^T u for the union of bases: [L][8][N][N] -> [L][N][N]."""
    s = 1.0 / np.sqrt(DB_BASES)
    return sum(s * dwt2_adjoint(u[:, p - 1], daubechies_lowpass(p), J) for p in range(1, DB_BASES + 1))


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
    dictionary: str = "iuwt"  # W_s: "iuwt" (Sec. 3) or "union" (eight Daubechies bases, Sec. 4)

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


def ws_planes(p: Problem) -> int:
    return DB_BASES if p.dictionary == "union" else p.J + 1


def ws_analysis(p: Problem, x: np.ndarray) -> np.ndarray:
    """W_s x for the problem's dictionary."""
    return union_analysis(x, p.J) if p.dictionary == "union" else iuwt_analysis(x, p.J, p.gen)


def ws_adjoint(p: Problem, u: np.ndarray) -> np.ndarray:
    """W_s^T u for the problem's dictionary."""
    return union_adjoint(u, p.J) if p.dictionary == "union" else iuwt_adjoint(u, p.J, p.gen)


def zero_state(p: Problem) -> State:
    L, n, _ = p.shape
    return State(np.zeros((L, n, n)), np.zeros((L, ws_planes(p), n, n)), np.zeros((L, n, n)))


def iterate(p: Problem, s: State, n_iter: int = 1) -> State:
    """n_iter passes of Algorithm 1, one statement per line of the algorithm."""
    X, U, V = s.X, s.U, s.V
    for _ in range(n_iter):
        grad = gradient(X, p.y, p.hhat, p.w)
        spatial = p.mu_s * ws_adjoint(p, U)
        spectral = p.mu_l * spectral_adjoint(V)
        Xt = positive(X - p.tau * (grad + spatial + spectral))
        Ut = sat(U + p.sigma * p.mu_s * ws_analysis(p, 2.0 * Xt - X))
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
    spatial = p.mu_s * float(np.sum(np.abs(ws_analysis(p, X))))
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


def union_norm2(n: int, J: int, n_iter: int = 30, seed: int = 7) -> float:
    """||W_s||^2 of the union of bases by the power method (1 for a tight frame)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = rng.standard_normal((1, n, n))
    return power_iteration(lambda v: union_adjoint(union_analysis(v, J), J), x0, n_iter)


def make_problem(y, psf, J, gen=1, mu_s=0.25, mu_l=3.0, sigma=1.0, rho=1.0, w=None,
                 tau=None, margin=1.01, power_iters=50, dictionary="iuwt") -> Problem:
    """Problem with step sizes from power-iteration norms (x margin) and Condat."""
    y = np.asarray(y, dtype=np.float64)
    hhat = psf_multiplier(psf)
    w = np.ones(y.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    if tau is None:
        beta = margin * data_lipschitz(hhat, w, power_iters)
        if dictionary == "union":
            wn = margin * union_norm2(y.shape[-1], J)
        else:
            wn = margin * iuwt_norm2(y.shape[-1], J, gen)
        tau, sigma, rho, _ = condat_steps(beta, dual_norm2(mu_s, mu_l, wn), sigma, rho=rho)
    return Problem(y=y, hhat=hhat, J=J, gen=gen, mu_s=mu_s, mu_l=mu_l, tau=tau,
                   sigma=sigma, rho=rho, w=w, dictionary=dictionary)
