"""Seeded synthetic multi-frequency radio cubes (inputs only).

This module produces the inputs of the reconstruction problem of Sec. 2
(Eq. 4): a sky cube x*, one point spread function per channel and the dirty
cube y_l = H_l x*_l + n_l.  It stands in for the MeerKAT PSFs and the M31 sky of
Sec. 4, which are not available.  It holds none of the reconstruction method's
arithmetic: no gradient, no wavelet, no spectral transform and no proximal
step.  The instrument simulation below uses numpy's own FFT for the circular
convolution by the PSF; both the CUDA path and the FP64 checker receive the same
float32 arrays from here and nothing else.

Recipe (one numpy ``Generator(PCG64(seed))`` per cube, draws in this order):

* channels: frequencies linear over [1.0, 1.5] GHz, reference 1.25 GHz;
* sky: ``n_src`` sources; centre uniform over the image, Gaussian width
  U(1, 4) px, peak U(0.5, 2), spectral index U(0.5, 1.0), spectrum
  ``peak * (nu / nu0) ** -alpha``; a fraction ``point_frac`` of the sources are
  single-pixel deltas instead of Gaussians;
* PSF: ``n_ant`` antennas uniform in [-1, 1]^2; every ordered pair i != j gives
  a baseline; the uv cell is ``round(b * (nu / nu_max) * N / 5)`` (so each
  component stays within 0.4 N); the mask is 1 on every hit cell and on (0, 0);
  the PSF is the real inverse FFT of the mask, moved so its peak sits at pixel
  (N/2, N/2), scaled to a peak of 1;
* noise: per channel, white Gaussian with variance mean((H x*)^2) / 10^(snr/10).
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict

import numpy as np


@dataclass(frozen=True)
class CubeConfig:
    """Shape and recipe of one synthetic cube."""

    name: str
    n: int                 # image side, pixels
    nchan: int             # spectral channels L
    n_src: int
    n_ant: int
    nscales: int           # IUWT detail scales J
    snr_db: float = 20.0
    point_frac: float = 0.0
    seed: int = 1
    iters: int = 100
    freq_lo: float = 1.0e9
    freq_hi: float = 1.5e9
    freq_ref: float = 1.25e9

    def as_dict(self) -> dict:
        return asdict(self)


# The workloads (sizes, source/antenna counts, scales, seeds).
CONFIGS = {
    "64x64x8": CubeConfig("64x64x8", n=64, nchan=8, n_src=5, n_ant=20, nscales=3, seed=1, iters=100),
    "256x256x64": CubeConfig("256x256x64", n=256, nchan=64, n_src=40, n_ant=60, nscales=4, seed=2, iters=200),
    "128x128x16": CubeConfig("128x128x16", n=128, nchan=16, n_src=40, n_ant=60, nscales=4, seed=11),
    "256x256x32": CubeConfig("256x256x32", n=256, nchan=32, n_src=40, n_ant=60, nscales=4, seed=12),
    "512x512x64": CubeConfig("512x512x64", n=512, nchan=64, n_src=40, n_ant=60, nscales=4, seed=13),
    "1024x1024x8": CubeConfig("1024x1024x8", n=1024, nchan=8, n_src=40, n_ant=60, nscales=4, seed=14),
    "512x512x256": CubeConfig("512x512x256", n=512, nchan=256, n_src=200, n_ant=128, nscales=5,
                    point_frac=0.1, seed=3, iters=100),
}


@dataclass
class Cube:
    cfg: CubeConfig
    freqs: np.ndarray       # [L] Hz
    sky: np.ndarray         # [L][N][N] float32, x*
    psf: np.ndarray         # [L][N][N] float32, peak at (N/2, N/2)
    dirty: np.ndarray       # [L][N][N] float32, y
    noise_sigma: np.ndarray = field(default=None)  # [L] float64


def channel_freqs(cfg: CubeConfig) -> np.ndarray:
    return np.linspace(cfg.freq_lo, cfg.freq_hi, cfg.nchan)


def _sky(cfg: CubeConfig, rng: np.random.Generator, freqs: np.ndarray) -> np.ndarray:
    n, L, k = cfg.n, cfg.nchan, cfg.n_src
    cy = rng.uniform(0, n, k)
    cx = rng.uniform(0, n, k)
    width = rng.uniform(1.0, 4.0, k)
    peak = rng.uniform(0.5, 2.0, k)
    alpha = rng.uniform(0.5, 1.0, k)
    is_point = rng.uniform(0.0, 1.0, k) < cfg.point_frac
    spectra = peak[:, None] * (freqs[None, :] / cfg.freq_ref) ** (-alpha[:, None])  # [k][L]
    yy = np.arange(n, dtype=np.float64)[:, None]
    xx = np.arange(n, dtype=np.float64)[None, :]
    profiles = np.zeros((k, n, n))
    for s in range(k):
        if is_point[s]:
            profiles[s, int(cy[s]) % n, int(cx[s]) % n] = 1.0
        else:
            profiles[s] = np.exp(-((yy - cy[s]) ** 2 + (xx - cx[s]) ** 2) / (2.0 * width[s] ** 2))
    sky = np.einsum("kl,kp->lp", spectra, profiles.reshape(k, n * n)).reshape(L, n, n)
    return sky


def _psf(cfg: CubeConfig, rng: np.random.Generator, freqs: np.ndarray) -> np.ndarray:
    n, L = cfg.n, cfg.nchan
    ant = rng.uniform(-1.0, 1.0, (cfg.n_ant, 2))
    i, j = np.nonzero(~np.eye(cfg.n_ant, dtype=bool))
    base = ant[i] - ant[j]                                   # [nb][2], both signs
    psf = np.empty((L, n, n))
    fmax = freqs.max()
    for l in range(L):
        cells = np.rint(base * (freqs[l] / fmax) * n / 5.0).astype(np.int64) % n
        mask = np.zeros((n, n))
        mask[cells[:, 0], cells[:, 1]] = 1.0
        mask[0, 0] = 1.0
        p = np.real(np.fft.ifft2(mask))
        p = np.fft.fftshift(p)
        psf[l] = p / p[n // 2, n // 2]
    return psf


def _instrument(psf: np.ndarray, sky: np.ndarray) -> np.ndarray:
    """Circular convolution of each channel by its PSF (the telescope)."""
    h = np.fft.fft2(np.fft.ifftshift(psf, axes=(-2, -1)), axes=(-2, -1))
    return np.real(np.fft.ifft2(h * np.fft.fft2(sky, axes=(-2, -1)), axes=(-2, -1)))


def make_cube(cfg: CubeConfig | str, seed: int | None = None) -> Cube:
    """Build one cube from its recipe; ``seed`` overrides the config's."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if seed is not None:
        cfg = CubeConfig(**{**cfg.as_dict(), "seed": seed})
    rng = np.random.Generator(np.random.PCG64(cfg.seed))
    freqs = channel_freqs(cfg)
    sky = _sky(cfg, rng, freqs)
    psf = _psf(cfg, rng, freqs)
    clean = _instrument(psf, sky)
    power = np.mean(clean ** 2, axis=(1, 2))
    sigma = np.sqrt(power / 10.0 ** (cfg.snr_db / 10.0))
    noise = rng.standard_normal(clean.shape) * sigma[:, None, None]
    dirty = clean + noise
    return Cube(cfg, freqs, sky.astype(np.float32), psf.astype(np.float32),
                dirty.astype(np.float32), sigma)


def random_state(shape_x: tuple, nscales: int, seed: int, scale: float = 1.0):
    """A random non-trivial primal-dual state (X >= 0, |U| <= 1, |V| <= 1).

    Used to start single-iteration parity checks away from the zero state.
    """
    L, n, _ = shape_x
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (scale * rng.uniform(0.0, 1.0, shape_x)).astype(np.float32)
    x[rng.uniform(0, 1, shape_x) < 0.3] = 0.0
    u = rng.uniform(-1.0, 1.0, (L, nscales + 1, n, n)).astype(np.float32)
    v = rng.uniform(-1.0, 1.0, shape_x).astype(np.float32)
    return x, u, v


def random_field(shape: tuple, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, shape)


# --------------------------------------------------------------------------
# inputs of the warm-start network
# --------------------------------------------------------------------------

# (input features, output features) of the six 3x3x3 layers.
NET_LAYERS = ((1, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 1))


def bf16_round(a) -> np.ndarray:
    """float32 copy of ``a`` rounded to the nearest bfloat16 (ties to even),
    so that a bfloat16 consumer and a float64 checker see the same numbers."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def net_init(seed: int, n_out: int = 1, bf16: bool = True) -> np.ndarray:
    """Seeded initial parameters of the network with n_out output maps, packed
    layer by layer as weights [co][ci][3][3][3] then biases [co]: He-normal
    weights (std sqrt(2 / (27 ci))), zero biases; the last layer is scaled down
    by 10 so the first predictions are small."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    layers = NET_LAYERS[:-1] + ((NET_LAYERS[-1][0], n_out),)
    for k, (ci, co) in enumerate(layers):
        w = rng.standard_normal(co * ci * 27) * np.sqrt(2.0 / (27 * ci))
        if k == len(layers) - 1:
            w *= 0.1
        parts += [w, np.zeros(co)]
    theta = np.concatenate(parts).astype(np.float32)
    return bf16_round(theta) if bf16 else theta


def cube_arrays(args) -> tuple:
    """(seed, dirty, psf) of make_cube(cfg, seed) for args = (cfg, seed); a
    top-level function so that worker processes can build cubes in parallel."""
    cfg, seed = args
    c = make_cube(cfg, seed=seed)
    return seed, c.dirty, c.psf
