"""The 8 x 8 x 2 test problem shared by the golden-fixture script and the tests.

A strictly convex instance of Eqs. 5-6: a Gaussian PSF of width 0.5 px with
unit sum (full rank on the 8 x 8 grid), two channels, two point sources with
different spectra and a little Gaussian noise.
"""
import numpy as np

N, L = 8, 2


def tiny_inputs(seed: int = 5):
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:N, 0:N]
    g = np.exp(-((yy - N // 2) ** 2 + (xx - N // 2) ** 2) / (2 * 0.5 ** 2))
    psf = np.stack([g / g.sum()] * L)
    sky = np.zeros((L, N, N))
    sky[:, 2, 3] = [1.0, 0.8]
    sky[:, 5, 5] = [0.5, 0.6]
    hhat = np.fft.fft2(np.fft.ifftshift(psf, axes=(-2, -1)), axes=(-2, -1))
    clean = np.real(np.fft.ifft2(hhat * np.fft.fft2(sky, axes=(-2, -1)), axes=(-2, -1)))
    y = clean + 0.01 * rng.standard_normal((L, N, N))
    return y, psf, sky


CASES = {
    "gen1_J1": dict(J=1, gen=1, mu_s=0.05, mu_l=0.05),
    "gen2_J1": dict(J=1, gen=2, mu_s=0.03, mu_l=0.08),
    "union_J2": dict(J=2, gen=1, mu_s=0.01, mu_l=0.02, dictionary="union"),
}
