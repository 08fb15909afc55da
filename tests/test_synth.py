"""The seeded input generator: deterministic, and shaped as its recipe says."""
import numpy as np

from paper_1602_08847_gb300 import synth


def small(seed=3, **kw):
    base = dict(name="t", n=32, nchan=4, n_src=6, n_ant=12, nscales=2, seed=seed)
    base.update(kw)
    return synth.make_cube(synth.CubeConfig(**base))


def test_same_seed_same_cube_other_seed_other_cube():
    a, b, c = small(3), small(3), small(4)
    assert np.array_equal(a.dirty, b.dirty) and np.array_equal(a.psf, b.psf)
    assert not np.array_equal(a.dirty, c.dirty)


def test_psf_peak_centre_and_point_symmetry():
    cube = small()
    n = cube.cfg.n
    for l in range(cube.cfg.nchan):
        p = cube.psf[l].astype(np.float64)
        assert np.unravel_index(np.argmax(p), p.shape) == (n // 2, n // 2)
        assert abs(p[n // 2, n // 2] - 1.0) < 1e-6
        # a mask holding both signs of every baseline gives a PSF symmetric about its peak
        flipped = np.roll(np.roll(p[::-1, ::-1], 1, axis=0), 1, axis=1)
        assert np.max(np.abs(p - flipped)) < 1e-5


def test_sky_positive_and_spectra_fall_with_frequency():
    cube = small(n_src=1)
    s = cube.sky.reshape(cube.cfg.nchan, -1).sum(axis=1)
    assert cube.sky.min() >= 0.0 and np.all(np.diff(s) < 0)


def test_noise_level_follows_snr():
    cube = small(snr_db=10.0)
    assert np.all(cube.noise_sigma > 0)
    hhat = np.fft.fft2(np.fft.ifftshift(cube.psf.astype(np.float64), axes=(-2, -1)), axes=(-2, -1))
    clean = np.real(np.fft.ifft2(hhat * np.fft.fft2(cube.sky.astype(np.float64), axes=(-2, -1)), axes=(-2, -1)))
    noise = cube.dirty - clean
    ratio = np.mean(clean ** 2) / np.mean(noise ** 2)
    assert 10 ** 0.8 < ratio < 10 ** 1.2


def test_point_sources_fraction():
    cube = small(n_src=40, point_frac=1.0, n=64)
    # all-delta sky: every non-zero pixel of a channel is an isolated source pixel
    assert np.count_nonzero(cube.sky[0]) <= 40


def test_bf16_round_is_nearest_even_on_the_bfloat16_grid():
    from paper_1602_08847_gb300 import synth
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -3.140625, 1e-30], dtype=np.float32)
    r = synth.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                          # tie -> even mantissa
    assert r[2] == np.float32(1.0 + 4 * 2.0 ** -8)   # tie -> even (rounds up)
    assert r[3] == 1.0
    assert r[4] == np.float32(-3.140625)        # already on the grid
    assert (r.view(np.uint32) & 0xFFFF == 0).all()


def test_net_init_sizes():
    from paper_1602_08847_gb300 import synth
    from oracle import warmstart_net as wn
    theta = synth.net_init(0)
    assert theta.size == wn.n_params() == 112481
    assert np.array_equal(theta, synth.bf16_round(theta))
