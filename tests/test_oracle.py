"""Pins of the FP64 oracle against facts fixed by the paper and the mathematics.

Nothing here compares the oracle with itself: every check is a closed form, an
invariant, a library special case, a brute-force computation on a tiny input or
an independent minimiser (tests/golden).
"""
import json
import os

import numpy as np
import pytest
import scipy.fft

from oracle import muffin_oracle as mo
from oracle import dense
from tiny_problem import tiny_inputs, CASES

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rnd(shape, seed, lo=-1.0, hi=1.0):
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, shape)


# ---------------------------------------------------------------- H (Eq. 4)

def test_H_equals_direct_circular_convolution():
    """Eq. 4: H_l is convolution by the PSF; compare with the O(N^4) double sum."""
    n = 8
    psf = rnd((n, n), 1)          # not symmetric: catches a flipped kernel
    x = rnd((n, n), 2)
    fast = mo.apply_H(x[None], mo.psf_multiplier(psf[None]))[0]
    slow = mo.convolve_direct(x, psf)
    assert np.max(np.abs(fast - slow)) < 1e-12


def test_H_of_delta_is_psf_centred_on_the_delta():
    n = 16
    psf = rnd((n, n), 3)
    x = np.zeros((n, n))
    x[3, 11] = 1.0
    out = mo.apply_H(x[None], mo.psf_multiplier(psf[None]))[0]
    expect = np.roll(np.roll(psf, 3 - n // 2, axis=0), 11 - n // 2, axis=1)
    assert np.max(np.abs(out - expect)) < 1e-12


def test_H_adjoint_identity():
    n, L = 16, 3
    hh = mo.psf_multiplier(rnd((L, n, n), 4))
    x, y = rnd((L, n, n), 5), rnd((L, n, n), 6)
    lhs = np.vdot(mo.apply_H(x, hh), y)
    rhs = np.vdot(x, mo.apply_Ht(y, hh))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_data_lipschitz_matches_closed_form():
    """||H_l^T H_l|| = max |hhat_l|^2 (H_l is circulant); beta = max over l of w_l times it."""
    n, L = 16, 3
    yy, xx = np.mgrid[0:n, 0:n]
    psf = np.stack([np.exp(-((yy - n // 2) ** 2 + (xx - n // 2) ** 2) / (2 * s * s)) for s in (0.7, 1.0, 1.5)])
    hh = mo.psf_multiplier(psf)
    w = np.array([1.0, 2.0, 0.5])
    closed = max(w[l] * np.max(np.abs(hh[l]) ** 2) for l in range(L))
    est = mo.data_lipschitz(hh, w, n_iter=300)
    assert abs(est - closed) / closed < 1e-6


def test_gradient_matches_finite_difference_of_data_term():
    """Eq. 8 is the gradient of the data term of Eq. 5 (weights included)."""
    n, L = 8, 2
    psf = rnd((L, n, n), 7)
    y = rnd((L, n, n), 8)
    p = mo.Problem(y=y, hhat=mo.psf_multiplier(psf), J=1, mu_s=0.0, mu_l=0.0, w=np.array([1.5, 0.25]))
    x, d = rnd((L, n, n), 9, 0, 1), rnd((L, n, n), 10)
    f = lambda z: mo.objective_terms(p, z)[0]  # noqa: E731
    h = 1e-5
    fd = (f(x + h * d) - f(x - h * d)) / (2 * h)
    assert abs(fd - np.vdot(mo.gradient(x, p.y, p.hhat, p.w), d)) < 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------- W_s (IUWT)

def test_b3_filter_impulse_response_at_each_dilation():
    """H_j of a delta is the outer product of [1,4,6,4,1]/16 with taps 2^j apart."""
    n = 32
    for j in range(4):
        d = 2 ** j
        x = np.zeros((n, n))
        x[0, 0] = 1.0
        out = mo.smooth(x, j)
        expect = np.zeros((n, n))
        for a in range(5):
            for b in range(5):
                expect[((a - 2) * d) % n, ((b - 2) * d) % n] += mo.B3[a] * mo.B3[b]
        assert np.max(np.abs(out - expect)) < 1e-15
    assert abs(mo.B3.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("J", [1, 3, 4])
def test_gen1_detail_planes_plus_coarse_reconstruct_input(J):
    x = rnd((2, 32, 32), 11)
    w = mo.iuwt_analysis(x, J, 1)
    assert w.shape == (2, J + 1, 32, 32)
    assert np.max(np.abs(w.sum(axis=-3) - x)) < 1e-12


@pytest.mark.parametrize("J", [1, 3, 4])
def test_gen2_recursive_synthesis_reconstructs_input(J):
    x = rnd((2, 32, 32), 12)
    w = mo.iuwt_analysis(x, J, 2)
    assert np.max(np.abs(mo.iuwt_synthesis(w, J, 2) - x)) < 1e-12
    # generation 2 is not generation 1: its details do not sum to x
    assert np.max(np.abs(w.sum(axis=-3) - x)) > 1e-3


@pytest.mark.parametrize("gen", [1, 2])
@pytest.mark.parametrize("n,J", [(16, 1), (16, 3), (32, 4), (64, 3)])
def test_iuwt_adjoint_identity(gen, n, J):
    """<W_s x, u> = <x, W_s^T u>, including dilations that wrap the grid."""
    x = rnd((2, n, n), 13)
    u = rnd((2, J + 1, n, n), 14)
    lhs = np.vdot(mo.iuwt_analysis(x, J, gen), u)
    rhs = np.vdot(x, mo.iuwt_adjoint(u, J, gen))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("gen", [1, 2])
def test_iuwt_adjoint_is_matrix_transpose(gen):
    n, J = 8, 2
    A = dense.operator_matrix(lambda x: mo.iuwt_analysis(x, J, gen), (n, n))
    At = dense.operator_matrix(lambda u: mo.iuwt_adjoint(u, J, gen), (J + 1, n, n))
    assert np.max(np.abs(A.T - At)) < 1e-14


def test_iuwt_special_cases():
    x = rnd((16, 16), 15)
    for gen in (1, 2):
        w0 = mo.iuwt_analysis(x, 0, gen)
        assert w0.shape == (1, 16, 16) and np.array_equal(w0[0], x)   # J = 0: identity
        c = np.full((16, 16), 2.5)                                    # DC: no detail
        w = mo.iuwt_analysis(c, 3, gen)
        assert np.max(np.abs(w[:3])) < 1e-14 and np.max(np.abs(w[3] - c)) < 1e-14


@pytest.mark.parametrize("gen", [1, 2])
def test_iuwt_norm_power_iteration_matches_transfer_functions(gen):
    n, J = 32, 3
    closed = mo.iuwt_norm2_closed_form(n, J, gen)
    est = mo.iuwt_norm2(n, J, gen, n_iter=400)
    # the power method approaches from below; the spectrum near the top is dense
    assert est <= closed * (1 + 1e-12) and (closed - est) / closed < 1e-3
    dense_norm = np.linalg.eigvalsh(
        (lambda A: A.T @ A)(dense.operator_matrix(lambda x: mo.iuwt_analysis(x, 2, gen), (8, 8)))).max()
    assert abs(dense_norm - mo.iuwt_norm2_closed_form(8, 2, gen)) < 1e-12


# ---------------------------------------------------------------- W_lambda (DCT)

def test_dct_orthonormal_and_equals_scipy():
    for L in (1, 2, 7, 8, 15, 64):
        C = mo.dct_matrix(L)
        assert np.max(np.abs(C @ C.T - np.eye(L))) < 1e-14
        x = rnd((L, 5, 6), 16)
        ref = scipy.fft.dct(x, type=2, norm="ortho", axis=0)
        assert np.max(np.abs(mo.spectral_analysis(x) - ref)) < 1e-13
        assert np.max(np.abs(mo.spectral_adjoint(x) - scipy.fft.idct(x, type=2, norm="ortho", axis=0))) < 1e-13
    x = rnd((1, 4, 4), 17)
    assert np.allclose(mo.spectral_analysis(x), x, atol=0, rtol=1e-15)


def test_dct_adjoint_identity():
    x, v = rnd((11, 6, 6), 18), rnd((11, 6, 6), 19)
    lhs = np.vdot(mo.spectral_analysis(x), v)
    rhs = np.vdot(x, mo.spectral_adjoint(v))
    assert abs(lhs - rhs) < 1e-12


# ---------------------------------------------------------------- prox maps (Eq. 7)

def test_sat_and_positive():
    u = np.array([-3.0, -1.0, -0.5, 0.0, 0.25, 1.0, 7.0])
    assert np.array_equal(mo.sat(u), [-1.0, -1.0, -0.5, 0.0, 0.25, 1.0, 1.0])
    assert np.array_equal(mo.positive(u), [0.0, 0.0, 0.0, 0.0, 0.25, 1.0, 7.0])


# ---------------------------------------------------------------- Algorithm 1

def _delta_psf(L, n):
    psf = np.zeros((L, n, n))
    psf[:, n // 2, n // 2] = 1.0
    return psf


def test_no_regularisation_identity_psf_fixed_point_is_positive_part():
    """mu_s = mu_lambda = 0 and H = I: the minimiser of Eq. 5 over X >= 0 is max(y, 0)."""
    L, n = 3, 16
    y = rnd((L, n, n), 20)
    p = mo.Problem(y=y, hhat=mo.psf_multiplier(_delta_psf(L, n)), J=2, mu_s=0.0, mu_l=0.0,
                   tau=0.9, sigma=1.0)
    s = mo.iterate(p, mo.zero_state(p), 200)
    assert np.max(np.abs(s.X - np.maximum(y, 0.0))) < 1e-12


def test_zero_spectral_weight_separates_channels():
    """Sec. 4, step 1: with mu_lambda = 0 each channel evolves on its own."""
    cube_y, psf, _ = tiny_inputs()
    y = np.concatenate([cube_y, 2 * cube_y])
    psf = np.concatenate([psf, psf])
    p = mo.make_problem(y, psf, 1, mu_s=0.05, mu_l=0.0, tau=0.8, sigma=2.0)
    whole = mo.iterate(p, mo.zero_state(p), 30)
    for l in range(y.shape[0]):
        pl = mo.make_problem(y[l:l + 1], psf[l:l + 1], 1, mu_s=0.05, mu_l=0.0, tau=0.8, sigma=2.0)
        one = mo.iterate(pl, mo.zero_state(pl), 30)
        assert np.array_equal(one.X[0], whole.X[l])
        assert np.array_equal(one.U[0], whole.U[l])


def test_iterates_stay_feasible():
    from paper_1602_08847_gb300 import synth
    cube = synth.make_cube(synth.CubeConfig("t", n=32, nchan=4, n_src=3, n_ant=10, nscales=2, seed=4))
    p = mo.make_problem(cube.dirty, cube.psf, 2, mu_s=0.25, mu_l=3.0)
    s = mo.zero_state(p)
    for _ in range(10):
        s = mo.iterate(p, s, 1)
        assert s.X.min() >= 0.0 and np.abs(s.U).max() <= 1.0 and np.abs(s.V).max() <= 1.0


@pytest.mark.parametrize("case", list(CASES))
def test_algorithm1_reaches_independent_minimiser(case):
    """Tiny 8x8x2 problem: Algorithm 1 ends at the minimiser found by dense ADMM
    and by smoothed projected gradient (tests/golden), and meets the KKT conditions."""
    with open(os.path.join(GOLDEN, f"tiny_minimizer_{case}.json")) as f:
        g = json.load(f)
    c = g["case"]
    y, psf, _ = tiny_inputs()
    dic = c.get("dictionary", "iuwt")
    p = mo.make_problem(y, psf, c["J"], gen=c["gen"], mu_s=c["mu_s"], mu_l=c["mu_l"], tau=1.0, dictionary=dic)
    beta = float(np.max(np.abs(p.hhat) ** 2))
    ws2 = 1.0 if dic == "union" else mo.iuwt_norm2_closed_form(8, p.J, p.gen)   # the union is a tight frame
    l2 = mo.dual_norm2(p.mu_s, p.mu_l, ws2)
    p.tau = 1.0 / beta
    p.sigma = 0.9 * (1.0 / p.tau - beta / 2) / l2          # Condat: 1/tau - sigma ||L||^2 > beta/2
    # the union's eight bases give 8x more dual coefficients, which converge more slowly
    s = mo.iterate(p, mo.zero_state(p), 12000 if dic == "union" else 4000)
    x_ref = np.array(g["x"])
    assert np.linalg.norm(s.X.ravel() - x_ref) / np.linalg.norm(x_ref) < 1e-6
    assert abs(mo.objective(p, s.X) - g["objective"]) / g["objective"] < 1e-9
    kkt = dense.kkt_residuals(p, s, tol_zero=1e-7)
    assert kkt["dual_box"] <= 0.0 and kkt["sign_U"] < 1e-6 and kkt["sign_V"] < 1e-6
    assert kkt["stationary"] < 1e-8 and kkt["complementary"] < 1e-8


def _p_norm2(p, dx, du, dv):
    """||(dx, du, dv)||^2 in the metric P = [[I/tau, -L^T], [-L, I/sigma]]."""
    cross = p.mu_s * np.vdot(mo.iuwt_analysis(dx, p.J, p.gen), du) \
        + p.mu_l * np.vdot(mo.spectral_analysis(dx), dv)
    return np.vdot(dx, dx) / p.tau + (np.vdot(du, du) + np.vdot(dv, dv)) / p.sigma - 2.0 * cross


@pytest.mark.parametrize("gen", [1, 2])
def test_successive_differences_shrink_in_condat_metric(gen):
    """Under Condat's step condition one pass of Algorithm 1 is an averaged
    operator in the metric P, so ||z_{k+1} - z_k||_P never grows.  This pins
    the extrapolation 2 X~ - X and the signs of the dual terms, which the
    minimiser alone does not."""
    y, psf, _ = tiny_inputs()
    p = mo.make_problem(y, psf, 1, gen=gen, mu_s=0.05, mu_l=0.05, tau=1.0)
    beta = float(np.max(np.abs(p.hhat) ** 2))
    l2 = mo.dual_norm2(p.mu_s, p.mu_l, mo.iuwt_norm2_closed_form(8, p.J, p.gen))
    p.tau = 0.5 / beta
    p.sigma = 0.9 * (1.0 / p.tau - beta / 2) / l2
    s = mo.zero_state(p)
    prev, first = None, None
    for _ in range(300):
        s2 = mo.iterate(p, s, 1)
        d = _p_norm2(p, s2.X - s.X, s2.U - s.U, s2.V - s.V)
        first = d if first is None else first
        if prev is not None and d > 1e-18 * first:
            assert d <= prev * (1 + 1e-9)
        prev, s = d, s2


def _relaxed_tiny_problem(case, rho):
    """The 8x8x2 problem of tests/golden with steps that admit rho up to delta = 1.6:
    tau = 1/(2 beta) and sigma ||L||^2 = (1/tau - beta/2)/2, so 1/tau - sigma ||L||^2 = 1.25 beta."""
    with open(os.path.join(GOLDEN, f"tiny_minimizer_{case}.json")) as f:
        g = json.load(f)
    c = g["case"]
    y, psf, _ = tiny_inputs()
    p = mo.make_problem(y, psf, c["J"], gen=c["gen"], mu_s=c["mu_s"], mu_l=c["mu_l"], tau=1.0)
    beta = float(np.max(np.abs(p.hhat) ** 2))
    l2 = mo.dual_norm2(p.mu_s, p.mu_l, mo.iuwt_norm2_closed_form(8, p.J, p.gen))
    p.tau = 0.5 / beta
    p.sigma = 0.5 * (1.0 / p.tau - beta / 2) / l2
    delta = 2.0 - 0.5 * beta / (1.0 / p.tau - p.sigma * l2)
    assert 0.0 < rho < delta
    p.rho = rho
    return p, g


@pytest.mark.parametrize("rho", [0.6, 1.5])
@pytest.mark.parametrize("case", ["gen1_J1", "gen2_J1"])
def test_relaxed_iteration_reaches_independent_minimiser(case, rho):
    """Alg. 1, relaxation step (Sec. 3, Eqs. 12 and 14): for any rho in (0, delta) the
    relaxed iteration has the fixed points of the unrelaxed one, so it must end at the
    minimiser that dense ADMM and smoothed projected gradient found (tests/golden).
    At rho = 1.5 a relaxation line with rho and 1 - rho swapped weighs the new iterate
    by -0.5 and diverges."""
    p, g = _relaxed_tiny_problem(case, rho)
    s = mo.iterate(p, mo.zero_state(p), 2000)
    x_ref = np.array(g["x"])
    assert np.linalg.norm(s.X.ravel() - x_ref) / np.linalg.norm(x_ref) < 1e-6
    assert abs(mo.objective(p, s.X) - g["objective"]) / g["objective"] < 1e-9


@pytest.mark.parametrize("rho", [0.6, 1.5])
def test_relaxed_successive_differences_shrink_in_condat_metric(rho):
    """For rho < delta the relaxed pass (1 - rho) I + rho T is still averaged in Condat's
    metric P (a Krasnosel'skii-Mann iteration), so ||z_{k+1} - z_k||_P never grows."""
    p, _ = _relaxed_tiny_problem("gen1_J1", rho)
    s = mo.zero_state(p)
    prev, first = None, None
    for _ in range(300):
        s2 = mo.iterate(p, s, 1)
        d = _p_norm2(p, s2.X - s.X, s2.U - s.U, s2.V - s.V)
        first = d if first is None else first
        if prev is not None and d > 1e-18 * first:
            assert d <= prev * (1 + 1e-9)
        prev, s = d, s2


@pytest.mark.parametrize("rho", [0.6, 1.3, 1.5])
def test_relaxed_primal_trajectory_closed_form(rho):
    """H = I and mu_s = mu_lambda = 0, from X = 0: where y > 0 the relaxed primal step is
    X <- X + rho tau (y - X), so X_k = y (1 - (1 - rho tau)^k) exactly; where y <= 0, X
    stays 0; the duals never move.  This fixes the weight rho of the new iterate in the
    primal relaxation line, which the fixed point alone does not."""
    L, n, tau = 2, 8, 0.5
    y = rnd((L, n, n), 23)
    p = mo.Problem(y=y, hhat=mo.psf_multiplier(_delta_psf(L, n)), J=1, mu_s=0.0, mu_l=0.0,
                   tau=tau, sigma=1.0, rho=rho)
    s = mo.zero_state(p)
    for k in range(1, 9):
        s = mo.iterate(p, s, 1)
        want = np.where(y > 0, y * (1.0 - (1.0 - rho * tau) ** k), 0.0)
        assert np.max(np.abs(s.X - want)) < 1e-14
        assert not s.U.any() and not s.V.any()


def test_condat_step_sizes():
    tau, sigma, rho, delta = mo.condat_steps(2.0, 5.0, sigma=1.0)
    assert 1.0 / tau - sigma * 5.0 > 1.0 and 1.0 <= delta < 2.0 and rho == 1.0
    with pytest.raises(ValueError):
        mo.condat_steps(2.0, 5.0, rho=delta + 1e-3)


def test_objective_special_cases():
    L, n = 2, 8
    y = rnd((L, n, n), 21)
    p = mo.Problem(y=y, hhat=mo.psf_multiplier(_delta_psf(L, n)), J=1, mu_s=0.3, mu_l=0.7,
                   w=np.array([2.0, 0.5]))
    data, sp, sl = mo.objective_terms(p, np.zeros((L, n, n)))
    assert abs(data - 0.5 * (2.0 * np.sum(y[0] ** 2) + 0.5 * np.sum(y[1] ** 2))) < 1e-12
    assert sp == 0.0 and sl == 0.0
    # a constant cube: IUWT puts it all in the coarse plane, the DCT all in DC
    X = np.full((L, n, n), 1.5)
    _, sp, sl = mo.objective_terms(p, X)
    assert abs(sp - 0.3 * L * n * n * 1.5) < 1e-11
    assert abs(sl - 0.7 * n * n * 1.5 * np.sqrt(L)) < 1e-11


def test_snr_definition():
    X = rnd((2, 8, 8), 22)
    assert abs(mo.snr_db(0.9 * X, X) - 20.0) < 1e-12


# ---------------------------------------------------------------- W_s as a union of Daubechies bases (Sec. 4)

@pytest.mark.parametrize("p", range(1, 9))
def test_daubechies_filter_definition(p):
    """Sum sqrt(2), orthonormal even shifts, p vanishing moments of the mirror filter."""
    h = mo.daubechies_lowpass(p)
    t = np.arange(h.size)
    assert h.size == 2 * p
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-12
    for m in range(p):
        assert abs(np.dot(h[:h.size - 2 * m], h[2 * m:]) - (1.0 if m == 0 else 0.0)) < 1e-12
    g = mo.daubechies_highpass(h)
    for m in range(p):
        assert abs(np.sum(t ** m * g)) <= 1e-12 * np.sum(t ** m * np.abs(g)) + 1e-14


def test_daubechies_closed_forms():
    assert np.allclose(mo.daubechies_lowpass(1), [2 ** -0.5, 2 ** -0.5], rtol=0, atol=1e-15)
    r3 = np.sqrt(3.0)
    db2 = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * np.sqrt(2.0))
    assert np.allclose(mo.daubechies_lowpass(2), db2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 5, 8])
@pytest.mark.parametrize("n,J", [(8, 2), (16, 3), (32, 1)])
def test_dwt2_orthogonal_and_adjoint(p, n, J):
    """The periodised filter bank is orthonormal at every level, including
    levels shorter than the filter (db8 at 4 x 4 wraps around)."""
    h = mo.daubechies_lowpass(p)
    x = rnd((2, n, n), 30 + p)
    u = rnd((2, n, n), 40 + p)
    c = mo.dwt2(x, h, J)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert abs(np.vdot(c, u) - np.vdot(x, mo.dwt2_adjoint(u, h, J))) < 1e-12 * n * n
    assert np.max(np.abs(mo.dwt2_adjoint(c, h, J) - x)) < 1e-12


def test_haar_level_on_two_by_two_blocks():
    """Haar (p = 1), one level: block [[a, b], [c, d]] gives (a+b+c+d)/2 (top-left
    quadrant), (a-b+c-d)/2 (top-right), (a+b-c-d)/2 (bottom-left), (a-b-c+d)/2."""
    x = rnd((1, 8, 8), 50)
    c = mo.dwt2(x, mo.daubechies_lowpass(1), 1)[0]
    a, b, cc, d = x[0, 0::2, 0::2], x[0, 0::2, 1::2], x[0, 1::2, 0::2], x[0, 1::2, 1::2]
    assert np.allclose(c[:4, :4], (a + b + cc + d) / 2, atol=1e-14)
    assert np.allclose(c[:4, 4:], (a - b + cc - d) / 2, atol=1e-14)
    assert np.allclose(c[4:, :4], (a + b - cc - d) / 2, atol=1e-14)
    assert np.allclose(c[4:, 4:], (a - b - cc + d) / 2, atol=1e-14)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_constant_image_has_only_coarse_coefficients(p):
    """Every detail filter kills constants; each level multiplies DC by 2 (sqrt 2 per axis)."""
    n, J = 16, 3
    c = mo.dwt2(np.full((1, n, n), 0.7), mo.daubechies_lowpass(p), J)[0]
    m = n >> J
    assert np.allclose(c[:m, :m], 0.7 * 2 ** J, atol=1e-12)
    c[:m, :m] = 0.0
    assert np.max(np.abs(c)) < 1e-12


def test_union_of_bases_is_a_tight_frame():
    x = rnd((2, 16, 16), 60)
    w = mo.union_analysis(x, 3)
    assert w.shape == (2, 8, 16, 16)
    assert abs(np.linalg.norm(w) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.max(np.abs(mo.union_adjoint(w, 3) - x)) < 1e-12
    u = rnd((2, 8, 16, 16), 61)
    assert abs(np.vdot(w, u) - np.vdot(x, mo.union_adjoint(u, 3))) < 1e-11
    assert abs(mo.union_norm2(16, 3) - 1.0) < 1e-12
    # the eight bases differ: the union is redundant, not eight copies of one basis
    assert np.linalg.norm(w[:, 0] - w[:, 1]) > 0.1 * np.linalg.norm(w[:, 0])


def test_planted_mirror_filter_mistake_is_caught(monkeypatch):
    """A highpass without the alternating sign is not orthogonal to the lowpass."""
    mo._step_matrices.cache_clear()          # the step matrices are built from the filters
    monkeypatch.setattr(mo, "daubechies_highpass", lambda h: h[::-1].copy())
    x = rnd((1, 16, 16), 62)
    c = mo.dwt2(x, mo.daubechies_lowpass(3), 2)
    mo._step_matrices.cache_clear()
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) > 1e-3 * np.linalg.norm(x)


def test_successive_differences_shrink_in_condat_metric_union():
    y, psf, _ = tiny_inputs()
    p = mo.make_problem(y, psf, 2, mu_s=0.01, mu_l=0.02, tau=1.0, dictionary="union")
    beta = float(np.max(np.abs(p.hhat) ** 2))
    p.tau = 0.5 / beta
    p.sigma = 0.9 * (1.0 / p.tau - beta / 2) / mo.dual_norm2(p.mu_s, p.mu_l, 1.0)
    s = mo.zero_state(p)
    prev, first = None, None
    for _ in range(200):
        s2 = mo.iterate(p, s, 1)
        dx, du, dv = s2.X - s.X, s2.U - s.U, s2.V - s.V
        cross = p.mu_s * np.vdot(mo.union_analysis(dx, p.J), du) + p.mu_l * np.vdot(mo.spectral_analysis(dx), dv)
        d = np.vdot(dx, dx) / p.tau + (np.vdot(du, du) + np.vdot(dv, dv)) / p.sigma - 2.0 * cross
        first = d if first is None else first
        if prev is not None and d > 1e-18 * first:
            assert d <= prev * (1 + 1e-9)
        prev, s = d, s2


# ---------------------------------------------------------------- the pins catch planted mistakes

@pytest.mark.parametrize("plant", ["grad_sign", "dilation", "dct_transpose", "adjoint_gen", "relax", "relax_rho"])
def test_planted_mistakes_are_caught(plant, monkeypatch):
    """Plant a plausible bug in the oracle (CPU) and check a pin above fails."""
    if plant == "grad_sign":
        orig = mo.apply_Ht
        monkeypatch.setattr(mo, "apply_Ht", lambda x, h: orig(x, np.conj(h)))   # H instead of H^T
        with pytest.raises(AssertionError):
            test_H_adjoint_identity()
    elif plant == "dilation":
        orig = mo.smooth
        monkeypatch.setattr(mo, "smooth", lambda c, j: orig(c, max(j - 1, 0)))
        with pytest.raises(AssertionError):
            test_b3_filter_impulse_response_at_each_dilation()
    elif plant == "dct_transpose":
        orig = mo.dct_matrix
        monkeypatch.setattr(mo, "dct_matrix", lambda L: orig(L).T)
        with pytest.raises(AssertionError):
            test_dct_orthonormal_and_equals_scipy()
    elif plant == "adjoint_gen":
        orig = mo.iuwt_adjoint
        monkeypatch.setattr(mo, "iuwt_adjoint", lambda u, J, gen=1: orig(u, J, 1))
        with pytest.raises(AssertionError):
            test_iuwt_adjoint_identity(2, 16, 3)
    elif plant == "relax":
        orig = mo.iterate

        def wrong(p, s, n_iter=1):   # dual step at X~ instead of 2 X~ - X
            X, U, V = s.X, s.U, s.V
            for _ in range(n_iter):
                Xt = mo.positive(X - p.tau * (mo.gradient(X, p.y, p.hhat, p.w)
                                              + p.mu_s * mo.iuwt_adjoint(U, p.J, p.gen)
                                              + p.mu_l * mo.spectral_adjoint(V)))
                U = mo.sat(U + p.sigma * p.mu_s * mo.iuwt_analysis(Xt, p.J, p.gen))
                V = mo.sat(V + p.sigma * p.mu_l * mo.spectral_analysis(Xt))
                X = Xt
            return mo.State(X, U, V, s.it + n_iter)
        monkeypatch.setattr(mo, "iterate", wrong)
        with pytest.raises(AssertionError):
            test_successive_differences_shrink_in_condat_metric(1)
    elif plant == "relax_rho":
        def swapped(p, s, n_iter=1):   # rho and 1 - rho exchanged in the three relaxation lines
            X, U, V = s.X, s.U, s.V
            for _ in range(n_iter):
                Xt = mo.positive(X - p.tau * (mo.gradient(X, p.y, p.hhat, p.w)
                                              + p.mu_s * mo.ws_adjoint(p, U)
                                              + p.mu_l * mo.spectral_adjoint(V)))
                Ut = mo.sat(U + p.sigma * p.mu_s * mo.ws_analysis(p, 2.0 * Xt - X))
                Vt = mo.sat(V + p.sigma * p.mu_l * mo.spectral_analysis(2.0 * Xt - X))
                X = (1.0 - p.rho) * Xt + p.rho * X
                U = (1.0 - p.rho) * Ut + p.rho * U
                V = (1.0 - p.rho) * Vt + p.rho * V
            return mo.State(X, U, V, s.it + n_iter)
        monkeypatch.setattr(mo, "iterate", swapped)
        with pytest.raises((AssertionError, FloatingPointError)):
            with np.errstate(all="ignore"):
                test_relaxed_iteration_reaches_independent_minimiser("gen1_J1", 1.5)
        with pytest.raises(AssertionError):
            test_relaxed_primal_trajectory_closed_form(0.6)
