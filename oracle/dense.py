"""Dense-matrix cross-checks for tiny problems (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` and scripts under ``tests/golden/`` use this module.  It builds
H, W_s and W_lambda of Eqs. 4-6 as explicit matrices acting on vec(X) (channel
major, then row, then column) and minimises Eq. 5 + Eq. 6 with a dense ADMM,
an algorithm of the family of the first MUFFIN version (Sec. 1), independent of
the primal-dual iteration of Algorithm 1.  It also checks the optimality
conditions of a candidate solution directly.
"""
from __future__ import annotations

import numpy as np

from . import muffin_oracle as mo


def operator_matrix(apply, in_shape: tuple) -> np.ndarray:
    """Matrix of a linear map, one column per unit input vector."""
    size = int(np.prod(in_shape))
    cols = []
    for i in range(size):
        e = np.zeros(size)
        e[i] = 1.0
        cols.append(np.asarray(apply(e.reshape(in_shape)), dtype=np.float64).ravel())
    return np.stack(cols, axis=1)


def dense_operators(p: mo.Problem):
    """(H, W_s, W_lambda) as matrices over vec(X), X of shape [L][N][N]."""
    L, n, _ = p.shape
    shape = (L, n, n)
    H = operator_matrix(lambda x: mo.apply_H(x, p.hhat), shape)
    Ws = operator_matrix(lambda x: mo.ws_analysis(p, x), shape)
    Wl = np.kron(mo.dct_matrix(L), np.eye(n * n))
    return H, Ws, Wl


def dense_objective(p: mo.Problem, x: np.ndarray, ops=None) -> float:
    H, Ws, Wl = ops if ops is not None else dense_operators(p)
    L, n, _ = p.shape
    wv = np.repeat(p.w, n * n)
    r = H @ x - p.y.ravel()
    return 0.5 * float(np.sum(wv * r * r)) + p.mu_s * float(np.abs(Ws @ x).sum()) \
        + p.mu_l * float(np.abs(Wl @ x).sum())


def admm_minimize(p: mo.Problem, iters: int = 20000, penalty: float = 1.0, ops=None) -> np.ndarray:
    """Minimise Eq. 5 + Eq. 6 by scaled-form ADMM on x with z = M x.

    M stacks I (positivity block), W_s and W_lambda.  Each pass: x solves
    (H^T W H + c M^T M) x = H^T W y + c M^T (z - u); z is the prox of each block
    at M x + u (projection on x >= 0, soft thresholds mu_s / c and
    mu_lambda / c); u accumulates M x - z.
    """
    H, Ws, Wl = ops if ops is not None else dense_operators(p)
    L, n, _ = p.shape
    wv = np.repeat(p.w, n * n)
    nx = L * n * n
    M = np.vstack([np.eye(nx), Ws, Wl])
    A = H.T @ (wv[:, None] * H) + penalty * (M.T @ M)
    chol = np.linalg.cholesky(A)
    rhs0 = H.T @ (wv * p.y.ravel())
    k1, k2 = nx, nx + Ws.shape[0]
    z = np.zeros(M.shape[0])
    u = np.zeros(M.shape[0])
    x = np.zeros(nx)
    for _ in range(iters):
        rhs = rhs0 + penalty * (M.T @ (z - u))
        x = np.linalg.solve(chol.T, np.linalg.solve(chol, rhs))
        mx = M @ x
        q = mx + u
        z = np.empty_like(q)
        z[:k1] = np.maximum(q[:k1], 0.0)
        z[k1:k2] = np.sign(q[k1:k2]) * np.maximum(np.abs(q[k1:k2]) - p.mu_s / penalty, 0.0)
        z[k2:] = np.sign(q[k2:]) * np.maximum(np.abs(q[k2:]) - p.mu_l / penalty, 0.0)
        u = u + mx - z
    return np.maximum(x, 0.0)


def kkt_residuals(p: mo.Problem, s: mo.State, tol_zero: float = 1e-9) -> dict:
    """Violations of the optimality conditions of Eqs. 5-6 at (X, U, V).

    With g = grad f(X) + mu_s W_s^T U + mu_lambda W_lambda^T V, X is optimal
    when (i) |U|, |V| <= 1, (ii) U = sign(W_s X) and V = sign(W_lambda X)
    wherever those coefficients are non-zero, (iii) g = 0 where X > 0 and
    g >= 0 where X = 0.  Returns the largest violation of each.
    """
    X, U, V = s.X, s.U, s.V
    g = mo.gradient(X, p.y, p.hhat, p.w) + p.mu_s * mo.ws_adjoint(p, U) \
        + p.mu_l * mo.spectral_adjoint(V)
    ws = mo.ws_analysis(p, X)
    wl = mo.spectral_analysis(X)
    scale = max(1.0, float(np.abs(g).max()))
    out = {
        "dual_box": float(max(np.abs(U).max(), np.abs(V).max()) - 1.0),
        "sign_U": float(np.abs(U - np.sign(ws))[np.abs(ws) > tol_zero].max(initial=0.0)),
        "sign_V": float(np.abs(V - np.sign(wl))[np.abs(wl) > tol_zero].max(initial=0.0)),
        "stationary": float(np.abs(g[X > tol_zero]).max(initial=0.0)) / scale,
        "complementary": float(np.maximum(-g[X <= tol_zero], 0.0).max(initial=0.0)) / scale,
    }
    return out


def smoothed_projected_gradient(p: mo.Problem, ops=None, eps_list=(1e-2, 1e-4, 1e-6, 1e-8, 1e-10),
                                iters_per_eps: int = 20000) -> np.ndarray:
    """Brute-force minimiser: accelerated projected gradient on x >= 0 of
    Eq. 5 + Eq. 6 with each |t| of the l1 terms replaced by the Huber function
    of width eps, eps decreasing to 1e-10 (continuation, warm-started).
    Its error against the exact minimiser is O(eps).
    """
    H, Ws, Wl = ops if ops is not None else dense_operators(p)
    L, n, _ = p.shape
    wv = np.repeat(p.w, n * n)
    yv = p.y.ravel()
    HtWH = H.T @ (wv[:, None] * H)
    HtWy = H.T @ (wv * yv)
    lip_data = float(np.linalg.eigvalsh(HtWH).max())
    lip_ws = float(np.linalg.eigvalsh(Ws.T @ Ws).max())
    lip_wl = float(np.linalg.eigvalsh(Wl.T @ Wl).max())

    def huber_grad(t, eps):
        return np.clip(t / eps, -1.0, 1.0)

    x = np.zeros(L * n * n)
    for eps in eps_list:
        step = 1.0 / (lip_data + (p.mu_s * lip_ws + p.mu_l * lip_wl) / eps)
        z, xprev, tk = x.copy(), x.copy(), 1.0
        for _ in range(iters_per_eps):
            g = HtWH @ z - HtWy + p.mu_s * (Ws.T @ huber_grad(Ws @ z, eps)) \
                + p.mu_l * (Wl.T @ huber_grad(Wl @ z, eps))
            xn = np.maximum(z - step * g, 0.0)
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
            z = xn + ((tk - 1.0) / tn) * (xn - xprev)
            xprev, tk = xn, tn
        x = xprev
    return x
