"""Pins of the oracle L-BFGS (Sec. II.A minimises the discrete free energy with
L-BFGS) against definitions other than its own code: the two-loop direction
equals the inverse BFGS updates applied one pair at a time to an explicit
matrix; every accepted line-search step satisfies the strong Wolfe conditions;
the minimiser reaches the closed-form minimum of a quadratic and the known
minimum of the Rosenbrock function."""
import math

import numpy as np
import pytest

from oracle import lbfgs


def _bfgs_inverse(S, Y, gamma):
    """H from H0 = gamma I by H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T."""
    n = S[0].size
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / float(s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


@pytest.mark.parametrize("m,n,seed", [(1, 5, 0), (4, 12, 1), (10, 40, 2)])
def test_two_loop_equals_explicit_bfgs_matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    Hs = A @ A.T + n * np.eye(n)          # SPD, so s.y > 0 for y = Hs s
    S = [rng.standard_normal(n) for _ in range(m)]
    Y = [Hs @ s for s in S]
    R = [1.0 / float(s @ y) for s, y in zip(S, Y)]
    g = rng.standard_normal(n)
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    Hg = _bfgs_inverse(S, Y, gamma) @ g
    np.testing.assert_allclose(lbfgs.two_loop(g, S, Y, R, gamma), Hg, rtol=1e-10,
                               atol=1e-12 * np.abs(Hg).max())


def test_two_loop_secant_condition():
    # the newest pair is reproduced exactly: H y_k = s_k
    rng = np.random.default_rng(3)
    n = 9
    A = rng.standard_normal((n, n))
    Hs = A @ A.T + np.eye(n)
    S = [rng.standard_normal(n) for _ in range(3)]
    Y = [Hs @ s for s in S]
    R = [1.0 / float(s @ y) for s, y in zip(S, Y)]
    out = lbfgs.two_loop(Y[-1], S, Y, R, 0.7)
    np.testing.assert_allclose(out, S[-1], rtol=1e-10, atol=1e-12)


def _rosenbrock(x):
    a, b = x[0], x[1]
    f = (1.0 - a) ** 2 + 100.0 * (b - a * a) ** 2
    g = np.array([-2.0 * (1.0 - a) - 400.0 * a * (b - a * a), 200.0 * (b - a * a)])
    return f, g


@pytest.mark.parametrize("x0", [(-1.2, 1.0), (0.0, 0.0), (2.0, -1.0), (-0.5, 2.5)])
def test_line_search_meets_strong_wolfe(x0):
    x = np.array(x0, dtype=float)
    f, g = _rosenbrock(x)
    for alpha0 in (1.0, 1e-3, 10.0):
        d = -g
        a, xn, fn, gn, trials = lbfgs.line_search(_rosenbrock, x, f, g, d, alpha0=alpha0)
        assert a > 0 and trials <= 20
        dg0 = float(g @ d)
        assert fn <= f + 1e-4 * a * dg0                     # sufficient decrease
        assert abs(float(gn @ d)) <= 0.9 * abs(dg0)         # curvature (strong form)
        np.testing.assert_allclose(xn, x + a * d, rtol=0, atol=1e-15)
        assert fn == _rosenbrock(xn)[0]


def test_line_search_refuses_an_ascent_direction():
    x = np.array([-1.2, 1.0])
    f, g = _rosenbrock(x)
    a, xn, fn, gn, trials = lbfgs.line_search(_rosenbrock, x, f, g, g)
    assert a == 0.0 and trials == 0 and fn == f


@pytest.mark.parametrize("n,seed", [(8, 0), (50, 1)])
def test_minimize_quadratic_closed_form(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = A @ A.T + 0.5 * np.eye(n)
    b = rng.standard_normal(n)

    def fg(x):
        return 0.5 * float(x @ A @ x) - float(b @ x), A @ x - b

    # (the Armijo test on f stalls a little above 1e-8 rms here: FP64 rounding of f)
    x, f, g, info = lbfgs.minimize(fg, np.zeros(n), tol=1e-7, max_iter=2000)
    assert info["rms_grad"] < 1e-7
    xs = np.linalg.solve(A, b)
    # x - x* = A^-1 g exactly, so |x - x*| <= |g| / lambda_min
    lam_min = float(np.linalg.eigvalsh(A)[0])
    assert np.linalg.norm(x - xs) <= np.linalg.norm(A @ x - b) / lam_min * (1 + 1e-6) + 1e-14
    assert np.linalg.norm(x - xs) < 1e-6
    # f - f* = (x - x*)^T A (x - x*) / 2
    e = x - xs
    assert abs((f - (-0.5 * float(b @ xs))) - 0.5 * float(e @ A @ e)) < 1e-12


def test_minimize_rosenbrock():
    x, f, g, info = lbfgs.minimize(_rosenbrock, np.array([-1.2, 1.0]), tol=1e-10, max_iter=500)
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-8)
    assert f < 1e-16
