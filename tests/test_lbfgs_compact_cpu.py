"""The compact form of the L-BFGS inverse Hessian (dsm_lbfgs_compact, the host
side of the native minimiser) against the inverse BFGS updates applied one pair
at a time from H0 = gamma I: H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T,
rho = 1 / (s.y).  Host code only: runs without a GPU."""
import numpy as np
import pytest

pytest.importorskip("torch")


@pytest.mark.parametrize("m,n,seed", [(1, 7, 0), (3, 20, 1), (10, 60, 2)])
def test_compact_equals_bfgs_updates(m, n, seed):
    from paper_2504_19941_gb300 import _lib
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    Hs = A @ A.T + n * np.eye(n)         # an SPD Hessian: y = Hs s gives s.y > 0
    S = rng.standard_normal((m, n))
    Y = S @ Hs
    g = rng.standard_normal(n)
    gamma = float(S[-1] @ Y[-1] / (Y[-1] @ Y[-1]))
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    cx, cs, cy = _lib.dsm_lbfgs_compact(S @ Y.T, Y @ Y.T, S @ g, Y @ g, gamma)
    d = cx * g + cs @ S + cy @ Y
    np.testing.assert_allclose(d, -H @ g, rtol=1e-10, atol=1e-12 * np.abs(H @ g).max())
