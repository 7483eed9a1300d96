"""Kuhn length from <R^2(n)> (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Eq. 14 of
arXiv:2109.11001 (Sec. II.B): the chain statistics are fitted by the
worm-like-chain form

    <R^2(n)> / (n l0) = l_K { 1 - l_K / (2 n l0) [1 - exp(-2 n l0 / l_K)] }

at intermediate n (the paper's example range N/4 <= n <= N/2), l_K the one
free parameter.  The paper does not state the fit's weighting; this takes the
unweighted least squares in <R^2(n)> / (n l0), minimised by SciPy's bounded
scalar minimiser (a library primitive).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize_scalar

L0 = 0.960897


def wlc(n, lk, l0=L0):
    """Right-hand side of Eq. 14: <R^2(n)> / (n l0) of a worm-like chain."""
    n = np.asarray(n, dtype=np.float64)
    a = 2.0 * n * l0 / lk
    return lk * (1.0 - (1.0 - np.exp(-a)) / a)


def fit_lk(r2n, l0=L0, n_lo=None, n_hi=None):
    """l_K minimising sum_n [r2n[n] / (n l0) - wlc(n, l_K)]^2 over n_lo..n_hi
    (default N/4 .. N/2, N = len(r2n)); r2n[n] is <R^2(n)>, r2n[0] unused."""
    r2n = np.asarray(r2n, dtype=np.float64)
    N = len(r2n)
    lo = N // 4 if n_lo is None else n_lo
    hi = N // 2 if n_hi is None else n_hi
    n = np.arange(max(lo, 1), hi + 1, dtype=np.float64)
    y = r2n[n.astype(int)] / (n * l0)
    res = minimize_scalar(lambda lk: float(((y - wlc(n, lk, l0)) ** 2).sum()),
                          bounds=(1e-3 * l0, 1e3 * l0 * max(hi, 1)), method="bounded",
                          options={"xatol": 1e-12 * l0, "maxiter": 2000})
    return float(res.x)
