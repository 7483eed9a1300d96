"""Primitive-path analysis and the entanglement length of Eq. 22 (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. III of arXiv:2109.11001 measures N_e with primitive-path analysis (PPA),
the method of Everaers et al. (Science 303, 823 (2004)), which the paper cites
but does not restate.  The reading implemented here is that method in its
common form:

* both end monomers of every chain stay fixed in space;
* the non-bonded interaction acts only between monomers of different chains
  (any periodic image); inside a chain it is off, between 1-2 bonded monomers
  too, so a bond keeps only its FENE part -1/2 k R0^2 ln(1 - r^2/R0^2)
  (Eq. 10 without the U_MLJ term);
* the bending energy (Eq. 4) is off;
* the non-bonded interaction is the n = 12 member of Eq. 5, truncated and
  shifted at r_c = 2^(1/6) (the final stage of the schedule);
* the energy is minimised by the MD integrator of the path at T = 0: Langevin
  velocity Verlet with zero noise, i.e. damped dynamics, from rest.

A chain's primitive-path length is the length of its minimised contour,
sum_i |r_{i+1} - r_i|; L_pp is the mean over chains.  Eq. 22 turns
(L_pp / L)^2, L = (N - 1) l0, into N_eK, the Kuhn segments per entanglement,
and N_e = N_eK l_K / l0.

Pair candidates come from SciPy's periodic KD-tree (a library neighbour
search); every distance that decides or enters a force is the binary64
minimum-image distance ((dx^2 + dy^2) + dz^2), dx = d - L rint(d / L).
Positions are (3, M) float64, chain-major slots s = c N + i.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq
from scipy.spatial import cKDTree

RC = 2.0 ** (1.0 / 6.0)
L0 = 0.960897


class Overstretch(RuntimeError):
    """A bond reached the FENE divergence r >= R0 (Eq. 10)."""


def _candidate_pairs(x, L):
    """Unordered pairs (i < j) whose wrapped positions lie within slightly more
    than r_c of each other (periodic KD-tree); the caller applies the exact test."""
    w = x.T - L * np.floor(x.T / L)
    w[w >= L] = 0.0
    tree = cKDTree(w, boxsize=L)
    return tree.query_pairs(RC * (1.0 + 1e-9) + 1e-12, output_type="ndarray")


def _interchain(x, N, L):
    """Interchain pairs with r^2 < r_c^2: index arrays i, j and d = min-image(x_j - x_i)."""
    P = _candidate_pairs(x, L)
    if len(P) == 0:
        e = np.zeros(0, dtype=np.int64)
        return e, e, np.zeros((3, 0)), np.zeros(0)
    i, j = P[:, 0].astype(np.int64), P[:, 1].astype(np.int64)
    keep = (i // N) != (j // N)
    i, j = i[keep], j[keep]
    d = x[:, j] - x[:, i]
    d = d - L * np.rint(d / L)
    r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
    m = r2 < RC * RC
    return i[m], j[m], d[:, m], r2[m]


def _bonds(x, N):
    """Bond vectors b_s = x_{s+1} - x_s (unwrapped) for every slot s that is not a chain's last."""
    M = x.shape[1]
    s = np.arange(M - 1)
    s = s[(s % N) != N - 1]
    return s, x[:, s + 1] - x[:, s]


def forces(x, N, L, k_fene, R0=1.5):
    """Conservative PPA force on every monomer (binary64)."""
    F = np.zeros_like(x)
    i, j, d, r2 = _interchain(x, N, L)
    if len(i):
        ir2 = 1.0 / r2
        ir6 = ir2 * ir2 * ir2
        g = (48.0 * ir6 * ir6 - 24.0 * ir6) * ir2        # -U'(r)/r of U = 4(r^-12 - r^-6) + 1
        for a in range(3):
            np.add.at(F[a], i, -g * d[a])
            np.add.at(F[a], j, g * d[a])
    s, b = _bonds(x, N)
    q = ((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]) / (R0 * R0)
    if np.any(q >= 1.0):
        raise Overstretch("bond at or beyond R0")
    gb = k_fene / (1.0 - q)                                  # FENE: -U'(r)/r
    for a in range(3):
        np.add.at(F[a], s, gb * b[a])
        np.add.at(F[a], s + 1, -gb * b[a])
    return F


def energy(x, N, L, k_fene, R0=1.5):
    """PPA potential energy: interchain WCA + FENE (no U_MLJ in the bonds, no bending)."""
    _, _, _, r2 = _interchain(x, N, L)
    ir6 = 1.0 / (r2 * r2 * r2)
    e = float((4.0 * (ir6 * ir6 - ir6) + 1.0).sum())
    _, b = _bonds(x, N)
    q = ((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]) / (R0 * R0)
    if np.any(q >= 1.0):
        raise Overstretch("bond at or beyond R0")
    return e + float((-0.5 * k_fene * R0 * R0 * np.log1p(-q)).sum())


def minimise(x, N, L, n_iter, dt, gamma, k_fene, R0=1.5):
    """n_iter steps of the T = 0 Langevin velocity Verlet from rest with both
    ends of every chain fixed; returns the final positions.  One step:
    v <- v + dt/2 F; x <- x + dt v; F <- F_c(x) - gamma v; v <- v + dt/2 F,
    with F = v = 0 on end monomers throughout."""
    x = np.array(x, dtype=np.float64, copy=True)
    M = x.shape[1]
    idx = np.arange(M) % N
    fixed = (idx == 0) | (idx == N - 1)
    v = np.zeros_like(x)
    F = forces(x, N, L, k_fene, R0)
    F[:, fixed] = 0.0
    for _ in range(n_iter):
        v = v + 0.5 * dt * F
        x = x + dt * v
        F = forces(x, N, L, k_fene, R0) - gamma * v
        F[:, fixed] = 0.0
        v = v + 0.5 * dt * F
    return x


def path_lengths(x, N):
    """Contour length of every chain, sum of |x_{i+1} - x_i| along it."""
    M = x.shape[1]
    xs = x.reshape(3, M // N, N)
    b = xs[:, :, 1:] - xs[:, :, :-1]
    return np.sqrt((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]).sum(axis=1)


def eq22_lhs(n_ek):
    """Left-hand side of Eq. 22, (2 x + exp(-2 x) - 1) / (2 x^2), x = N_eK; a
    series for small x avoids the cancellation of the closed form."""
    x = float(n_ek)
    if x < 1e-3:
        return 1.0 - 2.0 * x / 3.0 + x * x / 3.0 - 2.0 * x ** 3 / 15.0
    return (2.0 * x + np.expm1(-2.0 * x)) / (2.0 * x * x)


def n_ek_from_ratio(lpp_over_L):
    """N_eK solving Eq. 22 for (L_pp / L) in (0, 1); the left-hand side falls
    monotonically from 1 (x -> 0) to 0 (x -> infinity)."""
    y = float(lpp_over_L) ** 2
    if not 0.0 < y < 1.0:
        raise ValueError("L_pp / L must lie in (0, 1)")
    t = brentq(lambda t: eq22_lhs(np.exp(t)) - y, -40.0, 40.0, xtol=1e-14, rtol=1e-15, maxiter=500)
    return float(np.exp(t))


def entanglement_length(lpp_mean, N, l_k, l0=L0):
    """(N_eK, N_e) from the mean primitive-path length: Eq. 22 with L = (N - 1) l0,
    then N_e = N_eK l_K / l0."""
    n_ek = n_ek_from_ratio(lpp_mean / ((N - 1) * l0))
    return n_ek, n_ek * l_k / l0
