"""Static structure factor and pair distribution (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).  App. A of
arXiv:2109.11001 checks equilibration with S(q) (and g(r)).  Definitions, in
binary64 NumPy:

    S(q) = (1/M) |sum_j exp(i q . r_j)|^2,  q = 2 pi (h, k, l) / L

for integer (h, k, l) (the reciprocal lattice of the periodic box, on which
S(q) does not depend on how positions are unwrapped);

    g(r) in bins of width dr over [0, r_max): the number of ordered pairs
    i != j with minimum-image distance in the bin, divided by M rho 4 pi /3
    (r_hi^3 - r_lo^3), rho = M / L^3.
"""
from __future__ import annotations

import numpy as np


def structure_factor(x, L, hkl):
    """x: (3, M) positions; hkl: (nq, 3) integers -> S for each q."""
    x = np.asarray(x, dtype=np.float64)
    q = 2.0 * np.pi * np.asarray(hkl, dtype=np.float64) / L
    M = x.shape[1]
    out = np.empty(len(q))
    for a in range(len(q)):
        ph = q[a] @ x
        re, im = np.cos(ph).sum(), np.sin(ph).sum()
        out[a] = (re * re + im * im) / M
    return out


def pair_distribution(x, L, r_max, nbins):
    """g(r) by brute force over all pairs (small M only)."""
    x = np.asarray(x, dtype=np.float64)
    M = x.shape[1]
    counts = np.zeros(nbins)
    dr = r_max / nbins
    for i in range(M):
        d = x - x[:, i:i + 1]
        d -= L * np.rint(d / L)
        r = np.sqrt((d * d).sum(axis=0))
        r[i] = np.inf
        r = r[r < r_max]
        counts += np.bincount((r / dr).astype(int), minlength=nbins)[:nbins]
    edges = np.arange(nbins + 1) * dr
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    return counts / (M * (M / L ** 3) * shell)
