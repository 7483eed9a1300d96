"""The paper's initial-state generator (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sec. II.B of
arXiv:2109.11001: chains are placed as freely rotating (FR) chains whose
fixed bending angle theta* gives the Kuhn length l_K(kappa) of Eq. 12, and a
state is redrawn when the fit of Eq. 14 to its <R^2(n)> (N/4 <= n <= N/2)
misses Eq. 12 by more than 2%.  Eq. 13 is garbled in the text (it gives
cos theta* > 1); the FR relation l_K / l0 = (1 + c) / (1 - c) is inverted
instead: cos theta* = (l_K/l0 - 1) / (l_K/l0 + 1).

Random numbers: Philox4x32-10 with key = seed and counter
(bond index i, chain, attempt, 5); u = (w + 1/2) 2^-32.  Monomer 0 of a chain
is uniform in the box, bond 1 points uniformly on the sphere, and every
further bond keeps angle theta* with the previous one at a uniform azimuth
about it.  Scalar IEEE arithmetic and libm (math) in a fixed order.
"""
from __future__ import annotations

import math

import numpy as np

from . import kuhn, philox4x32_10, schedule

L0 = 0.960897
TWO_PI = 6.283185307179586
U32 = 2.3283064365386963e-10          # 2^-32


def _u(w):
    return (float(w) + 0.5) * U32


def _basis(b):
    a = (0.0, 0.0, 1.0) if abs(b[2]) < 0.9 else (1.0, 0.0, 0.0)
    cx = b[1] * a[2] - b[2] * a[1]
    cy = b[2] * a[0] - b[0] * a[2]
    cz = b[0] * a[1] - b[1] * a[0]
    n = math.sqrt((cx * cx + cy * cy) + cz * cz)
    e1 = (cx / n, cy / n, cz / n)
    e2 = (b[1] * e1[2] - b[2] * e1[1], b[2] * e1[0] - b[0] * e1[2], b[0] * e1[1] - b[1] * e1[0])
    return e1, e2


def fr_state(n_chains, N, box, cos_t, seed, attempt, l0=L0):
    """One draw of FR chains, (3, n_chains N) unwrapped positions, chain-major."""
    s_t = math.sqrt(1.0 - cos_t * cos_t)
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    x = np.zeros((3, n_chains * N))
    for c in range(n_chains):
        p = [0.0, 0.0, 0.0]
        b = (0.0, 0.0, 1.0)
        for i in range(N):
            w = philox4x32_10([i, c, attempt, 5], key)
            if i == 0:
                p = [box * _u(w[0]), box * _u(w[1]), box * _u(w[2])]
            else:
                if i == 1:
                    ct = 2.0 * _u(w[0]) - 1.0
                    st = math.sqrt(max(0.0, 1.0 - ct * ct))
                    ph = TWO_PI * _u(w[1])
                    nb = (st * math.cos(ph), st * math.sin(ph), ct)
                else:
                    ph = TWO_PI * _u(w[0])
                    e1, e2 = _basis(b)
                    cp, sp = math.cos(ph), math.sin(ph)
                    nb = tuple(cos_t * b[k] + s_t * (cp * e1[k] + sp * e2[k]) for k in range(3))
                n = math.sqrt((nb[0] * nb[0] + nb[1] * nb[1]) + nb[2] * nb[2])
                b = (nb[0] / n, nb[1] / n, nb[2] / n)
                p = [p[k] + l0 * b[k] for k in range(3)]
            x[:, c * N + i] = p
    return x


def r2n_range(x, n_chains, N, lo, hi):
    """<R^2(n)> for lo <= n <= hi (definition: mean over chains and positions)."""
    out = np.zeros(N)
    X = x.reshape(3, n_chains, N)
    for n in range(lo, hi + 1):
        d = X[:, :, n:] - X[:, :, :-n]
        out[n] = float((d * d).sum(axis=0).mean())
    return out


def generate(n_chains, N, box, kappa, seed, l0=L0, max_attempts=100, tol=0.02):
    """(x, l_K fitted, attempts used) of the first state within tol of Eq. 12."""
    r = schedule.lk_over_l0(kappa)
    cos_t = (r - 1.0) / (r + 1.0)
    lo, hi = max(N // 4, 1), N // 2
    for a in range(max_attempts):
        x = fr_state(n_chains, N, box, cos_t, seed, a, l0)
        lk = kuhn.fit_lk(r2n_range(x, n_chains, N, lo, hi), l0, lo, hi)
        if abs(lk / (r * l0) - 1.0) <= tol:
            return x, lk, a + 1
    raise RuntimeError("no state within tolerance")
