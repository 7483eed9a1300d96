"""Potential-softening schedule of the DBH + core-softening protocol (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain FP64 Python
restating Sec. II.B of arXiv:2109.11001: the exponent set (Eq. 11), the Kuhn
length estimate (Eq. 12), tau_fix (Eq. 16), tau_e (Eq. 17 in the paper's
approximated form), tau_eq (Eq. 18) and the two division schemes (Eqs. 19-20).
"""
from __future__ import annotations

import math

# Eq. 11: exponents n of U_MLJ^n, in the order they are used
XI = (2.0, 3.0, 4.0, 5.0, 5.75, 6.5, 7.0, 8.0, 9.0, 10.0, 11.0, 12.0)
# Eq. 15 fit of the swap success rate: a, b (d is not used by the schedule)
A_FIT = 1.6
B_FIT = 0.77
# Sec. II.B: prefactor f_0 that makes tau_fix(kappa = 5.5) = 1e8 steps at dt = 0.008
F0 = 46.3354
L0 = 0.960897


def lk_over_l0(kappa: float) -> float:
    """Eq. 12: Svaneborg et al. Kuhn length over l0 (Flory term + melt correction)."""
    k = float(kappa)
    if k < 1e-4:
        flory = 1.0 + 2.0 * k / 3.0          # limit of the Flory term as kappa -> 0
    else:
        flory = (2.0 * k + math.exp(-2.0 * k) - 1.0) / (1.0 - math.exp(-2.0 * k) * (2.0 * k + 1.0))
    return flory + 0.77 * (math.tanh(-0.03 * k * k - 0.41 * k + 0.16) + 1.0)


def tau_fix(kappa: float, N: int, f: float = F0) -> float:
    """Eq. 16: (f N / a) exp(b kappa), in tau_LJ."""
    return f * N / A_FIT * math.exp(B_FIT * kappa)


def ne_initial(kappa: float) -> float:
    """Sec. II.B initial entanglement-length estimate 77 exp(-kappa/1.1) + 9.4."""
    return 77.0 * math.exp(-kappa / 1.1) + 9.4


def tau_e(kappa: float) -> float:
    """Eq. 17 with the O(1) prefactor dropped: N_e^2 (l_K / l0) tau_LJ."""
    return ne_initial(kappa) ** 2 * lk_over_l0(kappa)


def tau_eq(kappa: float, N: int, f: float = F0) -> float:
    """Eq. 18: max[2 tau_e, tau_fix, 200 N tau]."""
    return max(2.0 * tau_e(kappa), tau_fix(kappa, N, f), 200.0 * N)


def stage_durations(kappa: float, N: int, f: float = F0) -> list[float]:
    """Durations tau_i (in tau_LJ) of the twelve stages n = XI[i].

    Scheme 1 (Eq. 19) for kappa <= 2.5, scheme 2 (Eq. 20) above.  READING: the
    paper states the boundary both as kappa <= 2.5 and kappa >= 2.5; the n = 2
    stage lengths it quotes in App. B (1.15e4 to 3.56e4 tau for 2 <= kappa <= 4)
    match scheme 1 at kappa = 2.5, so the boundary case takes scheme 1.
    """
    w = [x ** -0.5 for x in XI]
    if kappa <= 2.5:
        total = 200.0 * N - 2.0 * tau_e(kappa)
        s11 = sum(w[:11])
        return [wi / s11 * total for wi in w[:11]] + [2.0 * tau_e(kappa)]
    s12 = sum(w)
    return [wi / s12 * tau_fix(kappa, N, f) for wi in w]


def stage_steps(kappa: float, N: int, dt: float, f: float = F0) -> list[int]:
    """Steps per stage: tau_i / dt rounded half to even (READING: unspecified)."""
    return [int(round(t / dt)) for t in stage_durations(kappa, N, f)]
