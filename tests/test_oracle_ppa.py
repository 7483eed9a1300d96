"""Pins of the primitive-path oracle (Everaers et al. 2004, cited in Sec. III)
and of Eq. 22, against results the mathematics fixes independently of the
oracle's code: the worm-like-chain double integral behind Eq. 22, the exact
minimiser of a free chain with fixed ends, and the force balance of two hooked
chains.
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

import kg_inputs as KI
from conftest import relaxed_melt
from oracle import ppa as P

K12 = 30.0
R0 = 1.5


def wlc_ratio_quadrature(x):
    """<R^2> / L_c^2 of a worm-like chain of contour L_c = 2 x l_p (x Kuhn
    segments of length 2 l_p), from its tangent correlation exp(-|s - t| / l_p):
    (2 / L_c^2) int_0^{L_c} int_0^s exp(-(s - t)) dt ds with l_p = 1, the inner
    integral done by quadrature too."""
    Lc = 2.0 * x
    inner = lambda s: quad(lambda t: np.exp(-(s - t)), 0.0, s, epsabs=1e-14, epsrel=1e-13)[0]
    outer = quad(inner, 0.0, Lc, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    return 2.0 * outer / (Lc * Lc)


@pytest.mark.parametrize("x", [5e-4, 0.05, 0.5, 2.0, 10.0, 60.0])
def test_eq22_is_the_wlc_end_to_end_ratio(x):
    """Eq. 22's left-hand side equals <R^2>/L^2 of a primitive path that is a
    worm-like chain of N_eK Kuhn segments (Svaneborg and Everaers' reading)."""
    assert P.eq22_lhs(x) == pytest.approx(wlc_ratio_quadrature(x), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("x", [0.01, 0.3, 1.0, 7.5, 40.0, 300.0])
def test_eq22_inversion_round_trip(x):
    y = wlc_ratio_quadrature(x) if x <= 60 else (1.0 / x - (1.0 - np.exp(-2 * x)) / (2 * x * x))
    assert P.n_ek_from_ratio(np.sqrt(y)) == pytest.approx(x, rel=1e-7)


def test_eq22_limits_and_monotonicity():
    # strongly entangled paths: (L_pp/L)^2 -> 1/N_eK; unentangled: -> 1 - 2 N_eK / 3
    x = 1e4
    assert P.eq22_lhs(x) * x == pytest.approx(1.0 - 1.0 / (2.0 * x), rel=1e-12)
    assert P.eq22_lhs(1e-6) == pytest.approx(1.0 - 2e-6 / 3.0, rel=1e-13)
    g = np.logspace(-5, 4, 400)
    vals = np.array([P.eq22_lhs(t) for t in g])
    assert np.all(np.diff(vals) < 0)
    # continuity across the series / closed-form switch
    assert P.eq22_lhs(1e-3 * (1 - 1e-12)) == pytest.approx(P.eq22_lhs(1e-3), rel=1e-11)
    with pytest.raises(ValueError):
        P.n_ek_from_ratio(1.0)


def test_entanglement_length_scales_by_kuhn_ratio():
    N, lk = 400, 2.5
    lpp = 0.3 * (N - 1) * P.L0
    n_ek, n_e = P.entanglement_length(lpp, N, lk)
    assert P.eq22_lhs(n_ek) == pytest.approx(0.09, rel=1e-12)
    assert n_e == pytest.approx(n_ek * lk / P.L0, rel=1e-15)


def test_free_chain_straightens_with_equal_bonds():
    """One chain, ends fixed, no other chain: the FENE energy is a convex,
    increasing function of each bond length, so its minimum puts the monomers
    on the end-to-end segment at equal spacing, and L_pp = |R_ee|.  The walk
    crosses itself; intrachain excluded volume is off, so it must pass."""
    m = KI.random_walk_melt(1, 12, 0.02, 0.0, 5)
    x = P.minimise(m.x, 12, m.box, 4000, 0.01, 2.0, K12, R0)
    a, b = m.x[:, 0], m.x[:, -1]
    t = np.arange(12) / 11.0
    want = a[:, None] + t[None, :] * (b - a)[:, None]
    assert np.abs(x - want).max() < 1e-9
    assert P.path_lengths(x, 12)[0] == pytest.approx(np.linalg.norm(b - a), rel=1e-9)
    assert np.array_equal(x[:, [0, 11]], m.x[:, [0, 11]])


def hook_balance(D=1.2, k=K12, R0=R0):
    """Height u of the two middle monomers of the hooked pair at rest: each
    middle is pulled towards its chain's line by two FENE bonds of length
    sqrt(D^2 + u^2) (force 2 k u / (1 - (D^2 + u^2) / R0^2) along y) and pushed
    back by the LJ 12-6 repulsion of the other middle at distance 2 u,
    48 r^-13 - 24 r^-7."""
    f = lambda u: 2 * k * u / (1 - (D * D + u * u) / (R0 * R0)) - (48 * (2 * u) ** -13 - 24 * (2 * u) ** -7)
    return brentq(f, 0.3, 2 ** (1 / 6) / 2 - 1e-12, xtol=1e-15)


def test_hooked_pair_force_balance():
    D = 1.2
    m = KI.hooked_pair(D=D)
    u = hook_balance(D)
    assert 2 * u < 2 ** (1 / 6)          # the middles touch
    assert np.hypot(D, u) > 2 ** (1 / 6)  # no other interchain pair does
    x = P.minimise(m.x, 3, m.box, 6000, 0.005, 2.0, K12, R0)
    c = 0.5 * m.box
    assert np.abs(x[:, 1] - np.array([c, c + u, c])).max() < 1e-9
    assert np.abs(x[:, 4] - np.array([c, c - u, c])).max() < 1e-9
    assert P.path_lengths(x, 3) == pytest.approx(2 * np.hypot(D, u), rel=1e-10)


def test_hooked_pair_needs_the_interchain_term():
    """Planted mistake: with the pair term dropped the chains pass through
    each other and both straighten (L_pp = 2 D), so the pin above would fail."""
    m = KI.hooked_pair()
    orig = P._interchain
    try:
        P._interchain = lambda x, N, L: (np.zeros(0, int), np.zeros(0, int), np.zeros((3, 0)), np.zeros(0))
        x = P.minimise(m.x, 3, m.box, 6000, 0.005, 2.0, K12, R0)
    finally:
        P._interchain = orig
    assert P.path_lengths(x, 3) == pytest.approx(2 * 1.2, rel=1e-9)
    assert abs(P.path_lengths(x, 3)[0] - 2 * np.hypot(1.2, hook_balance())) > 0.05


def test_melt_minimisation_invariants():
    """A generated melt: the energy falls, ends do not move, and every chain's
    path lies between its end-to-end distance and its starting contour."""
    m = relaxed_melt(24, 16, 1.0, 9)
    N, L = m.chain_len, m.box
    e0 = P.energy(m.x, N, L, K12, R0)
    l0 = P.path_lengths(m.x, N)
    x = P.minimise(m.x, N, L, 400, 0.002, 1.0, K12, R0)
    assert P.energy(x, N, L, K12, R0) < e0
    xs = x.reshape(3, 24, N)
    x0 = m.x.reshape(3, 24, N)
    assert np.array_equal(xs[:, :, [0, N - 1]], x0[:, :, [0, N - 1]])
    lpp = P.path_lengths(x, N)
    ree = np.linalg.norm(x0[:, :, -1] - x0[:, :, 0], axis=0)
    assert np.all(lpp < l0)
    assert np.all(lpp >= ree * (1 - 1e-12))


def test_forces_are_minus_energy_gradient():
    m = relaxed_melt(10, 8, 1.0, 3)
    N, L = m.chain_len, m.box
    x = P.minimise(m.x, N, L, 50, 0.002, 1.0, K12, R0)
    F = P.forces(x, N, L, K12, R0)
    rng = np.random.default_rng(1)
    h = 1e-6
    for s in rng.choice(m.M, 12, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, s] += h
            xm[a, s] -= h
            g = (P.energy(xp, N, L, K12, R0) - P.energy(xm, N, L, K12, R0)) / (2 * h)
            assert -g == pytest.approx(F[a, s], abs=1e-5 * max(1.0, abs(F[a, s])))
