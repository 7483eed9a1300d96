"""Oracle pins for the interaction potentials (Sec. II.A, Eqs. 2-10).

Each pin checks the oracle against something other than its own formula: the
standard LJ form of Eq. 2, the position of the Mie minimum stated in Sec. II.A,
the k = 30 of the standard model, the force balance of Eq. 8, and finite
differences of the energies.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_cutoff_is_lj_minimum():
    assert O.rc() == pytest.approx(2.0 ** (1.0 / 6.0), rel=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 5.75, 6.5, 7, 8, 9, 10, 11, 12])
def test_mlj_vanishes_smoothly_at_cutoff(n):
    # Sec. II.A: the Mie minimum sits at 2^(1/6) for every n; truncating and
    # shifting there makes U and dU/dr continuous and zero at r_c.
    rc = O.rc()
    assert O.mlj_u(n, rc * (1 - 1e-7)) == pytest.approx(0.0, abs=1e-10)
    assert O.mlj_du(n, rc * (1 - 1e-7)) == pytest.approx(0.0, abs=1e-5)
    assert O.mlj_u(n, rc * 1.01) == 0.0 and O.mlj_du(n, rc * 1.01) == 0.0
    # purely repulsive below r_c
    for r in np.linspace(0.6, rc * 0.999, 25):
        assert O.mlj_u(n, r) > 0.0
        assert O.mlj_du(n, r) < 0.0


def test_n12_is_standard_wca():
    # Eq. 2 with r_c = 2^(1/6): the truncated and shifted 12-6 LJ potential
    rc = 2.0 ** (1.0 / 6.0)
    for r in np.linspace(0.7, 1.12, 40):
        lj = 4.0 * ((1 / r) ** 12 - (1 / r) ** 6 - (1 / rc) ** 12 + (1 / rc) ** 6)
        assert O.mlj_u(12, r) == pytest.approx(lj, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("n", [2, 3, 5.75, 6.5, 9, 12])
def test_mlj_force_finite_difference(n):
    for r in np.linspace(0.65, 1.1, 17):
        h = 1e-6
        fd = (O.mlj_u(n, r + h) - O.mlj_u(n, r - h)) / (2 * h)
        assert O.mlj_du(n, r) == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_mlj_softens_with_decreasing_n():
    # Fig. 2(a): the core softens as n decreases (m = 6 fixed)
    for r in (0.6, 0.8, 0.95, 1.05):
        vals = [O.mlj_u(n, r) for n in (2, 3, 4, 5, 5.75, 6.5, 7, 8, 9, 10, 11, 12)]
        assert all(a < b for a, b in zip(vals, vals[1:]))


def test_k12_is_standard(golden):
    assert O.kn(12, golden["R0"], golden["l0"]) == pytest.approx(golden["k_standard"], rel=1e-4)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 5.75, 6.5, 7, 8, 9, 10, 11, 12])
def test_bond_minimum_at_l0(n, golden):
    # Eq. 8: d/dr [U_MLJ^n + FENE(k_n)] = 0 at r = l0 (finite difference of the energies)
    l0, R0 = golden["l0"], golden["R0"]
    k = O.kn(n, R0, l0)
    U = lambda r: O.mlj_u(n, r) + O.fene_u(k, R0, r)
    h = 1e-6
    assert (U(l0 + h) - U(l0 - h)) / (2 * h) == pytest.approx(0.0, abs=1e-6)
    assert U(l0 + 0.01) > U(l0) and U(l0 - 0.01) > U(l0)
    assert k > 0


def test_fene_finite_difference():
    for r in np.linspace(0.5, 1.45, 12):
        h = 1e-7
        fd = (O.fene_u(30, 1.5, r + h) - O.fene_u(30, 1.5, r - h)) / (2 * h)
        assert O.fene_du(30, 1.5, r) == pytest.approx(fd, rel=1e-6)


def _small_melt(kappa=1.5, n_exp=3.0, n_chains=6, N=7, L=4.2, seed=3):
    import kg_inputs as KI
    m = KI.random_walk_melt(n_chains, N, n_chains * N / L ** 3, kappa, seed)
    p = O.params(n_chains, N, m.box, kappa, n_exp=n_exp)
    return m, p


def _energy(p, x):
    _, e = O.forces(p, x)
    return e[0] + e[1] + e[2]


@pytest.mark.parametrize("n_exp,kappa", [(2.0, 1.5), (5.75, 0.0), (12.0, 3.0)])
def test_total_force_is_minus_energy_gradient(n_exp, kappa):
    m, p = _small_melt(kappa=kappa, n_exp=n_exp)
    F, _ = O.forces(p, m.x)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(30):
        k, s = rng.integers(3), rng.integers(m.M)
        xp, xm = m.x.copy(), m.x.copy()
        xp[k, s] += h
        xm[k, s] -= h
        fd = -(_energy(p, xp) - _energy(p, xm)) / (2 * h)
        assert F[k, s] == pytest.approx(fd, rel=1e-5, abs=1e-5)
    # Newton's third law: every term is internal
    assert np.abs(F.sum(axis=1)).max() < 1e-9 * max(1.0, np.abs(F).max())


def test_angle_term():
    # straight chain: zero bending energy and force; kappa = 0: no bending energy
    N = 5
    x = np.zeros((3, N))
    x[0] = np.arange(N) * 0.97 + 1.0
    x[1] = 1.0
    x[2] = 1.0
    p = O.params(1, N, 20.0, 2.0, n_exp=12.0)
    F, e = O.forces(p, x)
    assert e[2] == pytest.approx(0.0, abs=1e-14)
    # only bonds act, along x
    assert np.abs(F[1:]).max() < 1e-12
    # a right angle costs kappa * (1 - 0)
    x2 = np.array([[0.0, 0.97, 0.97], [0.0, 0.0, 0.97], [0.0, 0.0, 0.0]]) + 5.0
    p2 = O.params(1, 3, 20.0, 2.0, n_exp=12.0)
    _, e2 = O.forces(p2, x2)
    assert e2[2] == pytest.approx(2.0, rel=1e-12)
    p3 = O.params(1, 3, 20.0, 0.0, n_exp=12.0)
    _, e3 = O.forces(p3, x2)
    assert e3[2] == 0.0


def test_overstretched_bond_is_an_error():
    x = np.array([[1.0, 2.6], [1.0, 1.0], [1.0, 1.0]])
    p = O.params(1, 2, 20.0, 0.0, n_exp=2.0)
    with pytest.raises(O.OracleError):
        O.forces(p, x)


@pytest.mark.parametrize("qmin", [0.01, 0.1])
def test_regularised_fene(qmin):
    # equals Eq. 3 below r* = R0 sqrt(1 - qmin); value and slope continuous at r*;
    # harmonic beyond (second derivative k/qmin in r^2); finite past R0
    k, R0 = 2.25, 1.5
    rs = R0 * (1 - qmin) ** 0.5
    for r in np.linspace(0.5, rs * 0.999, 9):
        assert O.fene_reg_u(k, R0, qmin, r) == O.fene_u(k, R0, r)
        assert O.fene_reg_du(k, R0, qmin, r) == O.fene_du(k, R0, r)
    e = 1e-10
    assert O.fene_reg_u(k, R0, qmin, rs + e) == pytest.approx(O.fene_u(k, R0, rs - e), rel=1e-6)
    assert O.fene_reg_du(k, R0, qmin, rs + e) == pytest.approx(O.fene_du(k, R0, rs - e), rel=1e-5)
    for r in (rs + 0.01, R0, 1.2 * R0):
        h = 1e-6
        fd = (O.fene_reg_u(k, R0, qmin, r + h) - O.fene_reg_u(k, R0, qmin, r - h)) / (2 * h)
        assert O.fene_reg_du(k, R0, qmin, r) == pytest.approx(fd, rel=1e-6)
        assert O.fene_reg_du(k, R0, qmin, r) == pytest.approx(k * r / qmin, rel=1e-12)
    assert O.fene_reg_u(k, R0, 0.0, 1.2) == O.fene_u(k, R0, 1.2)


def test_regularised_bond_is_finite_past_R0():
    x = np.array([[1.0, 2.6], [1.0, 1.0], [1.0, 1.0]])       # bond 1.6 > R0
    p = O.params(1, 2, 20.0, 0.0, n_exp=2.0, fene_qmin=0.01)
    F, e = O.forces(p, x)
    assert np.isfinite(F).all() and F[0, 0] > 0               # pulled back together
