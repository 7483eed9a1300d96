"""Oracle pins for the MD side: neighbour lists, the Langevin integrator and the
observables.

Pins: the cell-list construction against the all-pairs definition; energy
conservation of the Gamma = 0 integrator with fluctuations scaling as dt^2;
the Langevin free-particle mean-squared displacement and equipartition
(closed forms of the Ornstein-Uhlenbeck process); <R^2(n)> of freely rotating
chains against its closed form.
"""
import math

import numpy as np
import pytest

import kg_inputs as KI
import oracle as O


def _melt(n_chains=12, N=20, rho=0.85, kappa=1.5, seed=11, n_exp=2.0, **kw):
    m = KI.random_walk_melt(n_chains, N, rho, kappa, seed)
    p = O.params(n_chains, N, m.box, kappa, n_exp=n_exp, **kw)
    return m, p


@pytest.mark.parametrize("rlist", [1.12246 + 0.3, 1.6, 2.5])
def test_nlist_cells_equal_all_pairs(rlist):
    m, p = _melt(n_chains=30, N=25)
    o1, n1 = O.nlist(p, m.x, rlist, use_cells=True)
    o2, n2 = O.nlist(p, m.x, rlist, use_cells=False)
    assert np.array_equal(o1, o2) and np.array_equal(n1, n2)
    # symmetric, no self pairs, no 1-2 bonded pairs
    N = p.chain_len
    pairs = {(i, int(j)) for i in range(m.M) for j in n1[o1[i]:o1[i + 1]]}
    assert all((j, i) in pairs for i, j in pairs)
    assert all(i != j and not (i // N == j // N and abs(i - j) == 1) for i, j in pairs)
    # every pair within rlist - 1e-9 is present (distance check done here, independently)
    X = m.x.T
    for i in range(0, m.M, 37):
        d = X - X[i]
        d -= m.box * np.rint(d / m.box)
        r = np.linalg.norm(d, axis=1)
        want = {j for j in np.nonzero(r < rlist - 1e-9)[0] if j != i and not (j // N == i // N and abs(j - i) == 1)}
        got = set(n1[o1[i]:o1[i + 1]].tolist())
        assert want <= got
        assert all(r[j] < rlist + 1e-9 for j in got)


def _energy_trace(p, x, u, nsteps):
    step = 0
    E = []
    for _ in range(nsteps):
        ob = O.observe(p, x, u, step)
        E.append(ob["e_pair"] + ob["e_bond"] + ob["e_angle"] + ob["e_kin"])
        step = O.run(p, x, u, step, 1)
    return np.array(E)


def test_nve_energy_fluctuation_scales_as_dt2():
    # Gamma = 0: velocity Verlet conserves a shadow energy; the true energy
    # fluctuates with amplitude proportional to dt^2.
    m, p = _melt(n_chains=4, N=10, n_exp=2.0, kappa=1.0)
    x0, u0 = m.x.copy(), m.v.copy()
    # relax with the thermostat first so the start is not violent
    O.run(p, x0, u0, 0, 200)
    res = {}
    for dt, n in ((0.004, 400), (0.002, 800)):
        q = O.params(p.n_chains, p.chain_len, p.box, p.kappa, n_exp=p.n_exp, gamma=0.0, dt=dt)
        E = _energy_trace(q, x0.copy(), u0.copy(), n)
        res[dt] = E
        # no drift beyond the fluctuation itself
        assert abs(E[-50:].mean() - E[:50].mean()) < 5 * E.std() + 1e-6
    ratio = res[0.004].std() / res[0.002].std()
    assert 3.0 < ratio < 5.3, ratio


def test_langevin_free_particles():
    # Dilute gas without bonds (N = 1): Ornstein-Uhlenbeck velocities, D = T/gamma.
    # Starting from u = 0, <dx^2> per dimension
    #   = (2T/g)[t - 2(1 - e^{-gt})/g + (1 - e^{-2gt})/(2g)].
    n_side, a = 15, 10.0                  # simple cubic lattice, spacing far beyond r_c
    M, L = n_side ** 3, n_side * a
    g = np.arange(n_side) * a + 0.5 * a
    x = np.ascontiguousarray(np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1))
    u = np.zeros((3, M))
    p = O.params(M, 1, L, 0.0, n_exp=12.0, gamma=1.0, T=1.0, dt=0.01, seed=77)
    x0 = x.copy()
    t = 5.0
    step = O.run(p, x, u, 0, int(round(t / p.dt)))
    msd = ((x - x0) ** 2).mean()
    g, T = 1.0, 1.0
    want = 2 * T / g * (t - 2 * (1 - math.exp(-g * t)) / g + (1 - math.exp(-2 * g * t)) / (2 * g))
    assert msd == pytest.approx(want, rel=0.06)
    # equipartition once the velocities have relaxed
    temps = []
    for _ in range(10):
        step = O.run(p, x, u, step, 50)
        temps.append(O.observe(p, x, u, step)["temperature"])
    assert np.mean(temps) == pytest.approx(1.0, abs=0.03)


def test_langevin_melt_temperature():
    m, p = _melt(n_chains=10, N=20, n_exp=3.0, kappa=1.5, seed=2)
    x, u = m.x.copy(), m.v.copy()
    step = O.run(p, x, u, 0, 300)
    temps = []
    for _ in range(20):
        step = O.run(p, x, u, step, 25)
        temps.append(O.observe(p, x, u, step)["temperature"])
    assert np.mean(temps) == pytest.approx(1.0, abs=0.06)


@pytest.mark.parametrize("kappa", [0.0, 1.5, 3.0])
def test_r2n_of_freely_rotating_chains(kappa):
    # generator without overlap rejection: independent angles with
    # <cos> = coth(kappa) - 1/kappa; <R^2(n)> = n b^2 [(1+c)/(1-c) - 2c(1-c^n)/(n(1-c)^2)]
    nch, N, b = 3000, 16, 0.97
    m = KI.random_walk_melt(nch, N, 0.05, kappa, seed=9, d_min=0.0)
    p = O.params(nch, N, m.box, kappa)
    r2 = O.r2n(p, m.x)
    c = 0.0 if kappa == 0 else 1 / math.tanh(kappa) - 1 / kappa
    for n in range(1, N):
        want = n * b * b * ((1 + c) / (1 - c) - 2 * c * (1 - c ** n) / (n * (1 - c) ** 2))
        assert r2[n] == pytest.approx(want, rel=0.03), n
    assert r2[1] == pytest.approx(b * b, rel=1e-12)


def test_histograms_count_every_bond_and_angle():
    m, p = _melt(n_chains=8, N=15)
    bh, ch = O.hist(p, m.x, 30)
    assert bh.sum() == p.n_chains * (p.chain_len - 1)
    assert ch.sum() == p.n_chains * (p.chain_len - 2)
    # all generated bonds are 0.97: a single bin
    assert bh.max() == bh.sum()


def test_pressure_and_temperature_definitions():
    m, p = _melt(n_chains=6, N=10)
    ob = O.observe(p, m.x, m.v, 0)
    V = p.box ** 3
    assert ob["temperature"] == pytest.approx(2 * ob["e_kin"] / (3 * m.M), rel=1e-12)
    assert ob["pressure"] == pytest.approx((2 * ob["e_kin"] + ob["virial"]) / (3 * V), rel=1e-12)
