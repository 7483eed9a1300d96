"""Oracle pins for the reductions the MD observables are built from: the
virial, the pressure and the two histograms.

* Virial: under the affine scaling x -> lambda x, L -> lambda L every pair and
  bond distance scales by lambda and every bending angle is unchanged, so the
  total potential energy U(lambda) satisfies dU/dlambda at lambda = 1 equal to
  the sum over central terms of r dU/dr, i.e. minus the virial
  W = sum r . F.  The oracle's W is checked against a central finite
  difference of its own energy (whose terms are pinned by closed forms
  elsewhere), at several stages n, in a dense box where bonds and pairs cross
  the boundary and in a large box where nothing does.  A copy of the oracle
  with the virial's sign flipped is compiled on the CPU and must fail the same
  check.
* Pressure: P = (2 E_kin + W) / (3 V); for a dilute Langevin gas of monomers
  (rho = 1e-3, so collisions shift P / rho by about B_2 rho ~ 2e-3) the time
  average of P / rho is the temperature, 1.
* Histograms: cos(theta) of chains with freely rotating bonds whose cos(theta)
  is drawn from exp(kappa cos theta) (inverse CDF, independent of the oracle)
  fill each bin with the probability integral of that density over the bin;
  angles and bond lengths placed just inside either edge of every bin land in
  that bin.
"""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import kg_inputs as KI
import oracle as O


def _potential(p, x):
    ob = O.observe(p, x, np.zeros_like(x), 0)
    return ob["e_pair"] + ob["e_bond"] + ob["e_angle"], ob["virial"]


def _scaled(p, lam):
    return O.params(p.n_chains, p.chain_len, p.box * lam, p.kappa, n_exp=p.n_exp, k_fene=p.k_fene,
                    fene_qmin=p.fene_qmin)


def _affine_derivative(energy, p, x, h=1e-5):
    """dU/dlambda at 1 by a fourth-order central difference."""
    f = {k: energy(_scaled(p, 1 + k * h), x * (1 + k * h)) for k in (-2, -1, 1, 2)}
    return (8 * (f[1] - f[-1]) - (f[2] - f[-2])) / (12 * h)


def _dense_melt(n_exp, kappa=1.5, seed=5):
    m = KI.random_walk_melt(16, 20, 0.85, kappa, seed)       # L = 7.2: bonds and pairs cross the box
    return m, O.params(m.n_chains, m.chain_len, m.box, kappa, n_exp=n_exp)


def _thermal(m, kappa=1.5):
    """40 soft (n = 2) Langevin steps from the generated melt: a thermal
    configuration with many pairs inside r_c."""
    x = m.x.copy()
    O.run(O.params(m.n_chains, m.chain_len, m.box, kappa, n_exp=2.0, dt=0.002), x, m.v.copy(), 0, 40)
    return x


def _isolated_chains(n_exp, kappa=2.0):
    """Three 12-monomer chains well inside a box of side 60: no bond or pair
    crosses the boundary and no chain meets another."""
    rng = np.random.default_rng(4)
    xs = []
    for c in range(3):
        pos = [np.array([15.0 + 15.0 * c, 30.0, 30.0])]
        d = np.array([1.0, 0.0, 0.0])
        for _ in range(11):
            d = d + 0.6 * rng.normal(size=3)
            d /= np.linalg.norm(d)
            pos.append(pos[-1] + 0.97 * d)
        xs.append(np.array(pos))
    x = np.ascontiguousarray(np.concatenate(xs).T)
    return x, O.params(3, 12, 60.0, kappa, n_exp=n_exp)


@pytest.mark.parametrize("n_exp", [2.0, 6.5, 12.0])
def test_virial_is_minus_the_affine_derivative_of_the_energy(n_exp):
    m, p = _dense_melt(n_exp)
    x = _thermal(m)
    U, W = _potential(p, x)
    dU = _affine_derivative(lambda q, y: _potential(q, y)[0], p, x)
    assert abs(W) > 1.0
    assert W == pytest.approx(-dU, rel=1e-7, abs=1e-7)
    # unwrapped positions outside [0, L) on both sides: the box is crossed
    assert (x < 0).any() and (x >= p.box).any()


@pytest.mark.parametrize("n_exp", [3.0, 12.0])
def test_virial_of_chains_that_cross_nothing(n_exp):
    x, p = _isolated_chains(n_exp)
    U, W = _potential(p, x)
    dU = _affine_derivative(lambda q, y: _potential(q, y)[0], p, x)
    assert abs(W) > 1e-3
    assert W == pytest.approx(-dU, rel=1e-7, abs=1e-9)


def test_virial_with_the_fene_continuation():
    # a stretched bond beyond r* = R0 sqrt(1 - q): the continued FENE branch
    m, p0 = _dense_melt(2.0, seed=8)
    p = O.params(p0.n_chains, p0.chain_len, p0.box, p0.kappa, n_exp=2.0, fene_qmin=0.05)
    x = m.x.copy()
    d = x[:, 1] - x[:, 0]
    x[:, 1:20] += (1.49 / np.linalg.norm(d) - 1.0) * d[:, None]    # bond 0-1 of chain 0 at 1.49 > r*
    U, W = _potential(p, x)
    dU = _affine_derivative(lambda q, y: _potential(q, y)[0], p, x)
    assert W == pytest.approx(-dU, rel=1e-7, abs=1e-7)


def _planted_oracle(tmp_path):
    """A copy of the oracle with the sign of every virial term flipped."""
    src = os.path.join(os.path.dirname(O.__file__), "kg_oracle.c")
    text = open(src).read()
    assert text.count("vir += -du * r;") == 2
    planted = tmp_path / "kg_oracle_planted.c"
    planted.write_text(text.replace("vir += -du * r;", "vir += du * r;"))
    shutil.copy(os.path.join(os.path.dirname(O.__file__), "kg_oracle.h"), tmp_path / "kg_oracle.h")
    so = tmp_path / "libplanted.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(planted),
                           "-o", str(so), "-lm"])
    lib = C.CDLL(str(so))
    lib.orc_observe.restype = C.c_int
    lib.orc_observe.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
    return lib


def test_planted_virial_sign_flip_fails_the_affine_check(tmp_path):
    lib = _planted_oracle(tmp_path)

    def planted(p, x):
        out = np.zeros(7)
        x = np.ascontiguousarray(x)
        u = np.zeros_like(x)
        assert lib.orc_observe(C.byref(p), x.ctypes.data, u.ctypes.data, 0, out.ctypes.data) == 0
        return out[0] + out[1] + out[2], out[4]

    m, p = _dense_melt(12.0)
    x = _thermal(m)
    U, W = planted(p, x)
    dU = _affine_derivative(lambda q, y: planted(q, y)[0], p, x)
    assert abs(W + dU) > 0.5 * abs(dU)             # the planted oracle fails the pin
    assert W == pytest.approx(dU, rel=1e-7)        # (it is the exact negative)


def test_pressure_of_a_dilute_gas_is_rho_T():
    n_side, a = 12, 10.0                           # rho = 1e-3; Langevin at T = 1
    M, L = n_side ** 3, n_side * a
    g = np.arange(n_side) * a + 0.5 * a
    x = np.ascontiguousarray(np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1))
    u = np.zeros((3, M))
    p = O.params(M, 1, L, 0.0, n_exp=12.0, gamma=1.0, T=1.0, dt=0.01, seed=91)
    step = O.run(p, x, u, 0, 500)
    rho = M / L ** 3
    ratios = []
    for _ in range(24):
        step = O.run(p, x, u, step, 40)
        ob = O.observe(p, x, u, step)
        ratios.append(ob["pressure"] / rho)
    r = np.array(ratios)
    err = r.std(ddof=1) / math.sqrt(len(r))
    assert abs(r.mean() - 1.0) < 4 * err + 0.005, (r.mean(), err)


def _chains_from_angles(cos_t, b=0.97, rng=None):
    """Chains of 3 monomers whose single angle has the given cosines: bond 1
    along a random axis, bond 2 at the angle theta from it (theta between
    bond vectors, 0 = straight), random azimuth."""
    n = len(cos_t)
    rng = rng or np.random.default_rng(0)
    x = np.zeros((3, 3 * n))
    for k, c in enumerate(cos_t):
        e1 = rng.normal(size=3)
        e1 /= np.linalg.norm(e1)
        t = np.cross(e1, [0.3, 0.5, 0.8])
        t /= np.linalg.norm(t)
        w = np.cross(e1, t)
        phi = rng.uniform(0, 2 * np.pi)
        s = math.sqrt(max(0.0, 1 - c * c))
        e2 = c * e1 + s * (math.cos(phi) * t + math.sin(phi) * w)
        r0 = np.array([50.0, 50.0, 50.0])
        x[:, 3 * k] = r0
        x[:, 3 * k + 1] = r0 + b * e1
        x[:, 3 * k + 2] = r0 + b * e1 + b * e2
    return x


@pytest.mark.parametrize("kappa", [0.5, 2.5])
def test_cos_histogram_of_exp_kappa_cos_angles(kappa):
    # cos(theta) ~ exp(kappa c) on [-1, 1] by inverse CDF:
    #   c = log(exp(-kappa) + u (exp(kappa) - exp(-kappa))) / kappa
    rng = np.random.default_rng(17)
    n, nb = 40000, 16
    u = rng.uniform(size=n)
    c = np.log(np.exp(-kappa) + u * (np.exp(kappa) - np.exp(-kappa))) / kappa
    x = np.ascontiguousarray(_chains_from_angles(c, rng=rng))
    p = O.params(n, 3, 100.0, kappa)
    bh, ch = O.hist(p, x, nb)
    edges = np.linspace(-1, 1, nb + 1)
    prob = (np.exp(kappa * edges[1:]) - np.exp(kappa * edges[:-1])) / (np.exp(kappa) - np.exp(-kappa))
    want = n * prob
    chi2 = float(((ch - want) ** 2 / want).sum())
    # 15 degrees of freedom: P(chi2 > 45) ~ 1e-4
    assert chi2 < 45.0, (chi2, ch, want)
    assert ch.sum() == n and bh.sum() == 2 * n


def test_cos_histogram_edges():
    nb = 10
    w = 2.0 / nb
    vals, want = [], []
    for k in range(nb):
        lo = -1.0 + k * w
        for c, b in ((lo + 1e-6, k), (lo + 0.5 * w, k), (lo + w - 1e-6, k)):
            vals.append(c)
            want.append(b)
    x = np.ascontiguousarray(_chains_from_angles(np.array(vals)))
    p = O.params(len(vals), 3, 100.0, 1.0)
    _, ch = O.hist(p, x, nb)
    expect = np.bincount(np.array(want), minlength=nb)
    assert np.array_equal(ch, expect), (ch, expect)
    # the two end points fall in the end bins
    x = np.ascontiguousarray(_chains_from_angles(np.array([-1.0, 1.0])))
    _, ch = O.hist(O.params(2, 3, 100.0, 1.0), x, nb)
    assert ch[0] == 1 and ch[-1] == 1


def test_bond_histogram_edges():
    nb, R0 = 12, 1.5
    w = R0 / nb
    lengths, want = [], []
    for k in range(nb):
        for r, b in ((k * w + 1e-7, k), ((k + 0.5) * w, k), ((k + 1) * w - 1e-7, k)):
            if r > 0:
                lengths.append(r)
                want.append(b)
    n = len(lengths)
    x = np.zeros((3, 2 * n))
    for k, r in enumerate(lengths):
        x[:, 2 * k] = [50.0, 50.0, 50.0]
        x[:, 2 * k + 1] = [50.0 + r, 50.0, 50.0]
    p = O.params(n, 2, 100.0, 0.0)
    bh, _ = O.hist(p, np.ascontiguousarray(x), nb)
    assert np.array_equal(bh, np.bincount(np.array(want), minlength=nb))
