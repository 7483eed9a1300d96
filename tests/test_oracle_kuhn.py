"""Pins of the Kuhn-length fit (Eq. 14) and the library's host version of it."""
import numpy as np
import pytest

from oracle import kuhn

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("lk", [1.3, 3.7, 12.0])
def test_fit_recovers_the_kuhn_length_of_exact_wlc_data(lk):
    N = 400
    n = np.arange(N, dtype=np.float64)
    r2n = np.zeros(N)
    r2n[1:] = n[1:] * kuhn.L0 * kuhn.wlc(n[1:], lk)
    assert kuhn.fit_lk(r2n) == pytest.approx(lk, rel=1e-7)


def test_wlc_limits():
    # short chains are rods (<R^2> = n^2 l0^2), long ones random walks (<R^2> = n l0 l_K)
    lk, l0 = 5.0, kuhn.L0
    assert kuhn.wlc(1e-4, lk) * 1e-4 * l0 == pytest.approx((1e-4 * l0) ** 2, rel=1e-3)
    assert kuhn.wlc(1e7, lk) == pytest.approx(lk, rel=1e-5)


@pytest.mark.parametrize("kappa", [1.0, 3.0])
def test_fit_of_freely_rotating_chains(kappa):
    # FR chain (<cos> = c): <R^2(n)> = n b^2 [(1+c)/(1-c) - 2c(1-c^n)/(n(1-c)^2)] tends
    # to n b^2 (1+c)/(1-c): at n >> 1/(1-c) the WLC fit gives l_K = b^2 (1+c)/((1-c) l0)
    c = 1.0 / np.tanh(kappa) - 1.0 / kappa
    b = kuhn.L0
    N = 4000
    n = np.arange(N, dtype=np.float64)
    r2n = np.zeros(N)
    r2n[1:] = n[1:] * b * b * ((1 + c) / (1 - c) - 2 * c * (1 - c ** n[1:]) / (n[1:] * (1 - c) ** 2))
    want = b * b * (1 + c) / ((1 - c) * kuhn.L0)
    assert kuhn.fit_lk(r2n) == pytest.approx(want, rel=2e-3)


def test_library_fit_matches_the_oracle():
    kg = pytest.importorskip("paper_2109_11001_gb300")
    rng = np.random.default_rng(4)
    for N, lk in ((100, 2.0), (800, 6.5)):
        n = np.arange(N, dtype=np.float64)
        r2n = np.zeros(N)
        r2n[1:] = n[1:] * kuhn.L0 * kuhn.wlc(n[1:], lk) * (1 + 0.01 * rng.standard_normal(N - 1))
        assert kg.kg_fit_lk(r2n) == pytest.approx(kuhn.fit_lk(r2n), rel=1e-7)
        assert kg.kg_fit_lk(r2n, n_lo=5, n_hi=N - 1) == pytest.approx(kuhn.fit_lk(r2n, n_lo=5, n_hi=N - 1),
                                                                       rel=1e-7)


def test_fr_generator_geometry_and_acceptance():
    from oracle import frgen, schedule
    kappa, N, nch = 2.0, 40, 30
    r = schedule.lk_over_l0(kappa)
    c = (r - 1) / (r + 1)
    x, lk, att = frgen.generate(nch, N, 12.0, kappa, 99)
    X = x.reshape(3, nch, N)
    b = X[:, :, 1:] - X[:, :, :-1]
    assert np.sqrt((b * b).sum(axis=0)) == pytest.approx(frgen.L0, rel=1e-12)   # every bond l0
    bh = b / np.sqrt((b * b).sum(axis=0))
    cos = (bh[:, :, 1:] * bh[:, :, :-1]).sum(axis=0)
    assert cos == pytest.approx(c, abs=1e-12)                                     # fixed angle theta*
    assert abs(lk / (r * frgen.L0) - 1) <= 0.02 and att >= 1
    assert np.all((X[:, :, 0] >= 0) & (X[:, :, 0] < 12.0))                        # first monomers in the box
    # theta* inverts the FR relation: (1 + c) / (1 - c) = l_K / l0 of Eq. 12
    assert (1 + c) / (1 - c) == pytest.approx(r, rel=1e-14)


@pytest.mark.parametrize("kappa,N,nch", [(0.0, 48, 40), (2.5, 80, 25)])
def test_library_fr_generator_matches_the_oracle(kappa, N, nch):
    kg = pytest.importorskip("paper_2109_11001_gb300")
    from oracle import frgen
    x, lk, att = kg.kg_generate_fr(nch, N, 15.0, kappa, 2109)
    xo, lko, atto = frgen.generate(nch, N, 15.0, kappa, 2109)
    assert att == atto
    assert np.abs(x - xo).max() < 1e-9
    assert lk == pytest.approx(lko, rel=1e-7)          # two minimisers on a flat minimum
