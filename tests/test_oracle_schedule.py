"""Oracle pins for the softening schedule (Sec. II.B, Eqs. 11-20) against the
numbers the paper prints: k = 30 at n = 12, f_0 fixing 1e8 steps at kappa = 5.5,
1e7 steps for kappa <= 2.5 (Fig. 4), and the n = 2 stage lengths quoted in
App. B."""
import math

import pytest

import oracle as O
from oracle import schedule as S


def test_exponent_set(golden):
    assert list(S.XI) == [float(v) for v in golden["Xi"]]


def test_kuhn_length_flory_limit():
    # Eq. 12 Flory term -> 1 as kappa -> 0, and grows ~2 kappa for stiff chains
    assert S.lk_over_l0(0.0) == pytest.approx(1.0 + 0.77 * (math.tanh(0.16) + 1.0), rel=1e-12)
    assert S.lk_over_l0(1e-3) == pytest.approx(S.lk_over_l0(0.0), rel=1e-3)
    assert S.lk_over_l0(5.5) == pytest.approx(2 * 5.5 - 1 + 0.77 * (math.tanh(-0.03 * 30.25 - 0.41 * 5.5 + 0.16) + 1),
                                              rel=1e-3)


def test_f0_gives_1e8_steps_at_kappa_5p5(golden):
    # Sec. II.B: f_0 is the largest f meeting N_t <= 1e8 steps for N = 400 at kappa = 5.5
    steps = S.tau_fix(5.5, golden["N"], golden["f0"]) / golden["dt_final"]
    assert steps == pytest.approx(golden["Nt_max"], rel=1e-5)
    # scheme 2 at kappa = 5.5: the stages add up to tau_fix, i.e. 1e8 steps
    assert sum(S.stage_steps(5.5, golden["N"], golden["dt_final"])) == pytest.approx(golden["Nt_max"], rel=1e-6)


@pytest.mark.parametrize("kappa", [0.0, 1.0, 2.0, 2.5])
def test_scheme1_total_is_200N(kappa, golden):
    # Fig. 4: 1e7 steps for kappa <= 2.5 at N = 400, dt = 0.008
    steps = sum(S.stage_steps(kappa, golden["N"], golden["dt_final"]))
    assert steps == pytest.approx(golden["steps_kappa_le_2p5"], abs=12)
    d = S.stage_durations(kappa, golden["N"])
    assert d[-1] == pytest.approx(2 * S.tau_e(kappa))
    # tau_i proportional to Xi_i^(-1/2) over the first eleven stages
    for i in range(10):
        assert d[i] / d[i + 1] == pytest.approx((S.XI[i + 1] / S.XI[i]) ** 0.5, rel=1e-12)


def test_appendix_b_n2_stage_lengths(golden):
    # App. B: the n = 2 stages last between 1.15e4 and 3.56e4 tau for 2 <= kappa <= 4
    t2 = S.stage_durations(2.0, golden["N"])[0]
    t4 = S.stage_durations(4.0, golden["N"])[0]
    assert t2 == pytest.approx(golden["tau1_kappa2"], rel=0.005)
    assert t4 == pytest.approx(golden["tau1_kappa4"], rel=0.005)
    for k in (2.5, 3.0, 3.5):
        assert t2 <= S.stage_durations(k, golden["N"])[0] <= t4


def test_tau_eq_is_max_of_three():
    for k in (0.0, 2.0, 4.0, 5.5):
        te = S.tau_eq(k, 400)
        assert te == max(2 * S.tau_e(k), S.tau_fix(k, 400), 80000.0)
    # for N = 400, tau_12 >= tau_e in both schemes (Sec. II.B)
    for k in (0.0, 1.0, 2.5, 3.0, 4.0, 5.5):
        assert S.stage_durations(k, 400)[-1] >= S.tau_e(k)


def test_kn_table_monotone_and_positive(golden):
    ks = [O.kn(n, golden["R0"], golden["l0"]) for n in S.XI]
    assert all(k > 0 for k in ks)
    assert all(a < b for a, b in zip(ks, ks[1:]))
    assert ks[-1] == pytest.approx(golden["k_standard"], rel=1e-4)
