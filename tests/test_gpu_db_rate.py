"""Double-bridging success rate against the paper's fit (Sec. II.B, Eq. 15,
Fig. 3): S(kappa, n) = 1.6 exp(-0.77 kappa - 0.35 n) per attempted move, the
moves attempted only where criteria (i) and (ii) admit one.  Melts of 50
chains x N = 400 at kappa = 1, 2, 3 in the stages n = 2, 4, 6.5, exact
Metropolis-Hastings acceptance; the fitted exponents of the same form must
fall in a loose band around the paper's (b = 0.77 +- 0.015, d = 0.35 +- 0.01
there; our melts are briefly relaxed, 20k monomers each, and our move set
also requires both removed bonds to be <= 1.3 sigma): b within 0.77 +- 0.2,
d within 0.35 +- 0.12, and every measured rate within a factor of 3 of Eq. 15.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_11001_gb300 as kg
    kg.load()
    return kg


def test_success_rate_follows_eq15(kg):
    import torch

    import bench
    table, fit = bench.measure_db_success(kg, torch, [1.0, 2.0, 3.0], [2.0, 4.0, 6.5], rounds=20)
    print("fit", fit)
    for t in table:
        print(t)
    assert sum(t["accepted"] for t in table) > 500
    assert abs(fit["b"] - 0.77) < 0.2, fit
    assert abs(fit["d"] - 0.35) < 0.12, fit
    for t in table:
        assert t["admissible"] > 500
        assert 1 / 3 < t["S"] / t["S_eq15"] < 3, t
