import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU statistical test")


@pytest.fixture(scope="session")
def golden():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.json")) as f:
        return {k: v["value"] for k, v in json.load(f).items() if not k.startswith("_")}


# soft-to-WCA walk through the potential schedule: (n, steps, dt)
RELAX = [(2.0, 300, 0.0005), (2.0, 300, 0.001), (4.0, 300, 0.0015), (6.5, 300, 0.0025), (9.0, 300, 0.004),
         (12.0, 300, 0.005)]


def relaxed_melt(n_chains, chain_len, kappa, seed, rho=0.85):
    """A generated melt relaxed by the oracle's MD through RELAX (regularised
    FENE in the soft stages), as input for analyses that need a state without
    overlaps (primitive paths)."""
    import kg_inputs as KI
    import oracle as O
    m = KI.random_walk_melt(n_chains, chain_len, rho, kappa, seed)
    step = 0
    for n_exp, n, dt in RELAX:
        p = O.params(m.n_chains, m.chain_len, m.box, m.kappa, n_exp=n_exp, dt=dt, seed=seed, fene_qmin=0.01)
        step = O.run(p, m.x, m.v, step, n)
    return m
