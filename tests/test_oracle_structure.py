"""Pins of the structure-factor and pair-distribution oracles (App. A observables)."""
import numpy as np
import pytest

from oracle import structure as SF


def test_structure_factor_of_an_ideal_gas_averages_to_one():
    rng = np.random.default_rng(1)
    L, M = 10.0, 4000
    x = rng.uniform(0, L, (3, M))
    hkl = np.array([(h, k, l) for h in range(1, 11) for k in range(-5, 6) for l in range(-5, 6)])
    S = SF.structure_factor(x, L, hkl)                     # 1210 values, each exponential with mean 1
    assert S.mean() == pytest.approx(1.0, abs=0.12)        # 4 standard errors


def test_structure_factor_of_a_cubic_lattice():
    # simple cubic lattice, spacing a = L/n: Bragg peaks S = M at multiples of n, zero elsewhere
    n, L = 6, 9.0
    g = (np.arange(n) + 0.5) * (L / n)
    x = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1)
    M = x.shape[1]
    S = SF.structure_factor(x, L, [(n, 0, 0), (0, n, n), (1, 0, 0), (2, 3, 1)])
    assert S[:2] == pytest.approx([M, M], rel=1e-12)
    assert np.all(S[2:] < 1e-20 * M)


def test_structure_factor_ignores_box_images():
    rng = np.random.default_rng(2)
    L = 7.0
    x = rng.uniform(0, L, (3, 300))
    shifted = x + L * rng.integers(-3, 4, x.shape)
    hkl = [(1, 2, 3), (4, 0, 1)]
    assert SF.structure_factor(shifted, L, hkl) == pytest.approx(SF.structure_factor(x, L, hkl), rel=1e-9)


def test_pair_distribution_of_an_ideal_gas_is_one():
    rng = np.random.default_rng(3)
    L, M = 8.0, 1500
    x = rng.uniform(0, L, (3, M))
    g = SF.pair_distribution(x, L, 3.0, 6)
    assert g[2:] == pytest.approx(np.ones(4), abs=0.05)
