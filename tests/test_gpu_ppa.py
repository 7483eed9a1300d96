"""GPU primitive-path analysis (kg_primitive_path) against the closed forms
that pin the oracle and against the oracle itself on the same inputs.

Binary64 mode: both sides minimise in binary64 with the same update order and
differ only in the order of the force sums, so runs agree to ~1e-12 sigma.
Mixed mode: binary32 pair vectors (~1e-7 sigma) and pair forces (~1e-6
relative); the bars follow from those errors.  Lists and sums on the GPU are
deterministic run to run.
"""
import numpy as np
import pytest

import kg_inputs as KI
from conftest import RELAX, relaxed_melt
from oracle import ppa as P
from test_oracle_ppa import K12, hook_balance

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


def _ctx(kg, m, **kw):
    import torch
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=0, seed=3, **kw)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    kg.kg_load_config(ctx, 0, m.x, m.v)
    return ctx


FP64, MIXED = 0, 1
# (position bar, relative L_pp bar) of each mode after short runs
BARS = {FP64: (1e-11, 1e-12), MIXED: (1e-4, 1e-6)}


def _ppa(kg, m, n_iter, dt, gamma, skin=0.3, k=K12, precision=MIXED):
    ctx = _ctx(kg, m)
    try:
        x = np.zeros_like(m.x)
        lpp, res = kg.kg_primitive_path(ctx, 0, m.n_chains, n_iter, dt, gamma, skin, k, x, precision)
        return x, lpp, res["lpp_mean"], res["fmax"]
    finally:
        kg.kg_destroy(ctx)


@pytest.mark.parametrize("precision,tol,ftol", [(FP64, 1e-9, 1e-7), (MIXED, 1e-6, 1e-3)])
def test_hooked_pair_force_balance(kg, precision, tol, ftol):
    D = 1.2
    m = KI.hooked_pair(D=D)
    u = hook_balance(D)
    x, lpp, mean, fmax = _ppa(kg, m, 6000, 0.005, 2.0, precision=precision)
    c = 0.5 * m.box
    assert np.abs(x[:, 1] - np.array([c, c + u, c])).max() < tol
    assert np.abs(x[:, 4] - np.array([c, c - u, c])).max() < tol
    assert lpp == pytest.approx(2 * np.hypot(D, u), rel=tol)
    assert mean == pytest.approx(2 * np.hypot(D, u), rel=tol)
    assert fmax < ftol


# mixed: binary32 bond vectors (rounding ~6e-8 of a bond) set where the forces balance
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-9), (MIXED, 1e-6)])
def test_free_chain_straightens(kg, precision, tol):
    m = KI.random_walk_melt(1, 12, 0.02, 0.0, 5)
    x, lpp, _, _ = _ppa(kg, m, 4000, 0.01, 2.0, precision=precision)
    a, b = m.x[:, 0], m.x[:, -1]
    want = a[:, None] + (np.arange(12) / 11.0)[None, :] * (b - a)[:, None]
    assert np.abs(x - want).max() < tol
    assert lpp[0] == pytest.approx(np.linalg.norm(b - a), rel=tol)


@pytest.fixture(scope="module")
def melt():
    # 41 chains x 25 = 1025 monomers: several 128-thread blocks and a ragged tail
    return relaxed_melt(41, 25, 1.5, 17)


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n_iter", [0, 1, 60])
def test_matches_oracle_short(kg, melt, n_iter, precision):
    """60 iterations run two captured 25-iteration graphs and ten direct ones."""
    xtol, ltol = BARS[precision]
    x, lpp, mean, _ = _ppa(kg, melt, n_iter, 0.005, 1.0, precision=precision)
    xo = P.minimise(melt.x, melt.chain_len, melt.box, n_iter, 0.005, 1.0, K12, 1.5)
    print(precision, n_iter, "max |dx|", np.abs(x - xo).max())
    assert np.abs(x - xo).max() < xtol
    lo = P.path_lengths(xo, melt.chain_len)
    assert lpp == pytest.approx(lo, rel=ltol)
    assert mean == pytest.approx(lo.mean(), rel=ltol)


@pytest.mark.parametrize("precision,ltol", [(FP64, 1e-9), (MIXED, 1e-4)])
def test_matches_oracle_converged(kg, melt, precision, ltol):
    """A longer minimisation (10 tau): the primitive paths of both sides and
    the N_eK that Eq. 22 gives from them."""
    n_iter = 2000
    x, lpp, mean, fmax = _ppa(kg, melt, n_iter, 0.005, 1.0, precision=precision)
    xo = P.minimise(melt.x, melt.chain_len, melt.box, n_iter, 0.005, 1.0, K12, 1.5)
    lo = P.path_lengths(xo, melt.chain_len)
    print(precision, "max |dx|", np.abs(x - xo).max(), "max rel dLpp", np.abs(lpp / lo - 1).max(), "fmax", fmax)
    assert lpp == pytest.approx(lo, rel=ltol)
    n_ek, _ = kg.kg_entanglement_length(mean, melt.chain_len, 2.0)
    assert n_ek == pytest.approx(P.n_ek_from_ratio(lo.mean() / ((melt.chain_len - 1) * P.L0)), rel=10 * ltol)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_deterministic_and_state_untouched(kg, melt, precision):
    ctx = _ctx(kg, melt)
    try:
        x1 = np.zeros_like(melt.x)
        x2 = np.zeros_like(melt.x)
        _, r1 = kg.kg_primitive_path(ctx, 0, melt.n_chains, 300, 0.005, 1.0, 0.3, K12, x1, precision)
        _, r2 = kg.kg_primitive_path(ctx, 0, melt.n_chains, 300, 0.005, 1.0, 0.3, K12, x2, precision)
        assert r1 == r2 and r1["builds"] >= 1
        xs = np.zeros_like(melt.x)
        kg.kg_get_config(ctx, 0, xs, None)
    finally:
        kg.kg_destroy(ctx)
    assert np.array_equal(x1, x2)
    assert np.array_equal(xs, melt.x)


def test_default_spring_is_eq9_at_n12(kg, melt):
    a = _ppa(kg, melt, 40, 0.005, 1.0, k=0.0)
    b = _ppa(kg, melt, 40, 0.005, 1.0, k=kg.kg_kn(12.0, 1.5, 0.960897))
    assert np.array_equal(a[0], b[0])


def test_errors(kg):
    m = KI.hooked_pair(D=1.2)
    ctx = _ctx(kg, m)
    try:
        with pytest.raises(kg.KGError):          # 10 / (2^(1/6) + 3) < 3 cells a side
            kg.kg_primitive_path(ctx, 0, 2, 10, 0.005, 1.0, 3.0, K12)
        with pytest.raises(kg.KGError):
            kg.kg_primitive_path(ctx, 0, 2, 10, -0.005, 1.0, 0.3, K12)
        with pytest.raises(kg.KGError):
            kg.kg_primitive_path(ctx, 1, 2, 10, 0.005, 1.0, 0.3, K12)
        with pytest.raises(kg.KGError):
            kg.kg_primitive_path(ctx, 0, 2, 10, 0.005, 1.0, 0.3, K12, None, 7)
        # the context still works after the rejected calls
        kg.kg_primitive_path(ctx, 0, 2, 10, 0.005, 1.0, 0.3, K12)
    finally:
        kg.kg_destroy(ctx)
    m = KI.hooked_pair(D=1.55)                   # bonds longer than R0 = 1.5
    ctx = _ctx(kg, m, fene_qmin=0.01)
    try:
        with pytest.raises(kg.KGError) as e:
            kg.kg_primitive_path(ctx, 0, 2, 10, 0.005, 1.0, 0.3, K12)
        assert e.value.status == kg.KG_ERR_BOND_OVERSTRETCH
        kg.kg_step(ctx, 1)                       # not latched
    finally:
        kg.kg_destroy(ctx)


def test_full_size_properties(kg):
    """The 1.6M-monomer melt (1000 x 1600), relaxed on the GPU through the
    soft-to-WCA walk, then 200 PPA steps: the minimisation leaves every end
    in place, shortens every chain and stays between its end-to-end distance
    and its contour."""
    import torch
    m = KI.make(5)
    sched = [kg.stage(n, k, dt) for n, k, dt in RELAX]
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=1, seed=5, fene_qmin=0.01)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, sched)
        kg.kg_load_config(ctx, 0, m.x, m.v)
        kg.kg_step(ctx, sum(k for _, k, _ in RELAX))
        x0 = np.zeros_like(m.x)
        kg.kg_get_config(ctx, 0, x0, None)
        x = np.zeros_like(m.x)
        lpp, res = kg.kg_primitive_path(ctx, 0, m.n_chains, 200, 0.005, 1.0, 0.3, K12, x)
        mean, fmax = res["lpp_mean"], res["fmax"]
        # interchain neighbours within 2^(1/6) + 0.3 at rho = 0.85: a few to a few tens
        assert 2.0 < res["mean_neighbours"] < 64.0 and res["builds"] >= 1
    finally:
        kg.kg_destroy(ctx)
    N = m.chain_len
    xs, x0s = x.reshape(3, -1, N), x0.reshape(3, -1, N)
    assert np.array_equal(xs[:, :, [0, N - 1]], x0s[:, :, [0, N - 1]])
    contour0 = P.path_lengths(x0, N)
    ree = np.linalg.norm(x0s[:, :, -1] - x0s[:, :, 0], axis=0)
    assert np.all(lpp < contour0)
    assert np.all(lpp >= ree * (1 - 1e-12))
    assert np.allclose(lpp, P.path_lengths(x, N), rtol=1e-12)
    assert mean == pytest.approx(lpp.mean(), rel=1e-12)
    assert np.isfinite(fmax)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_second_melt_of_a_batch(kg, melt, precision):
    """The analysis of melt 1 in a two-melt context reads that melt's slots
    only: bit-identical to the same melt in a context of its own."""
    import torch
    other = KI.hooked_pair()
    p = kg.make_params([(other.n_chains, other.chain_len, other.box, other.kappa),
                        (melt.n_chains, melt.chain_len, melt.box, melt.kappa)], precision=0, seed=3)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_load_config(ctx, 0, other.x, other.v)
        kg.kg_load_config(ctx, 1, melt.x, melt.v)
        x = np.zeros_like(melt.x)
        lpp, _ = kg.kg_primitive_path(ctx, 1, melt.n_chains, 60, 0.005, 1.0, 0.3, K12, x, precision)
    finally:
        kg.kg_destroy(ctx)
    x1, lpp1, _, _ = _ppa(kg, melt, 60, 0.005, 1.0, precision=precision)
    assert np.array_equal(x, x1)
    assert np.array_equal(lpp, lpp1)


def test_entanglement_length_of_a_relaxed_melt(kg):
    """End to end: generated melt (250 x 200, kappa = 3.5), the soft-to-WCA
    walk and 1000 WCA steps on the GPU, primitive paths (10,000 steps), Eq. 22
    with Eq. 12's Kuhn length.  The paper's fit for equilibrated melts,
    N_e = 71.2 - 61.3 tanh(kappa / 1.631) = 11.55 at kappa = 3.5, bounds the
    result loosely: this melt is not DBH-equilibrated and its chains are
    short (about 17 N_e).  The 1.6M-monomer benchmark melt gives 11.3."""
    import math

    import torch
    from oracle import schedule as SC
    kappa = 3.5
    m = KI.random_walk_melt(250, 200, 0.85, kappa, 77)
    sched = [kg.stage(n, k, dt) for n, k, dt in RELAX] + [kg.stage(12.0, 10 ** 9, 0.01)]
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=1, seed=7, fene_qmin=0.01)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, sched)
        kg.kg_load_config(ctx, 0, m.x, m.v)
        kg.kg_step(ctx, sum(k for _, k, _ in RELAX) + 1000)
        lpp, res = kg.kg_primitive_path(ctx, 0, m.n_chains, 10000, 0.005, 1.0, 0.3)
    finally:
        kg.kg_destroy(ctx)
    lk = SC.lk_over_l0(kappa) * P.L0
    n_ek, n_e = kg.kg_entanglement_length(res["lpp_mean"], m.chain_len, lk)
    paper = 71.2 - 61.3 * math.tanh(kappa / 1.631)
    print("L_pp/L", res["lpp_mean"] / ((m.chain_len - 1) * P.L0), "N_eK", n_ek, "N_e", n_e, "paper", paper)
    assert 0.6 * paper < n_e < 1.4 * paper
