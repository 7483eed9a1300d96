"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Bars: Verlet lists and double-bridging topology bit-exact; forces <= 1e-5
relative (binary64 path: 1e-10); positions after 10 steps <= 1e-4 sigma.
The force bar is norm-wise per monomer against the larger of its own force
and the melt's rms force, because a single net force can cancel to near zero.
"""
import contextlib

import numpy as np
import pytest

import kg_inputs as KI
import oracle as O
from oracle import structure as SF

pytestmark = pytest.mark.gpu

RL = 2.0 ** (1 / 6) + 0.3


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


@contextlib.contextmanager
def context(kg, melts, precision, seed=11, schedule=None, flags=0, **kw):
    import torch
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa) for m in melts], precision=precision,
                       seed=seed, flags=flags, **kw)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        if schedule is not None:
            kg.kg_set_potential_schedule(ctx, schedule)
        for i, m in enumerate(melts):
            kg.kg_load_config(ctx, i, m.x, m.v)
        yield ctx
    finally:
        kg.kg_destroy(ctx)


def oparams(m, n_exp, seed=11, stream=0, dt=0.01, **kw):
    return O.params(m.n_chains, m.chain_len, m.box, m.kappa, n_exp=n_exp, seed=seed, stream=stream, dt=dt, **kw)


CASES = {
    "cfg1": lambda: KI.make(1),
    "ragged": lambda: KI.random_walk_melt(37, 29, 0.85, 2.0, 5),            # M = 1073, not a tile multiple
    "short": lambda: KI.random_walk_melt(400, 3, 0.85, 0.0, 6),            # N = 3: one angle per chain
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_nlist_bit_exact(kg, case, precision):
    m = CASES[case]()
    with context(kg, [m], precision) as ctx:
        offs, nbr = kg.kg_get_nlist(ctx, 0, m.M)
    oo, on = O.nlist(oparams(m, 12), m.x, RL, use_cells=True)
    assert np.array_equal(offs, oo)
    assert np.array_equal(nbr, on)


@pytest.mark.parametrize("precision", [0, 1])
def test_smallest_cell_grid(kg, precision):
    """Three Verlet cells a side, the fewest the library accepts: a box just
    above the 7 sigma minimum with skin 1.0 (r_c + skin = 2.12), so every
    stencil of 27 cells covers the whole box and each neighbouring cell is
    reached by exactly one image shift.  The list is bit-exact and 10 steps
    follow the oracle."""
    import torch
    m = KI.random_walk_melt(16, 19, 0.85, 1.0, 7)              # M = 304, L = 7.10
    rl = 2.0 ** (1 / 6) + 1.0
    assert int(m.box // rl) == 3
    dt = 0.002
    with context(kg, [m], precision, schedule=[kg.stage(2.0, 100, dt)], skin=1.0) as ctx:
        offs, nbr = kg.kg_get_nlist(ctx, 0, m.M)
        kg.kg_step(ctx, 10)
        x = np.zeros_like(m.x)
        kg.kg_get_config(ctx, 0, x)
    oo, on = O.nlist(oparams(m, 12), m.x, rl, use_cells=False)   # all pairs, minimum image
    assert np.array_equal(offs, oo) and np.array_equal(nbr, on)
    xo, uo = m.x.copy(), m.v.copy()
    O.run(oparams(m, 2.0, dt=dt), xo, uo, 0, 10)
    assert np.abs(x - xo).max() < (1e-9 if precision == 0 else 1e-4)


def _force_err(F, Fo):
    n = np.linalg.norm(F - Fo, axis=0)
    ref = np.maximum(np.linalg.norm(Fo, axis=0), np.sqrt((Fo ** 2).sum(axis=0).mean()))
    return (n / ref).max()


@pytest.mark.parametrize("n_exp", [2.0, 3.0, 5.75, 6.5, 9.0, 12.0])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_forces(kg, n_exp, precision, tol):
    m = KI.random_walk_melt(30, 40, 0.85, 1.5, 21)
    with context(kg, [m], precision, schedule=[kg.stage(n_exp, 10, 0.005)]) as ctx:
        F = np.zeros_like(m.x)
        e4 = np.zeros(4)
        kg.kg_forces(ctx, 0, F, e4)
    Fo, eo = O.forces(oparams(m, n_exp), m.x)
    assert _force_err(F, Fo) < tol
    assert e4 == pytest.approx(eo, rel=1e-9 if precision == 0 else 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_exp,dt", [(2.0, 0.002), (12.0, 0.0005)])   # unrelaxed start: small dt
def test_trajectory_10_steps(kg, precision, n_exp, dt):
    m = KI.make(1)
    with context(kg, [m], precision, schedule=[kg.stage(n_exp, 100, dt)]) as ctx:
        kg.kg_step(ctx, 10)
        x = np.zeros_like(m.x)
        v = np.zeros_like(m.v)
        kg.kg_get_config(ctx, 0, x, v)
    xo, uo = m.x.copy(), m.v.copy()
    O.run(oparams(m, n_exp, dt=dt), xo, uo, 0, 10)
    assert np.abs(x - xo).max() < 1e-4
    if precision == 0:
        assert np.abs(x - xo).max() < 1e-9


@pytest.mark.parametrize("case", ["cfg1", "ragged"])
@pytest.mark.parametrize("block", [64, 256])
def test_two_threads_per_monomer(kg, case, block):
    """Mixed step with two threads per monomer (split Verlet list, shuffled
    forces): 10 steps against the oracle at the trajectory bar, and against
    the one-thread kernel, which differs only in binary32 summation order."""
    m = CASES[case]()
    dt = 0.002
    out = {}
    for tpm in (1, 2):
        with context(kg, [m], 1, schedule=[kg.stage(2.0, 100, dt)], threads_per_monomer=tpm,
                     block_size=block) as ctx:
            kg.kg_step(ctx, 10)
            x = np.zeros_like(m.x)
            kg.kg_get_config(ctx, 0, x)
            out[tpm] = x
    xo, uo = m.x.copy(), m.v.copy()
    O.run(oparams(m, 2.0, dt=dt), xo, uo, 0, 10)
    assert np.abs(out[2] - xo).max() < 1e-4
    assert np.abs(out[2] - out[1]).max() < 1e-5


def _db_case(kappa=0.5, seed=31, n_chains=40, N=20):
    return KI.random_walk_melt(n_chains, N, 0.85, kappa, seed)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_exp,K", [(2.0, 300), (12.0, 400)])
def test_db_topology_bit_exact(kg, precision, n_exp, K):
    m = _db_case()
    q = oparams(m, n_exp)
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    acc_o = 0
    with context(kg, [m], precision, schedule=[kg.stage(n_exp, 10, 0.005)]) as ctx:
        for sweep in range(4):
            st = kg.kg_db_sweep_k(ctx, [K])
            a, e, acc = O.db_sweep(q, xo, uo, pido, sweep, K)
            assert (st.attempted, st.empty, st.accepted) == (a, e, acc)
            acc_o += acc
        x = np.zeros_like(m.x)
        v = np.zeros_like(m.v)
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, 0, x, v, pid)
    assert acc_o > 0
    assert np.array_equal(pid, pido)
    assert np.array_equal(x, xo)                  # moved and box-shifted bit for bit
    assert np.allclose(v, uo, rtol=0, atol=1e-6 if precision else 0)


def test_db_paper_metropolis_switch(kg):
    m = _db_case(seed=33)
    q = oparams(m, 2.0, paper_metropolis=True)
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    with context(kg, [m], 0, schedule=[kg.stage(2.0, 10, 0.005)], flags=1) as ctx:
        st = kg.kg_db_sweep_k(ctx, [500])
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, 0, None, None, pid)
    _, _, acc = O.db_sweep(q, xo, uo, pido, 0, 500)
    assert st.accepted == acc and np.array_equal(pid, pido)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_uneven_melts(kg, precision):
    """Three uneven melts in one context: forces and 10-step trajectories
    against the oracle, then one DB sweep per melt.  The sweep is checked
    bit for bit in both precisions from the GPU's own pre-sweep positions
    (the oracle's sequential loop on the same state): topology, accepted
    count, and positions with their box shifts."""
    melts = [KI.random_walk_melt(12, 30, 0.85, 0.0, 41), KI.random_walk_melt(7, 61, 0.85, 2.5, 42),
             KI.random_walk_melt(50, 8, 0.85, 1.0, 43)]
    dt = 0.002
    K = [200, 150, 100]
    with context(kg, melts, precision, seed=5, schedule=[kg.stage(3.0, 1000, dt)]) as ctx:
        forces = []
        for i, m in enumerate(melts):
            F = np.zeros_like(m.x)
            kg.kg_forces(ctx, i, F)
            forces.append(F)
        kg.kg_step(ctx, 10)
        pre = []
        for i, m in enumerate(melts):
            x, v = np.zeros_like(m.x), np.zeros_like(m.v)
            pid = np.zeros(m.M, dtype=np.int32)
            kg.kg_get_config(ctx, i, x, v, pid)
            pre.append((x, v, pid))
        st = kg.kg_db_sweep_k(ctx, K)
        out = []
        for i, m in enumerate(melts):
            x = np.zeros_like(m.x)
            pid = np.zeros(m.M, dtype=np.int32)
            kg.kg_get_config(ctx, i, x, None, pid)
            out.append((x, pid))
    acc = 0
    for i, m in enumerate(melts):
        q = oparams(m, 3.0, seed=5, stream=i, dt=dt)
        Fo, _ = O.forces(q, m.x)
        assert _force_err(forces[i], Fo) < (1e-10 if precision == 0 else 1e-5)
        xo, uo = m.x.copy(), m.v.copy()
        O.run(q, xo, uo, 0, 10)
        assert np.abs(pre[i][0] - xo).max() < (1e-9 if precision == 0 else 1e-4)
        xs, vs, ps = (a.copy() for a in pre[i])
        _, _, ac = O.db_sweep(q, xs, vs, ps, 0, K[i])
        acc += ac
        x, pid = out[i]
        assert np.array_equal(pid, ps)
        assert np.abs(x - xs).max() < 1e-9
    assert st.accepted == acc and acc > 0


def test_observables(kg):
    m = KI.random_walk_melt(25, 33, 0.85, 2.0, 51)
    with context(kg, [m], 0, schedule=[kg.stage(5.0, 10, 0.005)]) as ctx:
        r2 = np.zeros(m.chain_len)
        bh, ch = np.zeros(20), np.zeros(20)
        ob = kg.kg_observables(ctx, 0, r2, bh, ch, 20)
    q = oparams(m, 5.0, dt=0.005)
    want = O.observe(q, m.x, m.v, 0)
    for k in ("e_pair", "e_bond", "e_angle", "e_kin", "virial", "temperature", "pressure"):
        assert getattr(ob, k) == pytest.approx(want[k], rel=1e-9), k
    assert np.allclose(r2, O.r2n(q, m.x), rtol=1e-12, atol=0)
    obh, och = O.hist(q, m.x, 20)
    assert np.array_equal(bh, obh) and np.array_equal(ch, och)


def test_errors_and_recovery(kg):
    m = KI.random_walk_melt(4, 10, 0.05, 1.0, 61)     # dilute: L > 7
    bad = m.x.copy()
    bad[0, 5:] += 3.0                                   # bond 4-5 longer than 2 > R0
    with context(kg, [m], 1) as ctx:
        kg.kg_load_config(ctx, 0, bad, m.v)
        with pytest.raises(kg.KGError) as ei:
            kg.kg_step(ctx, 1)
        assert ei.value.status == kg.KG_ERR_BOND_OVERSTRETCH
        with pytest.raises(kg.KGError) as ei:
            kg.kg_step(ctx, 1)
        assert ei.value.status == kg.KG_ERR_STATE
        kg.kg_load_config(ctx, 0, m.x, m.v)            # a reload clears the latched error
        kg.kg_step(ctx, 2)
    with pytest.raises(kg.KGError) as ei:
        kg.kg_create(kg.make_params([(2, 5, 5.0, 1.0)]), 0)   # box below 7 sigma
    assert ei.value.status == kg.KG_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_degenerate_calls(kg, precision):
    """Zero steps and zero attempts change nothing; a lone chain has no
    partner chain, so every double-bridging draw is empty (as in the oracle),
    and MD on it still runs."""
    m = KI.make(1)
    with context(kg, [m], precision, schedule=[kg.stage(2.0, 100, 0.002)]) as ctx:
        kg.kg_step(ctx, 0)
        st = kg.kg_db_sweep_k(ctx, [0])
        x = np.zeros_like(m.x)
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, 0, x, None, pid)
    assert (st.attempted, st.accepted) == (0, 0)
    assert np.array_equal(x, m.x) and np.array_equal(pid, np.arange(m.M))
    one = KI.random_walk_melt(1, 40, 0.01, 1.0, 5)
    with context(kg, [one], precision, schedule=[kg.stage(2.0, 100, 0.002)]) as ctx:
        st = kg.kg_db_sweep_k(ctx, [500])
        kg.kg_step(ctx, 20)
        x = np.zeros_like(one.x)
        kg.kg_get_config(ctx, 0, x)
    a, e, acc = O.db_sweep(oparams(one, 2.0, dt=0.002), one.x.copy(), one.v.copy(),
                           np.arange(one.M, dtype=np.int32), 0, 500)
    assert (st.attempted, st.empty, st.accepted) == (a, e, acc) == (500, 500, 0)
    assert np.all(np.isfinite(x)) and not np.array_equal(x, one.x)


def test_runs_are_deterministic(kg):
    m = KI.make(1)
    outs = []
    for _ in range(2):
        with context(kg, [m], 1, schedule=[kg.stage(2.0, 10 ** 6, 0.002)]) as ctx:
            kg.kg_step(ctx, 60)
            kg.kg_db_sweep_k(ctx, [300])
            kg.kg_step(ctx, 60)
            x = np.zeros_like(m.x)
            kg.kg_get_config(ctx, 0, x)
            outs.append(x)
    assert np.array_equal(outs[0], outs[1])


def test_full_size_80k(kg):
    # 200 chains x 400 monomers (80,000), kappa = 2.5: the single-melt workload
    m = KI.make(2)
    for precision in (0, 1):
        with context(kg, [m], precision, schedule=[kg.stage(12.0, 10, 0.005)]) as ctx:
            offs, nbr = kg.kg_get_nlist(ctx, 0, m.M)
            F = np.zeros_like(m.x)
            kg.kg_forces(ctx, 0, F)
            if precision == 0:
                st = kg.kg_db_sweep_k(ctx, [800])
                pid = np.zeros(m.M, dtype=np.int32)
                kg.kg_get_config(ctx, 0, None, None, pid)
        q = oparams(m, 12.0)
        if precision == 0:
            oo, on = O.nlist(q, m.x, RL)
            assert np.array_equal(offs, oo) and np.array_equal(nbr, on)
        Fo, _ = O.forces(q, m.x)
        assert _force_err(F, Fo) < (1e-10 if precision == 0 else 1e-5)
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    _, _, acc = O.db_sweep(q, xo, uo, pido, 0, 800)
    assert st.accepted == acc and np.array_equal(pid, pido)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-3)])
def test_msd_without_db_matches_oracle(kg, precision, tol):
    """Core-softening-only ablation (no DB sweeps): the monomer MSD after 200
    steps against its definition (1/M) sum_i |r_i(t) - r_i(0)|^2 on the
    oracle's trajectory (relative bar: binary64 path 1e-8, mixed 1e-3, the
    trajectories' own divergence over 200 steps)."""
    m = KI.make(1)
    dt = 0.002
    with context(kg, [m], precision, schedule=[kg.stage(2.0, 10 ** 6, dt)]) as ctx:
        kg.kg_msd_reset(ctx, 0)
        assert kg.kg_msd(ctx, 0) == 0.0
        kg.kg_step(ctx, 200)
        msd = kg.kg_msd(ctx, 0)
    xo, uo = m.x.copy(), m.v.copy()
    O.run(oparams(m, 2.0, dt=dt), xo, uo, 0, 200)
    want = float(((xo - m.x) ** 2).sum(axis=0).mean())
    assert msd == pytest.approx(want, rel=tol)


def test_msd_is_unchanged_by_db_sweeps(kg):
    """A swap relabels monomers and shifts moved segments by box vectors but
    moves no monomer: the MSD before and after sweeps that accept swaps agree,
    and it still follows the monomers through a re-sort of the state."""
    m = _db_case(kappa=0.5)
    with context(kg, [m], 0, schedule=[kg.stage(2.0, 10 ** 6, 0.002)], sort_interval=7) as ctx:
        kg.kg_msd_reset(ctx, 0)
        kg.kg_step(ctx, 60)                      # crosses re-sorts
        before = kg.kg_msd(ctx, 0)
        acc = 0
        for _ in range(4):
            acc += kg.kg_db_sweep_k(ctx, [400]).accepted
        after = kg.kg_msd(ctx, 0)
    assert acc > 0
    assert after == pytest.approx(before, rel=1e-12)


def test_structure_factor_and_pair_distribution(kg):
    """App. A observables of the 1000-monomer melt after 100 steps, against the
    oracle's definitions on the same positions: S(q) for 300 reciprocal-lattice
    vectors (binary32 phases: 1e-5 relative + 1e-4 absolute), g(r) counts exact."""
    m = KI.make(1)
    rng = np.random.default_rng(5)
    hkl = rng.integers(-12, 13, (300, 3))
    hkl[0] = (0, 0, 0)                                   # S(0) = M
    with context(kg, [m], 1, schedule=[kg.stage(2.0, 10 ** 6, 0.002)]) as ctx:
        kg.kg_step(ctx, 100)
        S = kg.kg_structure_factor(ctx, 0, hkl)
        g = kg.kg_pair_distribution(ctx, 0, 4.0, 80)
        x = np.zeros_like(m.x)
        kg.kg_get_config(ctx, 0, x)
    assert S[0] == pytest.approx(m.M, rel=1e-6)
    So = SF.structure_factor(x, m.box, hkl)
    assert np.allclose(S, So, rtol=1e-5, atol=1e-4), np.abs(S - So).max()
    go = SF.pair_distribution(x, m.box, 4.0, 80)
    assert np.allclose(g, go, rtol=1e-12, atol=0)
    assert g.max() > 1.5                                   # the first-neighbour peak


def test_full_size_1600k(kg):
    """The benchmark melt (1000 chains x 1600, 1.6M monomers, kappa = 3.5) in
    the benchmark's launch configuration (mixed precision, skin 0.5, block 128,
    FENE continuation q = 0.01): Verlet list bit-exact, forces, a 400-attempt
    DB sweep (attempt, empty and accepted counts and the topology bit-exact),
    then positions two steps later, all against the oracle on the same input."""
    m = KI.make(5)
    dt = 0.0005
    with context(kg, [m], 1, schedule=[kg.stage(2.0, 100, dt)], skin=0.5, block_size=128,
                 fene_qmin=0.01) as ctx:
        offs, nbr = kg.kg_get_nlist(ctx, 0, m.M)
        F = np.zeros_like(m.x)
        kg.kg_forces(ctx, 0, F)
        st = kg.kg_db_sweep_k(ctx, [400])
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, 0, None, None, pid)
        kg.kg_step(ctx, 2)
        x = np.zeros_like(m.x)
        kg.kg_get_config(ctx, 0, x)
    q = oparams(m, 2.0, dt=dt, fene_qmin=0.01)
    oo, on = O.nlist(q, m.x, 2.0 ** (1 / 6) + 0.5)
    assert np.array_equal(offs, oo) and np.array_equal(nbr, on)
    del oo, on, offs, nbr
    Fo, _ = O.forces(q, m.x)
    assert _force_err(F, Fo) < 1e-5
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    a, e, acc = O.db_sweep(q, xo, uo, pido, 0, 400)
    assert (st.attempted, st.empty, st.accepted) == (a, e, acc)
    assert np.array_equal(pid, pido)
    O.run(q, xo, uo, 0, 2)
    assert np.abs(x - xo).max() < 1e-4


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_regularised_fene_forces(kg, precision, tol):
    # a few bonds pulled past r* = R0 sqrt(1 - qmin) and past R0 itself
    m = KI.random_walk_melt(20, 30, 0.85, 1.0, 81)
    x = m.x.copy()
    for c, f in ((0, 1.55), (3, 1.62), (7, 1.495)):
        s = c * 30 + 10
        b = x[:, s + 1] - x[:, s]
        x[:, s + 1:(c + 1) * 30] += (f / np.linalg.norm(b) - 1.0) * b[:, None]
    import torch
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=precision, seed=11,
                       fene_qmin=0.01)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, [kg.stage(2.0, 10, 0.002)])
        kg.kg_load_config(ctx, 0, x, m.v)
        F = np.zeros_like(x)
        e4 = np.zeros(4)
        kg.kg_forces(ctx, 0, F, e4)
    finally:
        kg.kg_destroy(ctx)
    q = oparams(m, 2.0, fene_qmin=0.01)
    Fo, eo = O.forces(q, x)
    assert _force_err(F, Fo) < tol
    assert e4[1] == pytest.approx(eo[1], rel=1e-9 if precision == 0 else 1e-5)


def test_long_run_across_resorts_and_sweeps(kg):
    # MD steps cross the periodic re-sort into cell order (every 200 steps) with
    # double-bridging sweeps in between; binary64 path against the oracle
    m = KI.random_walk_melt(30, 40, 0.85, 1.0, 91)
    dt = 0.002
    q = oparams(m, 2.0, dt=dt)
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    step = 0
    with context(kg, [m], 0, schedule=[kg.stage(2.0, 10 ** 9, dt)]) as ctx:
        for sweep, n in enumerate((150, 120, 90)):
            kg.kg_step(ctx, n)
            step = O.run(q, xo, uo, step, n)
            st = kg.kg_db_sweep_k(ctx, [300])
            _, _, acc = O.db_sweep(q, xo, uo, pido, sweep, 300)
            assert st.accepted == acc
        x = np.zeros_like(m.x)
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, 0, x, None, pid)
        offs, nbr = kg.kg_get_nlist(ctx, 0, m.M)
    assert np.array_equal(pid, pido)
    assert np.abs(x - xo).max() < 1e-8
    oo, on = O.nlist(q, x, RL)
    assert np.array_equal(offs, oo) and np.array_equal(nbr, on)


@pytest.mark.parametrize("sort_interval,tol", [(10 ** 6, 0.0), (50, 1e-6)])
def test_mixed_positions_do_not_depend_on_call_splitting(kg, sort_interval, tol):
    """Mixed mode folds its binary32 displacement into the binary64 positions
    at every Verlet build and at the end of every kg_step call: splitting the
    same steps into more calls, with the positions read in between, gives the
    same trajectory bit for bit, DB sweeps included.  With re-sorts the host
    tests the sort interval at call and graph boundaries, so a split run
    re-sorts a few steps later (step 257 instead of 250 here); the re-sort
    forces a Verlet build, which restarts the binary32 displacement, so the
    two runs differ at the binary32 rounding level of the positions."""
    m = KI.random_walk_melt(30, 40, 0.85, 1.0, 91)
    plan = [(120, 200), (120, 200), (60, 0)]          # (MD steps, DB attempts after them)

    def run(split):
        with context(kg, [m], 1, schedule=[kg.stage(2.0, 10 ** 9, 0.002)], sort_interval=sort_interval) as ctx:
            x = np.zeros_like(m.x)
            for n, k in plan:
                parts = [7, 13, n - 20] if split else [n]
                for q in parts:
                    kg.kg_step(ctx, q)
                    if split:
                        kg.kg_get_config(ctx, 0, x)
                if k:
                    kg.kg_db_sweep_k(ctx, [k])
            pid = np.zeros(m.M, dtype=np.int32)
            kg.kg_get_config(ctx, 0, x, None, pid)
            return x, pid

    xa, pa = run(False)
    xb, pb = run(True)
    assert np.array_equal(pa, pb)
    assert np.abs(xa - xb).max() <= tol



@pytest.mark.parametrize("skin,block", [(0.6, 64), (0.25, 256)])
def test_other_skin_and_block(kg, skin, block):
    import torch
    m = KI.make(1)
    dt = 0.002
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=0, seed=11, skin=skin,
                       block_size=block)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, [kg.stage(2.0, 10 ** 9, dt)])
        kg.kg_load_config(ctx, 0, m.x, m.v)
        offs, nbr = kg.kg_get_nlist(ctx, 0, m.M)
        kg.kg_step(ctx, 30)
        x = np.zeros_like(m.x)
        kg.kg_get_config(ctx, 0, x)
    finally:
        kg.kg_destroy(ctx)
    q = oparams(m, 2.0, dt=dt)
    oo, on = O.nlist(q, m.x, 2.0 ** (1 / 6) + skin)
    assert np.array_equal(offs, oo) and np.array_equal(nbr, on)
    xo, uo = m.x.copy(), m.v.copy()
    O.run(q, xo, uo, 0, 30)
    assert np.abs(x - xo).max() < 1e-9


def test_autotune_returns_a_working_setting(kg):
    import torch
    m = KI.random_walk_melt(60, 50, 0.85, 2.0, 93)
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=1, seed=3)
    best = kg.kg_autotune(p, [m.x], [m.v], kg.stage(2.0, -1, 0.002), 20, 0,
                          torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    assert best.trials >= 6 and best.block_size in (64, 128, 256) and 0.25 <= best.skin <= 0.6
    assert best.threads_per_monomer in (1, 2)
    assert 0 < best.ms_per_step < 100
