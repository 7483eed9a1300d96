"""Oracle pins for the double-bridging Monte Carlo moves (Fig. 1, Sec. II.B).

Pins: conservation of chains, chain length, monomers and bonds; every bond stays
a minimum image in unwrapped coordinates; the fast energy change (FENE log
terms + bending) equals the brute-force change of the total potential energy
(the U_MLJ parts cancel); the oracle's partner counts equal an independent
enumeration written here; and, on a tiny frozen system whose reachable
topologies are enumerated exhaustively, the sampled topology histogram matches
the Boltzmann distribution exp(-E)/Z (detailed balance).
"""
import itertools
import math
from collections import Counter, deque

import numpy as np
import pytest

import kg_inputs as KI
import oracle as O


def _dense(n_chains=10, N=12, kappa=1.0, n_exp=2.0, seed=4, rho=0.85, **kw):
    m = KI.random_walk_melt(n_chains, N, rho, kappa, seed)
    p = O.params(n_chains, N, m.box, kappa, n_exp=n_exp, **kw)
    return m, p


def _relaxed(steps=300, **kw):
    # the soft n = 2 bonds need a small first time step (Sec. II.B: dt_init ~ 0.001)
    m, p = _dense(**kw)
    x, u = m.x.copy(), m.v.copy()
    q = O.params(p.n_chains, p.chain_len, p.box, p.kappa, n_exp=p.n_exp, dt=0.002)
    O.run(q, x, u, 0, steps)
    return m, p, x, u


def _total_energy(p, x):
    _, e = O.forces(p, x)
    return e[0] + e[1] + e[2]


def _wrapped_by_pid(p, x, pid):
    w = x - p.box * np.floor(x / p.box)
    out = np.empty_like(w)
    out[:, pid] = w
    return out


def test_db_conserves_chains_monomers_and_bonds():
    m, p, x, u = _relaxed(n_chains=16, N=14, kappa=0.5)
    pid = np.arange(m.M, dtype=np.int32)
    w0 = _wrapped_by_pid(p, x, pid)
    u0 = u.copy()
    total_acc = 0
    for sweep in range(20):
        att, empty, acc = O.db_sweep(p, x, u, pid, sweep, 200)
        assert att == 200 and 0 <= acc <= att - empty
        total_acc += acc
        # pid is a permutation: every monomer kept exactly once
        assert np.array_equal(np.sort(pid), np.arange(m.M))
        # positions are unchanged up to box vectors, velocities travel with monomers
        w = _wrapped_by_pid(p, x, pid)
        dw = w - w0
        dw -= p.box * np.rint(dw / p.box)
        assert np.abs(dw).max() < 1e-9
        uu = np.empty_like(u)
        uu[:, pid] = u
        assert np.array_equal(uu, u0)
        # N_ch chains of N: every bond a minimum image, no longer than 1.3 after a swap
        b = np.diff(x.reshape(3, p.n_chains, p.chain_len), axis=2)
        blen = np.sqrt((b ** 2).sum(axis=0))
        assert blen.max() < p.R0 and np.abs(b).max() < 0.5 * p.box
    assert total_acc > 10


def test_fast_energy_change_equals_total_energy_change():
    m, p, x, u = _relaxed(n_chains=12, N=10, kappa=1.5)
    pid = np.arange(m.M, dtype=np.int32)
    seen = 0
    for sweep in range(400):
        e_tot0, e_topo0 = _total_energy(p, x), O.topo_energy(p, x)
        att, empty, acc = O.db_sweep(p, x, u, pid, sweep, 1)
        if acc:
            d_tot = _total_energy(p, x) - e_tot0
            d_topo = O.topo_energy(p, x) - e_topo0
            assert d_tot == pytest.approx(d_topo, rel=1e-9, abs=1e-9)
            seen += 1
    assert seen >= 5


# ---- an independent restatement of the move set, used to pin the oracle ----

def _d2(P, L, a, b):
    d = P[b] - P[a]
    d -= L * np.rint(d / L)
    return float(d @ d)


def _moves_of_bond(state, P, L, nch, N, c, b, lim2=1.3 * 1.3):
    """All admissible swaps removing bond (c, b): list of (kind, d, q)."""
    out = []
    u, w = state[c * N + b], state[c * N + b + 1]
    if _d2(P, L, u, w) > lim2:
        return out
    for d in range(nch):
        if d == c:
            continue
        # kind alpha: partner bond (d, b); new bonds (u, D_{b+1}), (D_b, w)
        Db, Db1 = state[d * N + b], state[d * N + b + 1]
        if _d2(P, L, u, Db1) <= lim2 and _d2(P, L, Db, w) <= lim2 and _d2(P, L, Db, Db1) <= lim2:
            out.append((0, d, b))
        # kind beta: partner bond (d, q), q = N-2-b; new bonds (u, D_q), (w, D_{q+1})
        q = N - 2 - b
        Dq, Dq1 = state[d * N + q], state[d * N + q + 1]
        if _d2(P, L, u, Dq) <= lim2 and _d2(P, L, w, Dq1) <= lim2 and _d2(P, L, Dq, Dq1) <= lim2:
            out.append((1, d, q))
    return out


def _apply(state, nch, N, kind, c, b, d, q):
    s = list(state)
    A, B = min(c, d), max(c, d)
    pA = b if A == c else q
    chA, chB = s[A * N:(A + 1) * N], s[B * N:(B + 1) * N]
    if kind == 0:
        nA = chA[:pA + 1] + chB[pA + 1:]
        nB = chB[:pA + 1] + chA[pA + 1:]
    else:
        qB = N - 2 - pA
        nA = chA[:pA + 1] + chB[:qB + 1][::-1]
        nB = chA[pA + 1:][::-1] + chB[qB + 1:]
    s[A * N:(A + 1) * N] = nA
    s[B * N:(B + 1) * N] = nB
    return tuple(s)


def test_partner_counts_match_independent_enumeration():
    m, p, x, u = _relaxed(n_chains=8, N=9, kappa=0.5, rho=1.2, steps=100)
    pid = np.arange(m.M, dtype=np.int32)
    P = x.T.copy()
    state = tuple(range(m.M))
    nz = 0
    for c in range(p.n_chains):
        for b in range(p.chain_len - 1):
            want = len(_moves_of_bond(state, P, p.box, p.n_chains, p.chain_len, c, b))
            assert O.db_partners(p, x, pid, c, b) == want
            nz += want > 0
    assert nz > 5


def _tiny_system(seed):
    nch, N = 3, 5
    m = KI.random_walk_melt(nch, N, 15 / 2.7 ** 3, 0.5, seed, d_min=0.6)
    return m, nch, N


def _reachable(P, L, nch, N, start):
    seen = {start}
    dq = deque([start])
    while dq:
        s = dq.popleft()
        for c in range(nch):
            for b in range(N - 1):
                for kind, d, q in _moves_of_bond(s, P, L, nch, N, c, b):
                    t = _apply(s, nch, N, kind, c, b, d, q)
                    if t not in seen:
                        seen.add(t)
                        dq.append(t)
    return seen


def _pick_tiny(seed=15):
    # 3 chains x 5 monomers, frozen; seed chosen for a 72-state topology space
    # with frequent acceptances at both tested stages
    m, nch, N = _tiny_system(seed)
    P = m.x.T.copy()
    states = _reachable(P, m.box, nch, N, tuple(range(nch * N)))
    assert 12 <= len(states) <= 400
    return m, nch, N, P, states


def _transition_matrix(P, L, nch, N, states, E, T, hastings=True):
    """Exact one-attempt kernel of the move set above with Metropolis-Hastings."""
    idx = {s: i for i, s in enumerate(states)}
    nb = nch * (N - 1)
    K = np.zeros((len(states), len(states)))
    cnt = lambda s, c, b: len(_moves_of_bond(s, P, L, nch, N, c, b))
    for s in states:
        i = idx[s]
        for c in range(nch):
            for b in range(N - 1):
                mv = _moves_of_bond(s, P, L, nch, N, c, b)
                for kind, d, q in mv:
                    t = _apply(s, nch, N, kind, c, b, d, q)
                    A, B = min(c, d), max(c, d)
                    pA, pB = (b, q) if A == c else (q, b)
                    ratio = (1 / cnt(t, A, pA) + 1 / cnt(t, B, pB)) / (1 / cnt(s, c, b) + 1 / cnt(s, d, q))
                    a = math.exp(-(E[idx[t]] - E[i]) / T) * (ratio if hastings else 1.0)
                    K[i, idx[t]] += min(1.0, a) / (nb * len(mv))
        K[i, i] += 1.0 - K[i].sum()
    return K


@pytest.mark.parametrize("n_exp,kappa", [(2.0, 0.5), (6.5, 1.5)])
def test_detailed_balance_exhaustive(n_exp, kappa):
    chi2 = pytest.importorskip("scipy.stats").chi2
    m, nch, N, P, states = _pick_tiny()
    states = sorted(states)
    idx = {s: i for i, s in enumerate(states)}
    p = O.params(nch, N, m.box, kappa, n_exp=n_exp, seed=99)
    # Boltzmann weights from the oracle's own topology energy
    E = np.array([O.topo_energy(p, np.ascontiguousarray(P[list(s)].T)) for s in states])
    boltz = np.exp(-(E - E.min()) / p.T)
    boltz /= boltz.sum()
    # (1) the exact kernel of the move set satisfies detailed balance w.r.t. exp(-E)
    K = _transition_matrix(P, m.box, nch, N, states, E, p.T)
    flux = boltz[:, None] * K
    assert np.abs(flux - flux.T).max() < 1e-15
    # (2) the oracle's one-attempt transitions follow that kernel
    x = np.ascontiguousarray(m.x.copy())
    u = np.zeros_like(x)
    pid = np.arange(nch * N, dtype=np.int32)
    counts = np.zeros_like(K)
    prev = idx[tuple(pid.tolist())]
    n_samples, acc = 60000, 0
    for sweep in range(n_samples):
        _, _, a = O.db_sweep(p, x, u, pid, sweep, 1)
        acc += a
        cur = idx[tuple(pid.tolist())]          # KeyError would mean an unreachable state
        counts[prev, cur] += 1
        prev = cur
    assert acc > 500
    visits = counts.sum(axis=1)
    expect = visits[:, None] * K
    assert np.all(counts[expect == 0] == 0)     # no transition the move set forbids
    use = expect > 5
    stat = (((counts - expect) ** 2)[use] / expect[use]).sum()
    dof = int(use.sum() - (visits > 0).sum())
    assert chi2.sf(stat, dof) > 1e-4, (stat, dof)


def test_metropolis_without_proposal_ratio_breaks_balance():
    # Fig. 1 states plain Metropolis acceptance.  With partner counts that
    # differ between x and x', dropping the proposal ratio breaks detailed
    # balance; the oracle's paper_metropolis switch follows that kernel.
    chi2 = pytest.importorskip("scipy.stats").chi2
    m, nch, N, P, states = _pick_tiny()
    states = sorted(states)
    idx = {s: i for i, s in enumerate(states)}
    p = O.params(nch, N, m.box, 0.5, n_exp=2.0, seed=5, paper_metropolis=True)
    E = np.array([O.topo_energy(p, np.ascontiguousarray(P[list(s)].T)) for s in states])
    boltz = np.exp(-(E - E.min()))
    boltz /= boltz.sum()
    Kp = _transition_matrix(P, m.box, nch, N, states, E, p.T, hastings=False)
    flux = boltz[:, None] * Kp
    assert np.abs(flux - flux.T).max() > 1e-6
    x = np.ascontiguousarray(m.x.copy())
    u = np.zeros_like(x)
    pid = np.arange(nch * N, dtype=np.int32)
    counts = np.zeros_like(Kp)
    prev = idx[tuple(pid.tolist())]
    for sweep in range(40000):
        O.db_sweep(p, x, u, pid, sweep, 1)
        cur = idx[tuple(pid.tolist())]
        counts[prev, cur] += 1
        prev = cur
    expect = counts.sum(axis=1)[:, None] * Kp
    use = expect > 5
    stat = (((counts - expect) ** 2)[use] / expect[use]).sum()
    dof = int(use.sum() - (counts.sum(axis=1) > 0).sum())
    assert chi2.sf(stat, dof) > 1e-4
