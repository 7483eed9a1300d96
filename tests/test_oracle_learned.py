"""Oracle pins for the learned double-bridging proposal (not in the paper).

Pins: the two FP64 network implementations (C and numpy) agree; the numpy
gradient equals finite differences of the loss; the move features do not depend
on which of the swap's two bonds was drawn; with zero weights the proposal is
exactly uniform over a bond's partner list; and for random weights the oracle's
one-attempt transitions on the exhaustively enumerated 72-state system follow
the exact kernel of that proposal with Metropolis-Hastings acceptance, whose
stationary distribution is exp(-E)/Z (detailed balance).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp
from test_oracle_db import _apply, _moves_of_bond, _pick_tiny


def test_mlp_implementations_agree():
    rng = np.random.default_rng(1)
    w = mlp.init(3)
    w[64 * 24:64 * 24 + 64] = rng.normal(size=64) * 0.1
    F = rng.normal(size=(20, 24))
    s, _ = mlp.forward(w, F)
    for i in range(20):
        assert O.mlp_forward(w, F[i]) == pytest.approx(s[i], rel=1e-12, abs=1e-12)


def test_mlp_gradient_finite_difference():
    rng = np.random.default_rng(2)
    w = mlp.init(5)
    F = rng.normal(size=(33, 24))
    t = rng.random(33)
    _, g = mlp.loss_and_grad(w, F, t)
    h = 1e-6
    for i in rng.choice(len(w), 60, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, F, t)[0] - mlp.loss_and_grad(wm, F, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def _energy_table(m, nch, N, P, states, p):
    return np.array([O.topo_energy(p, np.ascontiguousarray(P[list(s)].T)) for s in states])


def _learned_kernel(m, nch, N, P, states, p, w, lam):
    """Exact one-attempt kernel of the learned proposal with MH acceptance."""
    idx = {s: i for i, s in enumerate(states)}
    nb = nch * (N - 1)
    E = _energy_table(m, nch, N, P, states, p)

    def xs(s):
        return np.ascontiguousarray(P[list(s)].T)

    def weights(s, c, b):
        mv = _moves_of_bond(s, P, m.box, nch, N, c, b)
        # order as the proposal does: id of the monomer bonding to b's lower end, then partner bond's other id
        keys = []
        for kind, d, q in mv:
            if kind == 0:
                keys.append((s[d * N + b + 1], s[d * N + b]))
            else:
                keys.append((s[d * N + q], s[d * N + q + 1]))
        order = np.argsort([k[0] * 10 ** 6 + k[1] for k in keys], kind="stable")
        mv = [mv[i] for i in order]
        if not mv:
            return [], np.zeros(0)
        x = xs(s)
        logits = np.array([O.mlp_forward(w, O.move_features(p, x, c, b, kind, d, q)) for kind, d, q in mv])
        e = np.exp(logits - logits.max())
        return mv, (1 - lam) * e / e.sum() + lam / len(mv)

    def canon(c, b, kind, d, q):
        A, B = min(c, d), max(c, d)
        return (kind, A, B, b if A == c else q, q if A == c else b)

    def prob(s, c, b, key):
        mv, pi = weights(s, c, b)
        for (kind, d, q), pj in zip(mv, pi):
            if canon(c, b, kind, d, q) == key:
                return pj
        return 0.0

    K = np.zeros((len(states), len(states)))
    for s in states:
        i = idx[s]
        for c in range(nch):
            for b in range(N - 1):
                mv, pi = weights(s, c, b)
                for (kind, d, q), pj in zip(mv, pi):
                    key = canon(c, b, kind, d, q)
                    _, A, B, pA, pB = key
                    t = _apply(s, nch, N, kind, c, b, d, q)
                    q_f = prob(s, c, b, key) + prob(s, d, q, key)
                    q_r = prob(t, A, pA, key) + prob(t, B, pB, key)
                    a = math.exp(-(E[idx[t]] - E[i]) / p.T) * q_r / q_f
                    K[i, idx[t]] += pj * min(1.0, a) / nb
        K[i, i] += 1.0 - K[i].sum()
    return K, E


def _run_chain(m, nch, N, states, p, w, lam, n):
    idx = {s: i for i, s in enumerate(states)}
    x = np.ascontiguousarray(m.x.copy())
    u = np.zeros_like(x)
    pid = np.arange(nch * N, dtype=np.int32)
    counts = np.zeros((len(states), len(states)))
    prev = idx[tuple(pid.tolist())]
    acc = 0
    for sweep in range(n):
        (_, _, a), _, _ = O.db_sweep_learned(p, x, u, pid, sweep, 1, w, lam)
        acc += a
        cur = idx[tuple(pid.tolist())]
        counts[prev, cur] += 1
        prev = cur
    return counts, acc


@pytest.mark.parametrize("weights", ["zero", "random"])
def test_learned_proposal_detailed_balance(weights):
    chi2 = pytest.importorskip("scipy.stats").chi2
    m, nch, N, P, states = _pick_tiny()
    states = sorted(states)
    p = O.params(nch, N, m.box, 0.5, n_exp=2.0, seed=17)
    w = np.zeros(O.MLP_NPARAM) if weights == "zero" else mlp.init(7, scale=1.5)
    lam = 0.1
    K, E = _learned_kernel(m, nch, N, P, states, p, w, lam)
    boltz = np.exp(-(E - E.min()) / p.T)
    boltz /= boltz.sum()
    flux = boltz[:, None] * K
    assert np.abs(flux - flux.T).max() < 1e-14
    counts, acc = _run_chain(m, nch, N, states, p, w, lam, 30000)
    assert acc > 300
    expect = counts.sum(axis=1)[:, None] * K
    assert np.all(counts[expect == 0] == 0)
    use = expect > 5
    stat = (((counts - expect) ** 2)[use] / expect[use]).sum()
    dof = int(use.sum() - (counts.sum(axis=1) > 0).sum())
    assert chi2.sf(stat, dof) > 1e-4, (stat, dof)


def test_zero_weights_give_the_uniform_kernel():
    m, nch, N, P, states = _pick_tiny()
    states = sorted(states)
    p = O.params(nch, N, m.box, 0.5, n_exp=2.0)
    from test_oracle_db import _transition_matrix
    E = _energy_table(m, nch, N, P, states, p)
    K0 = _transition_matrix(P, m.box, nch, N, states, E, p.T)
    K1, _ = _learned_kernel(m, nch, N, P, states, p, np.zeros(O.MLP_NPARAM), 0.1)
    assert np.abs(K0 - K1).max() < 1e-13


def test_features_do_not_depend_on_the_drawn_bond():
    m, nch, N, P, states = _pick_tiny()
    p = O.params(nch, N, m.box, 1.5, n_exp=3.0)
    s = sorted(states)[5]
    x = np.ascontiguousarray(P[list(s)].T)
    n = 0
    for c in range(nch):
        for b in range(N - 1):
            for kind, d, q in _moves_of_bond(s, P, m.box, nch, N, c, b):
                f1 = O.move_features(p, x, c, b, kind, d, q)
                f2 = O.move_features(p, x, d, q, kind, c, b)
                assert np.allclose(f1, f2, rtol=1e-12, atol=1e-12)
                n += 1
    assert n > 0


def _features_by_move(p, P, state, nch, N, c, b):
    """features of every admissible swap of bond (c, b), keyed by the two new bonds"""
    x = np.ascontiguousarray(P[list(state)].T)
    u, w = state[c * N + b], state[c * N + b + 1]
    out = {}
    for kind, d, q in _moves_of_bond(state, P, p.box, nch, N, c, b):
        if kind == 0:
            Y, X = state[d * N + b], state[d * N + b + 1]
        else:
            X, Y = state[d * N + q], state[d * N + q + 1]
        out[frozenset([frozenset([u, X]), frozenset([Y, w])])] = O.move_features(p, x, c, b, kind, d, q)
    return out


def test_features_do_not_depend_on_slot_numbering_direction():
    # reversing the slot order of one chain relabels kinds 0 <-> 1 and p <-> N-2-p
    # but is the same melt: every move keeps its features
    m, nch, N, P, states = _pick_tiny()
    p = O.params(nch, N, m.box, 1.5, n_exp=3.0)
    n = 0
    for s in sorted(states)[:12]:
        for d in range(nch):
            r = list(s)
            r[d * N:(d + 1) * N] = r[d * N:(d + 1) * N][::-1]
            for c in range(nch):
                for b in range(N - 1):
                    f1 = _features_by_move(p, P, s, nch, N, c, b)
                    f2 = _features_by_move(p, P, tuple(r), nch, N, c, N - 2 - b if c == d else b)
                    assert f1.keys() == f2.keys()
                    for k in f1:
                        assert np.allclose(f1[k], f2[k], rtol=1e-12, atol=1e-12), (s, d, c, b)
                        n += 1
    assert n > 50


def test_sweep_log():
    m, nch, N, P, states = _pick_tiny()
    p = O.params(nch, N, m.box, 0.5, n_exp=2.0, seed=3)
    x = np.ascontiguousarray(m.x.copy())
    u = np.zeros_like(x)
    pid = np.arange(nch * N, dtype=np.int32)
    (att, empty, acc), lf, lt = O.db_sweep_learned(p, x, u, pid, 0, 200, np.zeros(O.MLP_NPARAM), 0.1, log_cap=1000)
    assert len(lf) >= att - empty and np.isfinite(lf).all()
    assert ((lt > 0) & (lt <= 1)).all()
    assert np.allclose(lt, np.minimum(1.0, np.exp(-lf[:, 22])))


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    # hand values: 8 significant bits, ties to even
    assert O.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert O.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert O.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7
    assert O.bf16_round(-3.0) == -3.0 and O.bf16_round(0.0) == 0.0
    rng = np.random.default_rng(4)
    v = rng.normal(size=2000) * 10.0 ** rng.uniform(-6, 3, 2000)
    # binary32 inputs: torch's float32 -> bfloat16 conversion rounds to nearest even
    v32 = v.astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(v32.astype(np.float64)), ref)
    assert all(O.bf16_round(a) == b for a, b in zip(v32.astype(np.float64), ref))
    # binary64 inputs: C and numpy agree, and the result is within half a bf16 ulp
    c = np.array([O.bf16_round(a) for a in v])
    assert np.array_equal(c, mlp.bf16(v))
    assert np.all(np.abs(c - v) <= np.abs(v) * 2.0 ** -8)


def test_bf16_network_tracks_fp64():
    rng = np.random.default_rng(6)
    w = mlp.init(9)
    F = rng.normal(size=(200, 24))
    t = rng.random(200)
    s64, _ = mlp.forward(w, F)
    s16, _ = mlp.forward_bf16(w, F)
    assert np.abs(s16 - s64).max() < 0.05 * (1 + np.abs(s64).max())
    l64, g64 = mlp.loss_and_grad(w, F, t)
    l16, g16 = mlp.loss_and_grad_bf16(w, F, t)
    assert l16 == pytest.approx(l64, rel=2e-2)
    assert np.dot(g16, g64) / np.linalg.norm(g16) / np.linalg.norm(g64) > 0.999
    # exactly representable weights and inputs: the two agree to rounding of sums
    wd = mlp.sparse_dyadic(1)
    Fb = mlp.bf16(F)
    assert np.allclose(mlp.forward_bf16(wd, Fb)[0], mlp.forward(wd, Fb)[0], rtol=1e-12, atol=1e-12)


def test_learned_sweep_bf16_inputs():
    # the input rounding changes features by <= 2^-9 relative; with the sparse
    # dyadic network the sweep still balances (exact kernel on bf16 inputs)
    m, nch, N, P, states = _pick_tiny()
    p = O.params(nch, N, m.box, 0.5, n_exp=2.0, seed=5)
    x = np.ascontiguousarray(m.x.copy())
    u = np.zeros_like(x)
    pid = np.arange(nch * N, dtype=np.int32)
    (att, empty, acc), _, _ = O.db_sweep_learned(p, x, u, pid, 0, 400, mlp.sparse_dyadic(2), 0.1,
                                                 bf16_inputs=True)
    assert att == 400 and acc > 0


def test_candidate_list_matches_enumeration():
    m, nch, N, P, states = _pick_tiny()
    p = O.params(nch, N, m.box, 0.5, n_exp=2.0)
    for s in sorted(states)[:10]:
        x = np.ascontiguousarray(P[list(s)].T)
        pid = np.array(s, dtype=np.int32)
        for c in range(nch):
            for b in range(N - 1):
                got = O.db_candidates(p, x, pid, c, b)
                assert sorted(got) == sorted(_moves_of_bond(s, P, m.box, nch, N, c, b))
                assert len(got) == O.db_partners(p, x, pid, c, b)
