"""GPU parity of the learned double-bridging proposal (through the C ABI).

Bars: candidate lists bit-exact; FP64 features <= 1e-12 (relative to 1 +
|value|); logits against the oracle network evaluated at the kernel's bf16
rounding points within 1e-3 of the logit scale (an fp32-summed value can land
on the other side of a bf16 rounding boundary of a hidden unit), and exact for
weights and inputs the bf16 network represents exactly; gradients within 1e-2
(norm-wise per parameter block) of the same emulation; sweeps with exactly
represented weights bit-exact against the oracle's sweep on bf16 inputs.
"""
import contextlib

import numpy as np
import pytest

import kg_inputs as KI
import oracle as O
from oracle import mlp

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


@contextlib.contextmanager
def context(kg, melts, precision=0, seed=11, n_exp=2.0):
    import torch
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa) for m in melts], precision=precision, seed=seed)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, [kg.stage(n_exp, 10, 0.005)])
        for i, m in enumerate(melts):
            kg.kg_load_config(ctx, i, m.x, m.v)
        yield ctx
    finally:
        kg.kg_destroy(ctx)


def oparams(m, n_exp=2.0, seed=11):
    return O.params(m.n_chains, m.chain_len, m.box, m.kappa, n_exp=n_exp, seed=seed)


def _melt(seed=31):
    return KI.random_walk_melt(40, 20, 0.85, 0.5, seed)


def _scale(w, F):
    """magnitude of the output sum: sum_j |w3_j h2_j| + |b3| (emulated network)"""
    W1, b1, W2, b2, w3, b3 = mlp.unpack_bf16(w)
    _, (_, _, _, a2, h2) = mlp.forward_bf16(w, F)
    return np.abs(h2 * w3).sum(axis=1) + abs(b3)


@pytest.mark.parametrize("n", [1, 37, 1000])
def test_forward_matches_bf16_network(kg, n):
    rng = np.random.default_rng(n)
    F = rng.normal(size=(n, 24)) * rng.choice([0.1, 1.0, 5.0], size=(n, 24))
    w = mlp.init(3)
    w[64 * 24:64 * 24 + 64] = rng.normal(size=64) * 0.2          # b1
    w[-1] = 0.3
    m = _melt()
    with context(kg, [m]) as ctx:
        assert np.array_equal(kg.kg_mlp_forward(ctx, F), np.zeros(n))   # fresh context: zero weights
        kg.kg_mlp_set_weights(ctx, w)
        s = kg.kg_mlp_forward(ctx, F)
        assert np.array_equal(kg.kg_mlp_get_weights(ctx), w.astype(np.float32).astype(np.float64))
        wd = mlp.sparse_dyadic(4)
        kg.kg_mlp_set_weights(ctx, wd)
        sd = kg.kg_mlp_forward(ctx, mlp.bf16(F))
    ref, _ = mlp.forward_bf16(w, F)
    S = _scale(w, F)
    err = np.abs(s - ref)
    assert np.all(err <= 1e-3 * S + 1e-6)
    assert np.mean(err <= 1e-5 * S + 1e-6) > 0.9
    # exactly representable network: the FP64 logits of the bf16 inputs
    ref_d, _ = mlp.forward(wd, mlp.bf16(F))
    assert np.allclose(sd, ref_d, rtol=1e-6, atol=1e-6)


# 5000 rows: 313 row tiles, so the weight gradients sum 20 chunks of 256 rows,
# the last one partial
@pytest.mark.parametrize("n", [16, 37, 1000, 5000])
def test_loss_gradient(kg, n):
    rng = np.random.default_rng(10 + n)
    F = rng.normal(size=(n, 24))
    t = rng.random(n)
    w = mlp.init(5)
    w[64 * 24:64 * 24 + 64] = rng.normal(size=64) * 0.1
    m = _melt()
    with context(kg, [m]) as ctx:
        kg.kg_mlp_set_weights(ctx, w)
        loss, g = kg.kg_mlp_loss_grad(ctx, F, t)
    l16, g16 = mlp.loss_and_grad_bf16(w, F, t)
    l64, g64 = mlp.loss_and_grad(w, F, t)
    assert loss == pytest.approx(l16, rel=1e-4)
    blocks = [(0, 1536), (1536, 1600), (1600, 5696), (5696, 5760), (5760, 5824), (5824, 5825)]
    for a, b in blocks:
        ref = np.linalg.norm(g16[a:b]) + 1e-9
        assert np.linalg.norm(g[a:b] - g16[a:b]) <= 1e-2 * ref, (a, b)
        # against the exact FP64 gradient: bf16 inputs and hidden units (and the
        # ReLU masks they flip) leave a few per cent on small batches
        cos = np.dot(g[a:b], g64[a:b]) / (np.linalg.norm(g[a:b]) * np.linalg.norm(g64[a:b]) + 1e-30)
        assert cos > 0.99 and np.linalg.norm(g[a:b] - g64[a:b]) <= 0.15 * np.linalg.norm(g64[a:b]) + 1e-9, (a, b)


def test_proposal_matches_oracle(kg):
    m = _melt(32)
    q = oparams(m)
    wd = mlp.sparse_dyadic(5)
    w = mlp.init(6)
    pid = np.arange(m.M, dtype=np.int32)
    checked = 0
    with context(kg, [m]) as ctx:
        for (weights, lam) in ((None, 1.0), (wd, 0.25), (w, 0.1)):
            if weights is not None:
                kg.kg_mlp_set_weights(ctx, weights)
            for c in range(0, m.n_chains, 3):
                for b in range(0, m.chain_len - 1, 2):
                    got = kg.kg_db_proposal(ctx, 0, c, b, lam)
                    exp = O.db_candidates(q, m.x, pid, c, b)
                    assert [(int(k), int(d), int(p)) for k, d, p in zip(got["kind"], got["chain"], got["bond"])] == exp
                    if not exp:
                        continue
                    Fo = np.array([O.move_features(q, m.x, c, b, *e) for e in exp])
                    assert np.all(np.abs(got["features"] - Fo) <= 1e-12 * (1 + np.abs(Fo)))
                    s = got["logits"]
                    if weights is None:
                        assert np.array_equal(s, np.zeros(len(exp)))
                    elif weights is wd:
                        assert np.allclose(s, mlp.forward(wd, mlp.bf16(Fo))[0], rtol=1e-6, atol=1e-6)
                    else:
                        ref = mlp.forward_bf16(w, Fo)[0]
                        assert np.all(np.abs(s - ref) <= 1e-3 * _scale(w, Fo) + 1e-6)
                    # mixture in FP64 from the kernel's own logits, list order
                    e = np.exp(s - s.max())
                    pi = (1 - lam) * e / e.sum() + lam / len(s)
                    assert np.allclose(got["prob"], pi, rtol=1e-14, atol=0)
                    assert abs(got["prob"].sum() - 1) < 1e-12
                    checked += 1
    assert checked > 30


@pytest.mark.parametrize("weights,lam", [("uniform", 1.0), ("zero", 0.3), ("dyadic", 0.1)])
@pytest.mark.parametrize("precision", [0, 1])
def test_learned_sweep_bit_exact(kg, weights, lam, precision):
    m = _melt(33)
    q = oparams(m)
    w = {"uniform": np.zeros(O.MLP_NPARAM), "zero": np.zeros(O.MLP_NPARAM),
         "dyadic": mlp.sparse_dyadic(7)}[weights]
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    acc_all = 0
    K = 300
    with context(kg, [m], precision) as ctx:
        kg.kg_mlp_set_weights(ctx, w)
        for sweep in range(3):
            st = kg.kg_db_sweep_learned_k(ctx, [K], lam)
            (a, e, acc), _, _ = O.db_sweep_learned(q, xo, uo, pido, sweep, K, w, lam, bf16_inputs=True)
            assert (st.attempted, st.empty, st.accepted) == (a, e, acc), sweep
            acc_all += acc
        x = np.zeros_like(m.x)
        v = np.zeros_like(m.v)
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, 0, x, v, pid)
    assert acc_all > 0
    assert np.array_equal(pid, pido)
    assert np.array_equal(x, xo)
    assert np.allclose(v, uo, rtol=0, atol=1e-6 if precision else 0)


def test_log_matches_oracle(kg):
    m = _melt(34)
    q = oparams(m)
    w = mlp.sparse_dyadic(8)
    xo, uo, pido = m.x.copy(), m.v.copy(), np.arange(m.M, dtype=np.int32)
    with context(kg, [m]) as ctx:
        kg.kg_mlp_set_weights(ctx, w)
        kg.kg_mlp_log(ctx, 100000)
        rows_f, rows_t = [], []
        for sweep in range(2):
            kg.kg_db_sweep_learned_k(ctx, [800], 0.2)
            _, lf, lt = O.db_sweep_learned(q, xo, uo, pido, sweep, 800, w, 0.2, log_cap=100000, bf16_inputs=True)
            rows_f.append(lf)
            rows_t.append(lt)
        f, t = kg.kg_mlp_log_read(ctx, 100000)
    fo, to = np.concatenate(rows_f), np.concatenate(rows_t)
    assert f.shape == fo.shape and len(fo) > 100
    assert np.all(np.abs(f - fo) <= 1e-12 * (1 + np.abs(fo)))
    assert np.allclose(t, to, rtol=1e-12, atol=0)


def test_log_ring_keeps_the_newest_rows(kg):
    m = _melt(35)
    with context(kg, [m]) as ctx:
        kg.kg_mlp_log(ctx, 1 << 16)
        kg.kg_db_sweep_learned_k(ctx, [400], 1.0)
        full_f, full_t = kg.kg_mlp_log_read(ctx, 1 << 16)
        n = len(full_t)
        assert n > 50
        cap = n // 3
        kg.kg_mlp_log(ctx, cap)                    # a fresh, smaller ring
        kg.kg_set_counters(ctx, 0, 0)
        # the same sweep again: identical rows (topology restored by reloading)
        kg.kg_load_config(ctx, 0, m.x, m.v)
        kg.kg_db_sweep_learned_k(ctx, [400], 1.0)
        f, t = kg.kg_mlp_log_read(ctx, cap)
    assert len(t) == cap
    assert np.array_equal(t, full_t[n - cap:])
    assert np.array_equal(f, full_f[n - cap:])


def test_training_lowers_the_loss(kg):
    m = KI.random_walk_melt(60, 40, 0.85, 1.5, 36)
    with context(kg, [m]) as ctx:
        kg.kg_mlp_log(ctx, 200000)
        for _ in range(10):
            kg.kg_db_sweep_learned_k(ctx, [4000], 1.0)
        f, t = kg.kg_mlp_log_read(ctx, 200000)
        assert len(t) > 1000
        kg.kg_mlp_set_weights(ctx, mlp.init(11, scale=0.5))
        w0 = kg.kg_mlp_get_weights(ctx)
        l0, _ = kg.kg_mlp_loss_grad(ctx, f, t)
        kg.kg_mlp_train(ctx, 1, 256, 1e-3)
        w1 = kg.kg_mlp_get_weights(ctx)
        kg.kg_mlp_train(ctx, 300, 256, 3e-3)
        l1, _ = kg.kg_mlp_loss_grad(ctx, f, t)
    # Adam's first step moves every parameter with a non-zero gradient by ~lr
    dw = np.abs(w1 - w0)
    assert dw.max() <= 1e-3 * 1.01 and np.median(dw[dw > 0]) > 0.5e-3
    assert l1 < l0 - 0.02, (l0, l1)
    # the network's loss against the oracle's emulation on the same rows
    l16, _ = mlp.loss_and_grad_bf16(w0, f, t)
    assert l0 == pytest.approx(l16, rel=1e-4)


def test_learned_sweep_rejects_bad_lambda(kg):
    m = _melt()
    with context(kg, [m]) as ctx:
        for lam in (0.0, -0.1, 1.5, float("nan")):
            with pytest.raises(kg.KGError):
                kg.kg_db_sweep_learned_k(ctx, [10], lam)
        with pytest.raises(kg.KGError):               # nothing logged yet
            kg.kg_mlp_train(ctx, 1, 16, 1e-3)


def test_trained_network_raises_acceptance(kg):
    """What the trained network gains over the uniform partner draw.  A
    learned proposal can only help when a drawn bond has two or more
    admissible partners; that is frequent only for short chains (at N = 800
    the lists hold at most one swap), so this uses 10,000 chains of N = 10 in
    the soft n = 2 stage.  The network is trained online on uniform sweeps of
    the same melt; then each round saves the state, runs a uniform sweep, restores
    the state and the sweep index, and runs a learned sweep (lambda = 0.1): both
    see the same configuration and the same bond draws, so single-partner draws
    cancel and the paired difference of accepted swaps measures the gain."""
    import torch
    m = KI.random_walk_melt(10000, 10, 0.85, 2.0, 77)
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=1, seed=17, fene_qmin=0.01)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, [kg.stage(2.0, 300, 0.0005), kg.stage(2.0, 300, 0.001),
                                           kg.stage(2.0, 300, 0.002), kg.stage(2.0, 10 ** 15, 0.005)])
        kg.kg_load_config(ctx, 0, m.x, m.v)
        kg.kg_step(ctx, 1200)
        K = m.M // 10
        kg.kg_mlp_log(ctx, 4_000_000)
        for _ in range(10):                        # log: uniform proposal through the learned path
            kg.kg_step(ctx, 50)
            kg.kg_db_sweep_learned_k(ctx, [K], 1.0)
        kg.kg_mlp_set_weights(ctx, mlp.init(0))
        kg.kg_mlp_train(ctx, 800, 2048, 2e-3)
        kg.kg_mlp_log(ctx, 0)
        x, v, pid = np.zeros_like(m.x), np.zeros_like(m.v), np.zeros(m.M, dtype=np.int32)
        diff, acc_u, acc_l, ne_u, ne_l = [], 0, 0, 0, 0
        for _ in range(12):
            kg.kg_step(ctx, 50)
            kg.kg_get_config(ctx, 0, x, v, pid)
            step, sweep = kg.kg_get_counters(ctx)
            su = kg.kg_db_sweep_k(ctx, [K])
            kg.kg_load_config(ctx, 0, x, v, pid)
            kg.kg_set_counters(ctx, step, sweep)
            sl = kg.kg_db_sweep_learned_k(ctx, [K], 0.1)
            diff.append(sl.accepted - su.accepted)
            acc_u += su.accepted
            acc_l += sl.accepted
            ne_u += su.attempted - su.empty
            ne_l += sl.attempted - sl.empty
    finally:
        kg.kg_destroy(ctx)
    d = np.asarray(diff, dtype=float)
    z = d.mean() / (d.std(ddof=1) / np.sqrt(len(d)))
    gain = (acc_l / ne_l) / (acc_u / ne_u) - 1.0
    assert z > 4.0 and gain > 0.02, (d, z, gain)
