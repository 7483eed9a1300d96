"""The persistent batched launch (KG_FLAG_PERSISTENT): every melt of a context
advanced by cooperative launches of 50 MD steps, the Verlet rebuild inside
the launch between grid barriers.

* Same arithmetic as the default path (one thread per monomer, the same list
  build and step code): with re-sorts out of the way, positions, velocities
  and double-bridging topology after 600 steps and four DB sweeps of three
  uneven melts are bit-identical to the default path's, across the stage
  changes of a dt-ramped walk from n = 2 to n = 12.
* The bounded barrier wait: a self-test launch in which one block never
  arrives makes the other blocks give up after a short poll limit; the call
  returns KG_ERR_TIMEOUT, the context refuses work until the next
  kg_load_config, after reloading it steps like a fresh context, and an
  ordinary self-test launch then succeeds.
"""
import contextlib

import numpy as np
import pytest

import kg_inputs as KI

pytestmark = pytest.mark.gpu

# a dt-ramped walk through Xi (Eq. 11) to the WCA stage, 100 steps per stage
SCHED = [(2.0, 100, 0.0005), (2.0, 100, 0.001), (4.0, 100, 0.0015), (6.5, 100, 0.0025), (9.0, 100, 0.004),
         (12.0, 10 ** 9, 0.005)]


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


def _melts():
    return [KI.random_walk_melt(40, 50, 0.85, 1.0, 301), KI.random_walk_melt(25, 120, 0.85, 2.5, 302),
            KI.random_walk_melt(90, 20, 0.85, 0.0, 303)]


@contextlib.contextmanager
def _ctx(kg, melts, flags):
    import torch
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa) for m in melts], precision=kg.KG_MIXED, seed=5,
                       flags=flags, fene_qmin=0.01, sort_interval=10 ** 9, block_size=256, threads_per_monomer=1)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_set_potential_schedule(ctx, [kg.stage(n, k, dt) for n, k, dt in SCHED])
        for i, m in enumerate(melts):
            kg.kg_load_config(ctx, i, m.x, m.v)
        yield ctx
    finally:
        kg.kg_destroy(ctx)


def _state(kg, ctx, melts):
    out = []
    for i, m in enumerate(melts):
        x, v = np.zeros_like(m.x), np.zeros_like(m.v)
        pid = np.zeros(m.M, dtype=np.int32)
        kg.kg_get_config(ctx, i, x, v, pid)
        out.append((x, v, pid))
    return out


def _run(kg, flags):
    melts = _melts()
    with _ctx(kg, melts, flags) as ctx:
        acc = 0
        for _ in range(4):
            kg.kg_step(ctx, 150)
            acc += kg.kg_db_sweep_k(ctx, [m.M // 10 for m in melts]).accepted
        launches = kg.kg_profile_read(ctx)[2]
        return _state(kg, ctx, melts), acc, launches


def test_persistent_launch_is_bit_identical_to_the_default_path(kg):
    ref, acc_ref, l_ref = _run(kg, 0)
    per, acc_per, l_per = _run(kg, kg.KG_FLAG_PERSISTENT)
    assert acc_ref == acc_per and acc_ref > 0
    for (xa, va, pa), (xb, vb, pb) in zip(ref, per):
        assert np.array_equal(pa, pb)
        assert np.array_equal(xa, xb)
        assert np.array_equal(va, vb)
    assert l_per < l_ref                                  # fewer launches for the same steps


def test_barrier_wait_gives_up_and_the_context_recovers(kg):
    melts = _melts()
    with _ctx(kg, melts, kg.KG_FLAG_PERSISTENT) as ctx:
        kg.kg_step(ctx, 10)
        st = kg.kg_persistent_selftest(ctx, 0, 20000)       # block 0 never arrives
        assert st == kg.KG_ERR_TIMEOUT
        with pytest.raises(kg.KGError):
            kg.kg_step(ctx, 10)                             # latched until the next load
        for i, m in enumerate(melts):
            kg.kg_load_config(ctx, i, m.x, m.v)
        kg.kg_set_counters(ctx, 0, 0)
        kg.kg_set_potential_schedule(ctx, [kg.stage(n, k, dt) for n, k, dt in SCHED])   # back to its start
        kg.kg_step(ctx, 100)
        after = _state(kg, ctx, melts)
        assert kg.kg_persistent_selftest(ctx, -1, 1 << 24) == kg.KG_OK   # an ordinary two-step launch
    with _ctx(kg, melts, kg.KG_FLAG_PERSISTENT) as ctx:
        kg.kg_step(ctx, 100)
        fresh = _state(kg, ctx, melts)
    for (xa, va, pa), (xb, vb, pb) in zip(after, fresh):
        assert np.array_equal(pa, pb)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
