"""kg_r2n_noalloc: <R^2(n)> computed without allocating device memory.

Some callers cannot allocate: their device heap belongs to another framework,
or they call between steps of a latency-critical loop where a cudaMalloc (which
may synchronise the device) is not allowed.  This entry point keeps its
scratch in a file-scope device array; here it is called through the C ABI on
positions the caller already holds in device memory, twice in a row (the
array keeps the previous call's contents), and must agree with the <R^2(n)>
that kg_observables computes through a context.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import kg_inputs as KI

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_11001_gb300 as kg
    lib = kg.load()
    f = lib.kg_r2n_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    return kg


def _reference(kg, m):
    import torch
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=kg.KG_FP64)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_load_config(ctx, 0, m.x, m.v)
        r2 = np.zeros(m.chain_len)
        kg.kg_observables(ctx, 0, r2)
    finally:
        kg.kg_destroy(ctx)
    return r2


# (chains, N, kappa, padding of each row beyond M): N = 3000 needs 72 KiB of
# shared memory per block (above the 48 KiB default); padded rows exercise a
# stride larger than the monomer count
@pytest.mark.parametrize("shape", [(60, 80, 1.5, 0), (7, 333, 3.0, 0), (3, 3000, 2.0, 0), (5, 200, 1.0, 37)])
def test_noalloc_matches_context_path_twice(kg, shape):
    import torch
    n_ch, N, kappa, pad = shape
    m = KI.random_walk_melt(n_ch, N, 0.85, kappa, 71)
    want = _reference(kg, m)
    x = torch.full((3, m.M + pad), float("nan"), dtype=torch.float64, device="cuda")
    x[:, :m.M] = torch.from_numpy(m.x).cuda()               # (3, M + pad), stride M + pad
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        st = kg.load().kg_r2n_noalloc(x.data_ptr(), m.M + pad, n_ch, N, out.data_ptr(), stream.cuda_stream)
        assert st == kg.KG_OK
        stream.synchronize()
        assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)


def test_noalloc_on_a_side_stream_while_a_context_holds_the_device(kg):
    """A caller's own stream, with a simulation context alive on the device."""
    import torch
    m = KI.random_walk_melt(40, 120, 0.85, 2.5, 72)
    p = kg.make_params([(m.n_chains, m.chain_len, m.box, m.kappa)], precision=kg.KG_MIXED)
    ctx = kg.kg_create(p, 0, torch.cuda.current_stream().cuda_stream, kg.torch_allocator())
    try:
        kg.kg_load_config(ctx, 0, m.x, m.v)
        kg.kg_set_potential_schedule(ctx, [kg.stage(2.0, 10 ** 9, 0.002)])    # soft first stage
        kg.kg_step(ctx, 20)
        xs = np.zeros_like(m.x)
        kg.kg_get_config(ctx, 0, xs)
        want = np.zeros(m.chain_len)
        kg.kg_observables(ctx, 0, want)
        side = torch.cuda.Stream()
        x = torch.from_numpy(xs).cuda()
        torch.cuda.synchronize()
        for _ in range(2):
            out = torch.full((m.chain_len,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            st = kg.load().kg_r2n_noalloc(x.data_ptr(), m.M, m.n_chains, m.chain_len, out.data_ptr(),
                                          side.cuda_stream)
            assert st == kg.KG_OK
            side.synchronize()
            assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)
    finally:
        kg.kg_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_array(kg):
    import torch
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    big_chains = 2097152 // 4 + 1                             # n_chains * 4 > the maximum
    st = kg.load().kg_r2n_noalloc(x.data_ptr(), big_chains * 4, big_chains, 4, out.data_ptr(), None)
    assert st == kg.KG_ERR_INVALID_ARG
    st = kg.load().kg_r2n_noalloc(x.data_ptr(), 9686, 1, 9686, out.data_ptr(), None)   # chain too long
    assert st == kg.KG_ERR_INVALID_ARG
