"""Oracle pins for the counter-based generator (Philox4x32-10) and its normals.

The oracle's Philox is written from Salmon et al. (SC'11); it is pinned here to
an independent implementation, Triton's ``tl.randint4x``/``philox`` run by
Triton's CPU interpreter, on arbitrary counters and keys.
"""
import os

os.environ.setdefault("TRITON_INTERPRET", "1")   # run Triton's reference on the CPU

import numpy as np  # noqa: E402
import pytest  # noqa: E402

import oracle as O  # noqa: E402


def _triton_philox(ctrs, keys):
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def kern(c_ptr, k_ptr, o_ptr, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32)
        c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32)
        c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32)
        c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32)
        k0 = tl.load(k_ptr + 2 * i + 0).to(tl.uint32)
        k1 = tl.load(k_ptr + 2 * i + 1).to(tl.uint32)
        r0, r1, r2, r3 = tl.random.philox_impl(c0, c1, c2, c3, k0, k1, 10)
        tl.store(o_ptr + 4 * i + 0, r0.to(tl.int64))
        tl.store(o_ptr + 4 * i + 1, r1.to(tl.int64))
        tl.store(o_ptr + 4 * i + 2, r2.to(tl.int64))
        tl.store(o_ptr + 4 * i + 3, r3.to(tl.int64))

    n = len(ctrs)
    c = torch.tensor(np.asarray(ctrs, dtype=np.int64).reshape(-1))
    k = torch.tensor(np.asarray(keys, dtype=np.int64).reshape(-1))
    o = torch.zeros(4 * n, dtype=torch.int64)
    kern[(1,)](c, k, o, n)
    return (o.numpy() & 0xFFFFFFFF).reshape(n, 4).astype(np.uint32)


def test_philox_matches_independent_implementation():
    rng = np.random.default_rng(7)
    n = 16
    ctrs = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    keys = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    ctrs[0] = 0
    keys[0] = 0
    ctrs[1] = 2 ** 32 - 1
    keys[1] = 2 ** 32 - 1
    ref = _triton_philox(ctrs, keys)
    for i in range(n):
        got = O.philox4x32_10(ctrs[i].astype(np.uint32), keys[i].astype(np.uint32))
        assert list(got) == list(ref[i]), i


def test_philox_counter_sensitivity():
    a = O.philox4x32_10([0, 0, 0, 0], [1, 2])
    b = O.philox4x32_10([1, 0, 0, 0], [1, 2])
    c = O.philox4x32_10([0, 0, 0, 0], [1, 3])
    assert (a != b).sum() >= 3 and (a != c).sum() >= 3


def test_gaussian_moments():
    # Box-Muller normals keyed by (seed, step, slot): mean 0, variance 1, no correlation
    g = np.array([O.gauss3(12345, 0, step, slot) for step in range(40) for slot in range(500)])
    assert abs(g.mean()) < 0.01
    assert g.var() == pytest.approx(1.0, abs=0.015)
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 0.02
    assert abs(np.corrcoef(g[:, 0], g[:, 2])[0, 1]) < 0.02
    # fourth moment of a normal is 3
    assert (g ** 4).mean() == pytest.approx(3.0, abs=0.1)
    # the draw is a pure function of its key and counter
    assert np.array_equal(O.gauss3(1, 2, 3, 4), O.gauss3(1, 2, 3, 4))
    assert not np.array_equal(O.gauss3(1, 2, 3, 4), O.gauss3(1, 3, 3, 4))
