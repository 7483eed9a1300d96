"""FP64 CPU oracle for the core-softened DBH method (arXiv:2109.11001).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product library never
loads it, and it shares no code with the CUDA library: the C source
``kg_oracle.c`` is compiled on its own with ``-ffp-contract=off``.

The Python side is argument marshalling over ctypes plus the schedule
arithmetic in :mod:`oracle.schedule`.  Arrays follow the oracle's layout:
positions and velocities ``(3, M)`` float64 (SoA), particle ids ``(M,)`` int32,
slot ``s = c*N + i``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kg_oracle.c")
_LIB = os.path.join(_HERE, "libkg_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP contraction off)."""
    hdr = os.path.join(_HERE, "kg_oracle.h")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("n_chains", C.c_int), ("chain_len", C.c_int), ("box", C.c_double),
                ("kappa", C.c_double), ("n_exp", C.c_double), ("k_fene", C.c_double),
                ("R0", C.c_double), ("T", C.c_double), ("gamma", C.c_double),
                ("dt", C.c_double), ("db_bond_max", C.c_double), ("seed", C.c_ulonglong),
                ("stream", C.c_uint), ("paper_metropolis", C.c_int), ("fene_qmin", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, ll, p = C.c_double, C.c_int, C.c_longlong, C.c_void_p
        sig = {
            "orc_rc": (d, []), "orc_mlj_u": (d, [d, d]), "orc_mlj_du": (d, [d, d]),
            "orc_kn": (d, [d, d, d]), "orc_fene_u": (d, [d, d, d]), "orc_fene_du": (d, [d, d, d]),
            "orc_fene_reg_u": (d, [d, d, d, d]), "orc_fene_reg_du": (d, [d, d, d, d]),
            "orc_philox4x32_10": (None, [p, p, p]),
            "orc_gauss3": (None, [C.c_ulonglong, C.c_uint, ll, C.c_uint, p]),
            "orc_nlist": (ll, [p, p, d, i, p, p, ll]),
            "orc_forces": (i, [p, p, p, p]),
            "orc_run": (i, [p, p, p, p, ll]),
            "orc_observe": (i, [p, p, p, ll, p]),
            "orc_r2n": (None, [p, p, p]),
            "orc_hist": (None, [p, p, i, p, p]),
            "orc_db_sweep": (i, [p, p, p, p, ll, ll, p]),
            "orc_db_partners": (i, [p, p, p, i, i]),
            "orc_db_candidates": (i, [p, p, p, i, i, p, p, p, i]),
            "orc_topo_energy": (d, [p, p]),
            "orc_mlp_forward": (d, [p, p]),
            "orc_move_features": (None, [p, p, i, i, i, i, i, p]),
            "orc_db_sweep_learned": (i, [p, p, p, p, ll, ll, p, d, i, p, p, p, ll, p]),
            "orc_bf16_round": (d, [d]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype, f.argtypes = res, args
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def params(n_chains, chain_len, box, kappa, n_exp=12.0, k_fene=None, R0=1.5, T=1.0,
           gamma=1.0, dt=0.01, db_bond_max=1.3, seed=0, stream=0, paper_metropolis=False,
           l0=0.960897, fene_qmin=0.0) -> Params:
    if k_fene is None:
        k_fene = kn(n_exp, R0, l0)
    return Params(int(n_chains), int(chain_len), float(box), float(kappa), float(n_exp),
                  float(k_fene), float(R0), float(T), float(gamma), float(dt),
                  float(db_bond_max), int(seed), int(stream), int(bool(paper_metropolis)),
                  float(fene_qmin))


class OracleError(RuntimeError):
    pass


_STATUS = {1: "bond overstretched (r >= R0)", 2: "non-finite force", 3: "capacity", 4: "bad argument"}


def _check(st):
    if st != 0:
        raise OracleError(_STATUS.get(st, f"status {st}"))


def rc() -> float:
    return lib().orc_rc()


def mlj_u(n, r):
    return lib().orc_mlj_u(float(n), float(r))


def mlj_du(n, r):
    return lib().orc_mlj_du(float(n), float(r))


def kn(n, R0=1.5, l0=0.960897):
    return lib().orc_kn(float(n), float(R0), float(l0))


def fene_u(k, R0, r):
    return lib().orc_fene_u(float(k), float(R0), float(r))


def fene_du(k, R0, r):
    return lib().orc_fene_du(float(k), float(R0), float(r))


def fene_reg_u(k, R0, qmin, r):
    return lib().orc_fene_reg_u(float(k), float(R0), float(qmin), float(r))


def fene_reg_du(k, R0, qmin, r):
    return lib().orc_fene_reg_du(float(k), float(R0), float(qmin), float(r))


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def gauss3(seed, stream, step, slot):
    g = np.zeros(3)
    lib().orc_gauss3(int(seed), int(stream), int(step), int(slot), _ptr(g))
    return g


def nlist(p: Params, x: np.ndarray, rlist: float, use_cells=True, cap=None):
    """Return (offs, nbr) CSR arrays; nbr sorted ascending per particle."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    M = p.n_chains * p.chain_len
    cap = cap or M * 96
    offs = np.zeros(M + 1, dtype=np.int32)
    nbr = np.zeros(cap, dtype=np.int32)
    tot = lib().orc_nlist(C.byref(p), _ptr(x), float(rlist), int(use_cells), _ptr(offs), _ptr(nbr), cap)
    if tot < 0:
        raise OracleError("neighbour capacity")
    return offs, nbr[:tot].copy()


def forces(p: Params, x: np.ndarray):
    """Conservative forces (3, M) and energies [pair, bond, angle, virial]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    F = np.zeros_like(x)
    e = np.zeros(4)
    _check(lib().orc_forces(C.byref(p), _ptr(x), _ptr(F), _ptr(e)))
    return F, e


def run(p: Params, x: np.ndarray, u: np.ndarray, step: int, nsteps: int) -> int:
    """Advance (x, u) in place by nsteps; returns the new step counter."""
    assert x.flags.c_contiguous and u.flags.c_contiguous and x.dtype == np.float64
    st = C.c_longlong(step)
    _check(lib().orc_run(C.byref(p), _ptr(x), _ptr(u), C.byref(st), int(nsteps)))
    return st.value


def observe(p: Params, x, u, step):
    """dict of integer-time observables."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(7)
    _check(lib().orc_observe(C.byref(p), _ptr(x), _ptr(u), int(step), _ptr(out)))
    keys = ["e_pair", "e_bond", "e_angle", "e_kin", "virial", "temperature", "pressure"]
    return dict(zip(keys, out.tolist()))


def r2n(p: Params, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(p.chain_len)
    lib().orc_r2n(C.byref(p), _ptr(x), _ptr(out))
    return out


def hist(p: Params, x, nbins):
    x = np.ascontiguousarray(x, dtype=np.float64)
    bh, ch = np.zeros(nbins), np.zeros(nbins)
    lib().orc_hist(C.byref(p), _ptr(x), int(nbins), _ptr(bh), _ptr(ch))
    return bh, ch


def db_sweep(p: Params, x, u, pid, sweep: int, K: int):
    """K double-bridging attempts in order; arrays permuted in place.
    Returns (attempted, empty, accepted)."""
    assert x.flags.c_contiguous and u.flags.c_contiguous and pid.dtype == np.int32
    stats = np.zeros(3, dtype=np.int64)
    _check(lib().orc_db_sweep(C.byref(p), _ptr(x), _ptr(u), _ptr(pid), int(sweep), int(K), _ptr(stats)))
    return tuple(int(s) for s in stats)


def db_partners(p: Params, x, pid, chain: int, bond: int) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64)
    pid = np.ascontiguousarray(pid, dtype=np.int32)
    return lib().orc_db_partners(C.byref(p), _ptr(x), _ptr(pid), int(chain), int(bond))


def db_candidates(p: Params, x, pid, chain: int, bond: int):
    """partner list of bond (chain, bond) in proposal order: list of (kind, d, q)"""
    x = np.ascontiguousarray(x, dtype=np.float64)
    pid = np.ascontiguousarray(pid, dtype=np.int32)
    cap = 2 * p.n_chains
    k, d, q = (np.zeros(cap, dtype=np.int32) for _ in range(3))
    n = lib().orc_db_candidates(C.byref(p), _ptr(x), _ptr(pid), int(chain), int(bond), _ptr(k), _ptr(d), _ptr(q), cap)
    return [(int(k[j]), int(d[j]), int(q[j])) for j in range(n)]


def topo_energy(p: Params, x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_topo_energy(C.byref(p), _ptr(x))


MLP_NPARAM = 64 * 24 + 64 + 64 * 64 + 64 + 64 + 1


def mlp_forward(w, f):
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().orc_mlp_forward(_ptr(w), _ptr(f))


def move_features(p: Params, x, c, b, kind, d, q):
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.zeros(24)
    lib().orc_move_features(C.byref(p), _ptr(x), int(c), int(b), int(kind), int(d), int(q), _ptr(f))
    return f


def bf16_round(v):
    return lib().orc_bf16_round(float(v))


def db_sweep_learned(p: Params, x, u, pid, sweep: int, K: int, w, lam: float, log_cap: int = 0,
                     bf16_inputs: bool = False):
    """Sweep with the learned proposal; returns (stats, log features, log targets)."""
    assert x.flags.c_contiguous and u.flags.c_contiguous and pid.dtype == np.int32
    w = np.ascontiguousarray(w, dtype=np.float64)
    stats = np.zeros(3, dtype=np.int64)
    lf = np.zeros((max(log_cap, 1), 24))
    lt = np.zeros(max(log_cap, 1))
    n = C.c_longlong(0)
    _check(lib().orc_db_sweep_learned(C.byref(p), _ptr(x), _ptr(u), _ptr(pid), int(sweep), int(K), _ptr(w),
                                      float(lam), int(bool(bf16_inputs)), _ptr(stats), _ptr(lf) if log_cap else None,
                                      _ptr(lt) if log_cap else None, int(log_cap), C.byref(n)))
    return tuple(int(v) for v in stats), lf[:n.value], lt[:n.value]
