"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds input generation only: it computes nothing of the method
(no potential, force, integrator or Monte Carlo arithmetic).  Both sides are
fed the arrays it returns.

Recipe (the initial states of the benchmark melts): every chain is a random
walk with bond length 0.97 sigma whose bond-to-bond angle has
cos(theta) ~ exp(kappa cos(theta)) on [-1, 1] and a uniform azimuth; the first
monomer of each chain is uniform in the periodic cube of side
L = (N_ch N / rho)^(1/3); velocities are Maxwell-Boltzmann at T with the
melt's total momentum removed.  Monomers are placed round-robin over chains,
one position index per round; a placement closer than ``d_min`` (0.7 sigma) to
any monomer already placed is redrawn, so that the soft first stage starts
without the overlaps the paper avoids with a tiny first time step (Sec. II.B).
Positions are returned unwrapped, (3, M) float64, chain-major slots c*N + i.
The generator itself is plain C (``gen.c``), compiled with gcc on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

# per-configuration seeds: 2109110010 + config index (melt m of the batched scan adds 100 m)
SEED_BASE = 2109110010


@dataclass
class Melt:
    n_chains: int
    chain_len: int
    box: float
    kappa: float
    x: np.ndarray      # (3, M) unwrapped positions
    v: np.ndarray      # (3, M) velocities

    @property
    def M(self) -> int:
        return self.n_chains * self.chain_len


def box_side(n_chains: int, chain_len: int, rho: float) -> float:
    return (n_chains * chain_len / rho) ** (1.0 / 3.0)


_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libkg_inputs.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator (plain C, gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        f = _lib.kgi_random_walk_melt
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_ulonglong, C.c_double, C.c_double,
                      C.c_double, C.c_void_p, C.c_void_p]
    return _lib


def random_walk_melt(n_chains: int, chain_len: int, rho: float, kappa: float, seed: int,
                     bond: float = 0.97, d_min: float = 0.7, T: float = 1.0) -> Melt:
    M = int(n_chains) * int(chain_len)
    L = box_side(n_chains, chain_len, rho)
    x = np.zeros((3, M))
    v = np.zeros((3, M))
    rc = _load().kgi_random_walk_melt(int(n_chains), int(chain_len), float(L), float(kappa), int(seed),
                                      float(bond), float(d_min), float(T), x.ctypes.data, v.ctypes.data)
    if rc:
        raise MemoryError("generator allocation failed")
    return Melt(int(n_chains), int(chain_len), float(L), float(kappa), x, v)


def config(index: int, melt: int = 0) -> dict:
    """Named workloads (n_chains, chain_len, kappa) with their seeds."""
    table = {
        1: dict(n_chains=20, chain_len=50, kappa=1.5),
        2: dict(n_chains=200, chain_len=400, kappa=2.5),
        4: dict(n_chains=500, chain_len=800, kappa=3.0),
        5: dict(n_chains=1000, chain_len=1600, kappa=3.5),
    }
    if index == 3:
        scan = [(0.0, 100, 200), (0.5, 200, 150), (1.0, 400, 100), (1.5, 800, 50),
                (2.0, 100, 250), (2.5, 200, 250), (3.0, 400, 200), (3.5, 800, 250)]
        k, N, nch = scan[melt]
        d = dict(n_chains=nch, chain_len=N, kappa=k)
    else:
        d = dict(table[index])
    d["seed"] = SEED_BASE + index + 100 * melt
    d["rho"] = 0.85
    return d


def make(index: int, melt: int = 0, **over) -> Melt:
    d = config(index, melt)
    d.update(over)
    return random_walk_melt(d["n_chains"], d["chain_len"], d["rho"], d["kappa"], d["seed"])


def hooked_pair(D: float = 1.2, lift: float = 0.6, box: float = 10.0) -> Melt:
    """Two three-monomer chains hooked around each other, for primitive-path
    tests: chain A has its ends at c -+ (D, 0, 0) and its middle monomer at
    c + (0, lift, 0); chain B has its ends at c -+ (0, 0, D) and its middle at
    c - (0, lift, 0); c is the box centre.  Velocities zero."""
    c = 0.5 * box
    pts = [(c - D, c, c), (c, c + lift, c), (c + D, c, c),
           (c, c, c - D), (c, c - lift, c), (c, c, c + D)]
    x = np.array(pts, dtype=np.float64).T.copy()
    return Melt(2, 3, float(box), 0.0, x, np.zeros_like(x))
