"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds input generation only: it computes nothing of the method
(no potential, force, integrator or Monte Carlo arithmetic).  Both sides are
fed the arrays it returns.

Recipe (the initial states of the benchmark melts): every chain is a random
walk with bond length 0.97 sigma whose bond-to-bond angle has
cos(theta) ~ exp(kappa cos(theta)) on [-1, 1] and a uniform azimuth; the first
monomer of each chain is uniform in the periodic cube of side
L = (N_ch N / rho)^(1/3); velocities are Maxwell-Boltzmann at T with the
melt's total momentum removed.  Monomers are placed chain-parallel, one
position index per round; a placement closer than ``d_min`` (0.7 sigma) to any
monomer already placed is redrawn, so that the soft first stage starts without
the overlaps the paper avoids with a tiny first time step (Sec. II.B).
Positions are returned unwrapped, (3, M) float64, chain-major slots c*N + i.
"""
from __future__ import annotations

import math
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


def _cos_theta(rng, kappa, n):
    """Inverse-CDF draw of c on [-1, 1] with density proportional to exp(kappa c)."""
    u = rng.random(n)
    if kappa < 1e-12:
        return 2.0 * u - 1.0
    return 1.0 + np.log(u + (1.0 - u) * math.exp(-2.0 * kappa)) / kappa


def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


_OFFS = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], dtype=np.int64)


def random_walk_melt(n_chains: int, chain_len: int, rho: float, kappa: float, seed: int,
                     bond: float = 0.97, d_min: float = 0.7, T: float = 1.0) -> Melt:
    rng = np.random.default_rng(seed)
    N, M = int(chain_len), int(n_chains) * int(chain_len)
    L = box_side(n_chains, chain_len, rho)
    nc = max(3, int(L // max(d_min, 0.5)))
    h = L / nc
    cap = 12
    grid = np.full((nc * nc * nc, cap), M, dtype=np.int64)      # M = empty sentinel
    fill = np.zeros(nc * nc * nc, dtype=np.int64)
    wpos = np.full((M + 1, 3), np.nan)                          # wrapped positions (+ NaN sentinel)
    pos = np.zeros((M, 3))
    prev_dir = np.zeros((n_chains, 3))
    nxt = np.zeros(n_chains, dtype=np.int64)
    tries = np.zeros(n_chains, dtype=np.int64)

    def cell_xyz(w):
        return np.minimum((w // h).astype(np.int64), nc - 1)

    def lin(c):
        return (c[..., 0] * nc + c[..., 1]) * nc + c[..., 2]

    while True:
        act = np.nonzero(nxt < N)[0]
        if act.size == 0:
            break
        i = nxt[act]
        k = act.size
        cand = np.empty((k, 3))
        first = i == 0
        if first.any():
            cand[first] = rng.random((int(first.sum()), 3)) * L
        grow = ~first
        if grow.any():
            ag = act[grow]
            prev = pos[ag * N + i[grow] - 1]
            second = i[grow] == 1
            d = np.empty((ag.size, 3))
            if second.any():
                d[second] = _unit_vectors(rng, int(second.sum()))
            later = ~second
            if later.any():
                b = prev_dir[ag[later]]
                c = _cos_theta(rng, kappa, int(later.sum()))
                s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
                a = np.where(np.abs(b[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
                e1 = np.cross(b, a)
                e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
                e2 = np.cross(b, e1)
                phi = rng.random(int(later.sum())) * 2.0 * math.pi
                d[later] = c[:, None] * b + s[:, None] * (np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2)
            cand[grow] = prev + bond * d
        w = cand - L * np.floor(cand / L)
        cxyz = cell_xyz(w)
        # clearance against monomers already placed (relaxed for chains that keep failing)
        dmin_eff = d_min * (0.9 ** (tries[act] // 100))
        nb = lin((cxyz[:, None, :] + _OFFS[None, :, :]) % nc)            # (k, 27)
        ids = grid[nb]                                                   # (k, 27, cap)
        dd = wpos[ids] - w[:, None, None, :]
        dd -= L * np.rint(dd / L)
        r2 = np.einsum("abcd,abcd->abc", dd, dd)
        ok = ~(r2 < (dmin_eff ** 2)[:, None, None]).any(axis=(1, 2))
        # clearance among this round's accepted candidates (lower chain index wins)
        okidx = np.nonzero(ok)[0]
        if okidx.size > 1:
            keys = lin(cxyz[okidx])
            order = np.argsort(keys, kind="stable")
            sk = keys[order]
            nbk = nb[okidx]
            for o in range(27):
                lo = np.searchsorted(sk, nbk[:, o], "left")
                hi = np.searchsorted(sk, nbk[:, o], "right")
                for j in range(int((hi - lo).max(initial=0))):
                    has = lo + j < hi
                    a_ = np.nonzero(has)[0]
                    other = order[lo[a_] + j]
                    mine = a_
                    dv = w[okidx[other]] - w[okidx[mine]]
                    dv -= L * np.rint(dv / L)
                    clash = (np.einsum("ab,ab->a", dv, dv) < dmin_eff[okidx[mine]] ** 2) & (other < mine)
                    ok[okidx[mine[clash]]] = False
        acc = np.nonzero(ok)[0]
        rej = np.nonzero(~ok)[0]
        tries[act[rej]] += 1
        if acc.size:
            ch = act[acc]
            slot = ch * N + i[acc]
            pos[slot] = cand[acc]
            wpos[slot] = w[acc]
            keys = lin(cxyz[acc])
            order = np.argsort(keys, kind="stable")
            sk = keys[order]
            first_of = np.searchsorted(sk, sk, "left")
            rank = np.arange(sk.size) - first_of
            where = fill[sk] + rank
            if (where >= cap).any():
                raise RuntimeError("generator cell capacity exceeded")
            grid[sk, where] = slot[order]
            np.add.at(fill, sk, 1)
            not_first = i[acc] > 0
            if not_first.any():
                dprev = cand[acc][not_first] - pos[ch[not_first] * N + i[acc][not_first] - 1]
                prev_dir[ch[not_first]] = dprev / np.linalg.norm(dprev, axis=1, keepdims=True)
            nxt[ch] += 1
            tries[ch] = 0

    v = rng.normal(0.0, math.sqrt(T), size=(M, 3))
    v -= v.mean(axis=0, keepdims=True)
    return Melt(int(n_chains), N, float(L), float(kappa),
                np.ascontiguousarray(pos.T), np.ascontiguousarray(v.T))


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
