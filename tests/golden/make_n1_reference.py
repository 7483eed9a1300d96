"""Writes n1_reference.json: the oracle's chain statistics at the end of the
scaled paper protocol, and after a long WCA continuation, for 16 melts of 20
chains x N = 50 at kappa = 1.5 (rho = 0.85).

Calls only the oracle (and kg_inputs for the seeded initial states).  The
protocol -- a dt ramp in the n = 2 stage, then the twelve stages of the
paper's schedule (Eqs. 16-20, scheme 1 for kappa <= 2.5) scaled by SCALE at
dt = tau/125 (Sec. II.B), double-bridging sweeps every SWEEP_EVERY steps with
the paper's rate R_MC = 1e-3 per monomer per tau (fractional attempts carried
to the next sweep) -- is stored in the JSON next to the results, so the GPU
side replays exactly the same protocol.

Usage: python tests/golden/make_n1_reference.py [processes]
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SETTINGS = dict(
    n_melts=16, n_chains=20, chain_len=50, kappa=1.5, rho=0.85, seed=11,
    ramp=[[2.0, 2000, 0.001], [2.0, 2000, 0.003], [2.0, 2000, 0.005]],
    dt=0.008, scale=0.2, sweep_every=50, r_mc=1e-3, fene_qmin=0.01,
    window_frac=0.4, sample_every=500, long_steps=100000,
)


def stages(S=SETTINGS):
    """The protocol's stages as (n, steps, dt)."""
    from oracle import schedule
    dur = schedule.stage_durations(S["kappa"], S["chain_len"])
    paper = [(n, int(round(S["scale"] * t / S["dt"])), S["dt"]) for n, t in zip(schedule.XI, dur)]
    return [tuple(r) for r in S["ramp"]] + paper


def melt_seed(i, S=SETTINGS):
    import kg_inputs as KI
    return KI.config(1)["seed"] + 100 * i


def _run(i):
    import kg_inputs as KI
    import oracle as O
    S = SETTINGS
    m = KI.random_walk_melt(S["n_chains"], S["chain_len"], S["rho"], S["kappa"], melt_seed(i))
    x, u = m.x.copy(), m.v.copy()
    pid = np.arange(m.M, dtype=np.int32)
    st = sweep = 0
    carry = 0.0
    plan = stages()
    last = len(plan) - 1
    win, lng = [], []
    for si, (n, k, dt) in enumerate(plan + [(12.0, S["long_steps"], S["dt"])]):
        p = O.params(m.n_chains, m.chain_len, m.box, m.kappa, n_exp=n, dt=dt, seed=S["seed"], stream=i,
                     fene_qmin=S["fene_qmin"])
        done = 0
        while done < k:
            q = min(S["sweep_every"], k - done)
            st = O.run(p, x, u, st, q)
            done += q
            want = S["r_mc"] * m.M * q * dt + carry
            K = int(np.floor(want))
            carry = want - K
            O.db_sweep(p, x, u, pid, sweep, K)
            sweep += 1
            if done % S["sample_every"] == 0:
                if si == last and done > (1 - S["window_frac"]) * k:
                    win.append(O.r2n(p, x))
                elif si == last + 1:
                    lng.append(O.r2n(p, x))
    return np.mean(win, axis=0), np.mean(lng, axis=0), len(win), len(lng)


def r2_mid(r2n, N):
    n = np.arange(N // 4, N // 2 + 1)
    return float(np.mean(r2n[n] / n))


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    S = SETTINGS
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_run, range(S["n_melts"]), chunksize=1)
    N = S["chain_len"]
    win = np.array([r[0] for r in res])
    lng = np.array([r[1] for r in res])
    mid_w = np.array([r2_mid(r, N) for r in win])
    mid_l = np.array([r2_mid(r, N) for r in lng])
    out = {
        "what": "oracle <R^2(n)> per melt: time average over the last window_frac of the final (n = 12) stage "
                "of the scaled paper protocol, and over a WCA continuation of long_steps steps",
        "made_by": "tests/golden/make_n1_reference.py (oracle only)",
        "settings": S,
        "stages": [list(s) for s in stages()],
        "samples": [int(res[0][2]), int(res[0][3])],
        "r2n_protocol_end": win.tolist(),
        "r2n_long_run": lng.tolist(),
        "r2_mid_protocol_end": {"mean": float(mid_w.mean()), "sem": float(mid_w.std(ddof=1) / np.sqrt(len(mid_w)))},
        "r2_mid_long_run": {"mean": float(mid_l.mean()), "sem": float(mid_l.std(ddof=1) / np.sqrt(len(mid_l)))},
        "cpu_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, "n1_reference.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("r2_mid_protocol_end", "r2_mid_long_run", "samples", "cpu_seconds")}))


if __name__ == "__main__":
    main()
