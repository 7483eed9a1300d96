"""A sampled oracle trajectory for long-run statistical comparisons.

TEST INFRASTRUCTURE ONLY (see the package docstring).  One melt is relaxed
through a list of stages (n, steps, dt), then run for ``prod`` steps of the
last stage with ``K`` double-bridging attempts every ``sweep_every`` steps;
every ``every`` steps after the first ``skip`` production steps it records
<R^2(n)> for n = 0..N-1 and the bond-length and cos(theta) histograms.  The
function takes and returns plain picklable values so that a process pool
(spawn start method) can run one melt per host core.
"""
from __future__ import annotations

import numpy as np


def trajectory(job: dict) -> dict:
    import oracle as O
    x = np.ascontiguousarray(job["x"], dtype=np.float64).copy()
    u = np.ascontiguousarray(job["u"], dtype=np.float64).copy()
    M = x.shape[1]
    pid = np.arange(M, dtype=np.int32)

    def params(n, dt):
        return O.params(job["n_chains"], job["chain_len"], job["box"], job["kappa"], n_exp=n, dt=dt,
                        seed=job["seed"], stream=job["stream"], fene_qmin=job["fene_qmin"])

    step = 0
    for n, k, dt in job["relax"]:
        step = O.run(params(n, dt), x, u, step, k)
    n_prod, dt_prod = job["prod_stage"]
    q = params(n_prod, dt_prod)
    r2, bh, ch = [], [], []
    every, sweep_every = job["every"], job["sweep_every"]
    for i in range(job["prod"] // sweep_every):
        step = O.run(q, x, u, step, sweep_every)
        O.db_sweep(q, x, u, pid, i, job["K"])
        done = (i + 1) * sweep_every
        if done > job["skip"] and done % every == 0:
            r2.append(O.r2n(q, x))
            b, c = O.hist(q, x, job["nbins"])
            bh.append(b)
            ch.append(c)
    return {"r2n": np.array(r2), "bond": np.array(bh), "cos": np.array(ch)}
