"""ctypes binding of ``libkg.so`` (include/kg.h), argument marshalling only.

Every function keeps the C name.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); their data pointers are passed as they are.  PyTorch
supplies device memory (through the ``kg_allocator`` hook, see
:func:`torch_allocator`) and the CUDA stream; all arithmetic runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing or
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkg.so")

KG_OK, KG_ERR_INVALID_ARG, KG_ERR_CUDA, KG_ERR_OOM = 0, 1, 2, 3
KG_ERR_BOND_OVERSTRETCH, KG_ERR_NONFINITE, KG_ERR_CAPACITY, KG_ERR_TIMEOUT, KG_ERR_STATE = 4, 5, 6, 7, 8
KG_FP64, KG_MIXED = 0, 1
KG_FLAG_PAPER_METROPOLIS = 1
KG_FLAG_PERSISTENT = 2

EXPORTS = ["kg_create", "kg_load_config", "kg_get_config", "kg_set_potential_schedule", "kg_step",
           "kg_db_sweep", "kg_db_sweep_k", "kg_observables", "kg_sync", "kg_get_counters",
           "kg_set_counters", "kg_get_nlist", "kg_forces", "kg_profile", "kg_profile_read", "kg_autotune", "kg_kn", "kg_schedule_paper", "kg_destroy",
           "kg_strerror", "kg_r2n_noalloc", "kg_persistent_selftest", "kg_mlp_set_weights", "kg_mlp_get_weights", "kg_mlp_forward",
           "kg_mlp_loss_grad", "kg_mlp_log", "kg_mlp_log_read", "kg_mlp_train", "kg_db_sweep_learned",
           "kg_db_sweep_learned_k", "kg_db_proposal", "kg_msd_reset", "kg_msd", "kg_fit_lk",
           "kg_structure_factor", "kg_pair_distribution", "kg_generate_fr", "kg_primitive_path",
           "kg_entanglement_length"]

KG_MLP_NPARAM = 5825
KG_DB_CAND_MAX = 48


class kg_melt(C.Structure):
    _fields_ = [("n_chains", C.c_int), ("chain_len", C.c_int), ("box", C.c_double), ("kappa", C.c_double)]


class kg_params(C.Structure):
    _fields_ = [("n_melts", C.c_int), ("melts", C.POINTER(kg_melt)), ("T", C.c_double),
                ("gamma", C.c_double), ("R0", C.c_double), ("l0", C.c_double),
                ("db_bond_max", C.c_double), ("r_mc", C.c_double), ("skin", C.c_double),
                ("fene_qmin", C.c_double), ("seed", C.c_ulonglong), ("sort_interval", C.c_int),
                ("block_size", C.c_int), ("precision", C.c_int), ("flags", C.c_int),
                ("threads_per_monomer", C.c_int), ("cell_scale", C.c_double)]


class kg_stage(C.Structure):
    _fields_ = [("n_exp", C.c_double), ("k_fene", C.c_double), ("n_steps", C.c_longlong), ("dt", C.c_double)]


class kg_obs(C.Structure):
    _fields_ = [("e_pair", C.c_double), ("e_bond", C.c_double), ("e_angle", C.c_double),
                ("e_kin", C.c_double), ("virial", C.c_double), ("temperature", C.c_double),
                ("pressure", C.c_double), ("step", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class kg_tuning(C.Structure):
    _fields_ = [("skin", C.c_double), ("block_size", C.c_int), ("ms_per_step", C.c_double), ("trials", C.c_int),
                ("threads_per_monomer", C.c_int), ("cell_scale", C.c_double)]


class kg_ppa_params(C.Structure):
    _fields_ = [("n_iter", C.c_longlong), ("dt", C.c_double), ("gamma", C.c_double), ("skin", C.c_double),
                ("k_fene", C.c_double), ("precision", C.c_int)]


class kg_ppa_result(C.Structure):
    _fields_ = [("lpp_mean", C.c_double), ("fmax", C.c_double), ("builds", C.c_longlong),
                ("mean_neighbours", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class kg_db_stats(C.Structure):
    _fields_ = [("attempted", C.c_longlong), ("empty", C.c_longlong), ("accepted", C.c_longlong),
                ("reevaluated", C.c_longlong), ("sweep", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class kg_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    i, d, p, ll = C.c_int, C.c_double, C.c_void_p, C.c_longlong
    sig = {
        "kg_create": (i, [p, C.POINTER(kg_params), i, p, p]),
        "kg_load_config": (i, [p, i, p, p, p]),
        "kg_get_config": (i, [p, i, p, p, p]),
        "kg_set_potential_schedule": (i, [p, C.POINTER(kg_stage), i]),
        "kg_step": (i, [p, ll]),
        "kg_db_sweep": (i, [p, d, C.POINTER(kg_db_stats)]),
        "kg_db_sweep_k": (i, [p, p, C.POINTER(kg_db_stats)]),
        "kg_observables": (i, [p, i, C.POINTER(kg_obs), p, p, p, i]),
        "kg_sync": (i, [p]),
        "kg_get_counters": (i, [p, C.POINTER(ll), C.POINTER(ll)]),
        "kg_set_counters": (i, [p, ll, ll]),
        "kg_get_nlist": (i, [p, i, p, p, ll, C.POINTER(ll)]),
        "kg_forces": (i, [p, i, p, p]),
        "kg_profile": (i, [p, i]),
        "kg_autotune": (i, [C.POINTER(kg_params), p, p, C.POINTER(kg_stage), i, i, p, p, C.POINTER(kg_tuning)]),
        "kg_profile_read": (i, [p, C.POINTER(d), C.POINTER(ll), C.POINTER(ll)]),
        "kg_kn": (d, [d, d, d]),
        "kg_schedule_paper": (i, [d, i, d, d, C.POINTER(kg_stage)]),
        "kg_destroy": (None, [p]),
        "kg_strerror": (C.c_char_p, [i]),
        "kg_r2n_noalloc": (i, [p, ll, i, i, p, p]),
        "kg_persistent_selftest": (i, [p, i, C.c_uint]),
        "kg_msd_reset": (i, [p, i]),
        "kg_msd": (i, [p, i, C.POINTER(d)]),
        "kg_fit_lk": (i, [p, i, d, i, i, C.POINTER(d)]),
        "kg_structure_factor": (i, [p, i, p, i, p]),
        "kg_generate_fr": (i, [i, i, d, d, d, C.c_ulonglong, i, p, C.POINTER(d), C.POINTER(i)]),
        "kg_pair_distribution": (i, [p, i, d, i, p]),
        "kg_primitive_path": (i, [p, i, C.POINTER(kg_ppa_params), p, p, C.POINTER(kg_ppa_result)]),
        "kg_entanglement_length": (i, [d, i, d, d, C.POINTER(d), C.POINTER(d)]),
        "kg_mlp_set_weights": (i, [p, p]),
        "kg_mlp_get_weights": (i, [p, p]),
        "kg_mlp_forward": (i, [p, p, ll, p]),
        "kg_mlp_loss_grad": (i, [p, p, p, ll, C.POINTER(d), p]),
        "kg_mlp_log": (i, [p, ll]),
        "kg_mlp_log_read": (i, [p, p, p, ll, C.POINTER(ll)]),
        "kg_mlp_train": (i, [p, i, i, d, C.POINTER(d)]),
        "kg_db_sweep_learned": (i, [p, d, d, C.POINTER(kg_db_stats)]),
        "kg_db_sweep_learned_k": (i, [p, p, d, C.POINTER(kg_db_stats)]),
        "kg_db_proposal": (i, [p, i, i, i, d, C.POINTER(i), p, p, p, p, p, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


class KGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().kg_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def _check(st, where):
    if st != KG_OK:
        raise KGError(st, where)
    return st


def ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def torch_allocator():
    """A kg_allocator whose buffers are torch CUDA tensors (kept alive here)."""
    import torch
    keep = {}

    def _alloc(nbytes, user):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        keep[t.data_ptr()] = t
        return t.data_ptr()

    def _free(p, user):
        keep.pop(int(p or 0), None)

    a = kg_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    a._keep = (keep, _alloc, _free)
    return a


# ---- the C entry points, same names ----

# allocators (and their ctypes callback trampolines) must outlive their context
_ALLOCATORS = {}


def kg_create(params: kg_params, device: int = 0, stream: int | None = None, allocator=None):
    ctx = C.c_void_p()
    _check(load().kg_create(C.byref(ctx), C.byref(params), int(device), stream,
                            C.byref(allocator) if allocator is not None else None), "kg_create")
    if allocator is not None:
        _ALLOCATORS[ctx.value] = allocator
    return ctx


def kg_load_config(ctx, melt, x, v=None, pid=None):
    return _check(load().kg_load_config(ctx, int(melt), ptr(x), ptr(v), ptr(pid)), "kg_load_config")


def kg_get_config(ctx, melt, x=None, v=None, pid=None):
    return _check(load().kg_get_config(ctx, int(melt), ptr(x), ptr(v), ptr(pid)), "kg_get_config")


def kg_set_potential_schedule(ctx, stages):
    arr = (kg_stage * len(stages))(*stages)
    return _check(load().kg_set_potential_schedule(ctx, arr, len(stages)), "kg_set_potential_schedule")


def kg_step(ctx, n_steps):
    return _check(load().kg_step(ctx, int(n_steps)), "kg_step")


def kg_db_sweep(ctx, attempts_per_monomer=-1.0):
    st = kg_db_stats()
    _check(load().kg_db_sweep(ctx, float(attempts_per_monomer), C.byref(st)), "kg_db_sweep")
    return st


def kg_db_sweep_k(ctx, attempts):
    a = np.ascontiguousarray(np.asarray(attempts, dtype=np.int64))
    st = kg_db_stats()
    _check(load().kg_db_sweep_k(ctx, a.ctypes.data, C.byref(st)), "kg_db_sweep_k")
    return st


def kg_msd_reset(ctx, melt):
    return _check(load().kg_msd_reset(ctx, int(melt)), "kg_msd_reset")


def kg_fit_lk(r2n, l0=0.960897, n_lo=0, n_hi=0):
    """Kuhn length of Eq. 14 fitted to <R^2(n)> (r2n[n], r2n[0] unused)."""
    r = np.ascontiguousarray(r2n, dtype=np.float64)
    out = C.c_double()
    _check(load().kg_fit_lk(ptr(r), len(r), float(l0), int(n_lo), int(n_hi), C.byref(out)), "kg_fit_lk")
    return out.value


def kg_generate_fr(n_chains, chain_len, box, kappa, seed, l0=0.960897, max_attempts=100):
    """(x (3, M), fitted l_K, attempts) of the paper's FR-chain initial state."""
    x = np.zeros((3, int(n_chains) * int(chain_len)))
    lk = C.c_double()
    att = C.c_int()
    _check(load().kg_generate_fr(int(n_chains), int(chain_len), float(box), float(kappa), float(l0), int(seed),
                                 int(max_attempts), ptr(x), C.byref(lk), C.byref(att)), "kg_generate_fr")
    return x, lk.value, att.value


def kg_structure_factor(ctx, melt, hkl):
    """S(q) for integer triples hkl (nq, 3): q = 2 pi (h, k, l) / L."""
    h = np.ascontiguousarray(hkl, dtype=np.int32).reshape(-1, 3)
    S = np.zeros(len(h))
    _check(load().kg_structure_factor(ctx, int(melt), ptr(h), len(h), ptr(S)), "kg_structure_factor")
    return S


def kg_pair_distribution(ctx, melt, r_max, nbins):
    g = np.zeros(int(nbins))
    _check(load().kg_pair_distribution(ctx, int(melt), float(r_max), int(nbins), ptr(g)), "kg_pair_distribution")
    return g


def kg_primitive_path(ctx, melt, n_chains, n_iter, dt=0.005, gamma=1.0, skin=0.3, k_fene=0.0, x_out=None,
                      precision=KG_MIXED):
    """Primitive-path analysis of a melt: returns (per-chain L_pp, result dict
    with lpp_mean, fmax, builds); x_out (3, M) float64 receives the minimised
    positions when given."""
    pp = kg_ppa_params(int(n_iter), float(dt), float(gamma), float(skin), float(k_fene), int(precision))
    lpp = np.zeros(int(n_chains))
    res = kg_ppa_result()
    _check(load().kg_primitive_path(ctx, int(melt), C.byref(pp), ptr(lpp), ptr(x_out), C.byref(res)),
           "kg_primitive_path")
    return lpp, res.as_dict()


def kg_entanglement_length(lpp_mean, chain_len, l_k, l0=0.960897):
    """(N_eK, N_e) from the mean primitive-path length (Eq. 22)."""
    n_ek, n_e = C.c_double(), C.c_double()
    _check(load().kg_entanglement_length(float(lpp_mean), int(chain_len), float(l0), float(l_k), C.byref(n_ek),
                                         C.byref(n_e)), "kg_entanglement_length")
    return n_ek.value, n_e.value


def kg_msd(ctx, melt):
    out = C.c_double()
    _check(load().kg_msd(ctx, int(melt), C.byref(out)), "kg_msd")
    return out.value


def kg_observables(ctx, melt, r2n=None, bond_hist=None, cos_hist=None, n_bins=0):
    ob = kg_obs()
    _check(load().kg_observables(ctx, int(melt), C.byref(ob), ptr(r2n), ptr(bond_hist), ptr(cos_hist),
                                 int(n_bins)), "kg_observables")
    return ob


def kg_sync(ctx):
    return load().kg_sync(ctx)


def kg_get_counters(ctx):
    s, w = C.c_longlong(), C.c_longlong()
    _check(load().kg_get_counters(ctx, C.byref(s), C.byref(w)), "kg_get_counters")
    return s.value, w.value


def kg_set_counters(ctx, step, sweep):
    return _check(load().kg_set_counters(ctx, int(step), int(sweep)), "kg_set_counters")


def kg_get_nlist(ctx, melt, M, cap=None):
    cap = cap or M * 96
    offs = np.zeros(M + 1, dtype=np.int32)
    nbr = np.zeros(cap, dtype=np.int32)
    tot = C.c_longlong()
    _check(load().kg_get_nlist(ctx, int(melt), ptr(offs), ptr(nbr), cap, C.byref(tot)), "kg_get_nlist")
    return offs, nbr[:tot.value].copy()


def kg_forces(ctx, melt, F=None, e4=None):
    return _check(load().kg_forces(ctx, int(melt), ptr(F), ptr(e4)), "kg_forces")


def kg_profile(ctx, enable):
    return _check(load().kg_profile(ctx, int(bool(enable))), "kg_profile")


def kg_profile_read(ctx):
    ms, n, launches = C.c_double(), C.c_longlong(), C.c_longlong()
    _check(load().kg_profile_read(ctx, C.byref(ms), C.byref(n), C.byref(launches)), "kg_profile_read")
    return ms.value, n.value, launches.value


def kg_autotune(params, xs, vs, stage, trial_steps=40, device=0, stream=None, allocator=None):
    """xs, vs: one (3, M) array per melt (vs may be None)."""
    xp = (C.c_void_p * len(xs))(*[ptr(a) for a in xs])
    vp = (C.c_void_p * len(vs))(*[ptr(a) for a in vs]) if vs is not None else None
    best = kg_tuning()
    _check(load().kg_autotune(C.byref(params), xp, vp, C.byref(stage), int(trial_steps), int(device), stream,
                              C.byref(allocator) if allocator is not None else None, C.byref(best)),
           "kg_autotune")
    return best


def kg_kn(n, R0=1.5, l0=0.960897):
    return load().kg_kn(float(n), float(R0), float(l0))


def kg_schedule_paper(kappa, chain_len, dt, scale=1.0):
    out = (kg_stage * 12)()
    _check(load().kg_schedule_paper(float(kappa), int(chain_len), float(dt), float(scale), out),
           "kg_schedule_paper")
    return list(out)


def kg_destroy(ctx):
    load().kg_destroy(ctx)
    _ALLOCATORS.pop(ctx.value, None)


def kg_persistent_selftest(ctx, skip_block, spin):
    """Status of a two-step persistent launch whose block `skip_block` skips the
    grid barrier (see kg.h); returned, not raised."""
    return load().kg_persistent_selftest(ctx, int(skip_block), int(spin))


def kg_r2n_noalloc(x, stride, n_chains, chain_len, out, stream=None):
    return _check(load().kg_r2n_noalloc(ptr(x), int(stride), int(n_chains), int(chain_len), ptr(out), stream),
                  "kg_r2n_noalloc")


def kg_strerror(status):
    return load().kg_strerror(int(status)).decode()


# ---- convenience: parameter construction ----

def make_params(melts, precision=KG_MIXED, seed=1, T=1.0, gamma=1.0, R0=1.5, l0=0.960897, db_bond_max=1.3,
                r_mc=1e-3, skin=0.3, flags=0, fene_qmin=0.0, sort_interval=0, block_size=0,
                threads_per_monomer=0, cell_scale=0.0):
    """melts: iterable of (n_chains, chain_len, box, kappa)."""
    arr = (kg_melt * len(melts))(*[kg_melt(int(a), int(b), float(c), float(d)) for a, b, c, d in melts])
    p = kg_params(len(melts), arr, T, gamma, R0, l0, db_bond_max, r_mc, skin, float(fene_qmin), int(seed),
                  int(sort_interval), int(block_size), int(precision), int(flags), int(threads_per_monomer),
                  float(cell_scale))
    p._keep = arr
    return p


def stage(n_exp, n_steps, dt, k_fene=-1.0):
    return kg_stage(float(n_exp), float(k_fene), int(n_steps), float(dt))


# ---- learned proposal ----

def _host_f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


def kg_mlp_set_weights(ctx, w):
    w = _host_f64(w, (KG_MLP_NPARAM,))
    return _check(load().kg_mlp_set_weights(ctx, ptr(w)), "kg_mlp_set_weights")


def kg_mlp_get_weights(ctx):
    w = np.zeros(KG_MLP_NPARAM)
    _check(load().kg_mlp_get_weights(ctx, ptr(w)), "kg_mlp_get_weights")
    return w


def kg_mlp_forward(ctx, features):
    f = _host_f64(features)
    n = f.shape[0]
    assert f.shape == (n, 24)
    out = np.zeros(n)
    _check(load().kg_mlp_forward(ctx, ptr(f), n, ptr(out)), "kg_mlp_forward")
    return out


def kg_mlp_loss_grad(ctx, features, targets):
    f = _host_f64(features)
    t = _host_f64(targets, (f.shape[0],))
    loss = C.c_double()
    g = np.zeros(KG_MLP_NPARAM)
    _check(load().kg_mlp_loss_grad(ctx, ptr(f), ptr(t), f.shape[0], C.byref(loss), ptr(g)), "kg_mlp_loss_grad")
    return loss.value, g


def kg_mlp_log(ctx, capacity):
    return _check(load().kg_mlp_log(ctx, int(capacity)), "kg_mlp_log")


def kg_mlp_log_read(ctx, cap):
    f = np.zeros((max(cap, 1), 24))
    t = np.zeros(max(cap, 1))
    n = C.c_longlong()
    _check(load().kg_mlp_log_read(ctx, ptr(f), ptr(t), int(cap), C.byref(n)), "kg_mlp_log_read")
    return f[:n.value], t[:n.value]


def kg_mlp_train(ctx, iters, batch, lr):
    loss = C.c_double()
    _check(load().kg_mlp_train(ctx, int(iters), int(batch), float(lr), C.byref(loss)), "kg_mlp_train")
    return loss.value


def kg_db_sweep_learned(ctx, attempts_per_monomer=-1.0, lam=0.1):
    st = kg_db_stats()
    _check(load().kg_db_sweep_learned(ctx, float(attempts_per_monomer), float(lam), C.byref(st)),
           "kg_db_sweep_learned")
    return st


def kg_db_sweep_learned_k(ctx, attempts, lam=0.1):
    a = np.ascontiguousarray(attempts, dtype=np.int64)
    st = kg_db_stats()
    _check(load().kg_db_sweep_learned_k(ctx, ptr(a), float(lam), C.byref(st)), "kg_db_sweep_learned_k")
    return st


def kg_db_proposal(ctx, melt, chain, bond, lam=0.1):
    """dict of the bond's candidate list: kind, chain, bond, features, logits, prob."""
    n = C.c_int()
    cap = KG_DB_CAND_MAX
    kind, pc, pb = (np.zeros(cap, dtype=np.int32) for _ in range(3))
    f = np.zeros((cap, 24))
    s, pi = np.zeros(cap), np.zeros(cap)
    _check(load().kg_db_proposal(ctx, int(melt), int(chain), int(bond), float(lam), C.byref(n), ptr(kind),
                                 ptr(pc), ptr(pb), ptr(f), ptr(s), ptr(pi)), "kg_db_proposal")
    k = n.value
    return {"n": k, "kind": kind[:k], "chain": pc[:k], "bond": pb[:k], "features": f[:k], "logits": s[:k],
            "prob": pi[:k]}
