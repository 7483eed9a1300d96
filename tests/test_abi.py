"""The C ABI: the library builds for sm_103a, loads without a GPU, and exports
every entry point include/kg.h declares; the Python binding carries the same
names.  No compute call is made here."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "kg.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2109_11001_gb300 import build as B
    return ctypes.CDLL(B.build())


def test_header_declares_the_boundary():
    names = declared()
    for n in ("kg_create", "kg_load_config", "kg_step", "kg_db_sweep", "kg_set_potential_schedule",
              "kg_observables", "kg_destroy", "kg_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared():
        assert hasattr(lib, n), n


def test_binding_has_the_same_names():
    import paper_2109_11001_gb300 as kg
    assert sorted(kg.EXPORTS) == declared()
    for n in declared():
        assert callable(getattr(kg, n)), n


def test_host_helpers_without_gpu(lib):
    import paper_2109_11001_gb300 as kg
    assert kg.kg_kn(12.0) == pytest.approx(30.0, rel=1e-4)
    assert kg.kg_strerror(kg.KG_ERR_BOND_OVERSTRETCH).startswith("bond overstretched")
    # the library's schedule (its own C++ restatement of Eqs. 16-20) agrees with the oracle's
    from oracle import schedule as S
    for kappa in (0.0, 2.0, 2.5, 4.0, 5.5):
        st = kg.kg_schedule_paper(kappa, 400, 0.008)
        assert [s.n_exp for s in st] == list(S.XI)
        assert [s.n_steps for s in st] == S.stage_steps(kappa, 400, 0.008)


def test_create_rejects_bad_arguments(lib):
    import paper_2109_11001_gb300 as kg
    with pytest.raises(kg.KGError) as e:
        kg.kg_create(kg.make_params([(10, 2, 20.0, 1.0)]), 0)      # chains shorter than 3
    assert e.value.status == kg.KG_ERR_INVALID_ARG
    with pytest.raises(kg.KGError) as e:
        kg.kg_create(kg.make_params([(10, 10, 20.0, 1.0)], precision=7), 0)
    assert e.value.status == kg.KG_ERR_INVALID_ARG


def test_entanglement_length_host_matches_oracle(lib):
    """Eq. 22 solved by the library's host bisection and by the oracle's root finder."""
    import paper_2109_11001_gb300 as kg
    from oracle import ppa as P
    N, lk = 400, 2.4
    for ratio in (0.05, 0.2, 0.45, 0.8, 0.999):
        n_ek, n_e = kg.kg_entanglement_length(ratio * (N - 1) * P.L0, N, lk)
        ref = P.n_ek_from_ratio(ratio)
        assert n_ek == pytest.approx(ref, rel=1e-12)
        assert n_e == pytest.approx(ref * lk / P.L0, rel=1e-12)
    for bad in (0.0, 1.0, 1.3):
        with pytest.raises(kg.KGError) as e:
            kg.kg_entanglement_length(bad * (N - 1) * P.L0, N, lk)
        assert e.value.status == kg.KG_ERR_INVALID_ARG
