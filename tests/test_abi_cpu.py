"""The C-ABI library without a GPU: it builds, loads, exports every entry point that include/rewl.h
declares, and rejects invalid arguments before touching the device."""
import math
import os
import re

import pytest

import paper_1411_4212_gb300 as rw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "rewl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rewl_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1411_4212_gb300 import _build
    _build.build()
    lib = rw.load_library()
    names = declared_entry_points()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_oracle_is_not_imported_by_the_library():
    src = open(os.path.join(ROOT, "paper_1411_4212_gb300", "__init__.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    for f in os.listdir(os.path.join(ROOT, "paper_1411_4212_gb300", "csrc")):
        assert "rewl_oracle" not in open(os.path.join(ROOT, "paper_1411_4212_gb300", "csrc", f)).read()


BAD = [
    dict(overlap=1.0), dict(overlap=-0.1), dict(flatness=0.0), dict(flatness=1.0), dict(lnf_final=0.0),
    dict(exchange_interval=0), dict(walkers_per_window=0), dict(L=1), dict(L=2, J=(1.0, 0.5, 0.1)),
    dict(J=(float("nan"), 0.5)), dict(n_bins=1), dict(n_windows=300),
    dict(e_min=0.0, e_max=-1.0), dict(e_min=float("inf"), e_max=0.0), dict(group_size=3), dict(overlap=0.0),
    dict(kind=rw.TABLE, nbr=[[0, 5]], Jt=[[1.0, 1.0]], e_min=-1.0, e_max=1.0),
    dict(kind=rw.TABLE, nbr=[[1, 0]], Jt=[[1.0, 1.0]]),
    dict(kind=7), dict(iteration=2), dict(resolver=4), dict(resolver=-1),
    dict(partition=(2, 2)), dict(partition=(-1, 2)), dict(partition=(0, 5)), dict(partition=(0, 2), iteration=1),
]


@pytest.mark.parametrize("bad", BAD)
def test_invalid_arguments_are_rejected(bad):
    cfg = dict(kind=rw.BCC, L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=2)
    cfg.update(bad)
    with pytest.raises(rw.RewlError) as e:
        rw.REWL(**cfg)
    assert e.value.status == rw.EINVAL
    assert rw.load_library().rewl_last_error(None)


def test_no_device_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rw.RewlError) as e:
        rw.REWL(kind=rw.BCC, L=4, J=(1.0, 0.5), n_bins=200, n_windows=4, walkers_per_window=2, stream=0)
    assert e.value.status == rw.ECUDA


def test_batch_entry_points_reject_invalid_arguments():
    import ctypes as C
    lib = rw.load_library()
    out = C.c_void_p()
    assert lib.rewl_batch_create(None, 0, None, C.byref(out)) == rw.EINVAL and not out.value
    assert b"no jobs" in lib.rewl_last_error(None)
    arr = (C.c_void_p * 1)(None)
    assert lib.rewl_batch_create(arr, 1, None, C.byref(out)) == rw.EINVAL
    assert lib.rewl_batch_create(arr, 1, None, None) == rw.EINVAL
    assert lib.rewl_batch_get_info(None, None) == rw.EINVAL
    assert lib.rewl_batch_run_intervals(None, 1) == rw.EINVAL
    assert lib.rewl_batch_autotune(None, 10, None, None) == rw.EINVAL
    assert lib.rewl_autotune(None, 10, None, None) == rw.EINVAL
    assert lib.rewl_batch_run_to_convergence(None, 1, 1, None) == rw.EINVAL
    lib.rewl_batch_destroy(None)
    t = C.c_double()
    assert lib.rewl_peak_temperature(None, None, 0, C.byref(t), None) == rw.EINVAL
    n = C.c_int64()
    assert lib.rewl_state_bytes(None, C.byref(n)) == rw.EINVAL
    assert lib.rewl_save_state(None, None, 0) == rw.EINVAL and lib.rewl_load_state(None, None, 0) == rw.EINVAL
    assert lib.rewl_slot_export(None, 0, None) == rw.EINVAL and lib.rewl_partition_observe(None) == rw.EINVAL
