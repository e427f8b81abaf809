"""The C ABI library builds, loads and exports every entry point that
include/prgb.h declares (no GPU needed: only host-side argument checks run)."""
import ctypes as C
import os
import re
import shutil

import pytest

import paper_1609_09068_gb300 as prgb
from paper_1609_09068_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "prgb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pr_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not _build.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        _build.build()
    return prgb.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(prgb._SIGS), "binding signatures drift from the header"


def test_status_strings(lib):
    for code in range(7):
        assert lib.pr_status_str(code)
    assert lib.pr_status_str(1) == b"invalid argument"


def test_null_arguments_rejected_on_host(lib):
    out = C.c_void_p()
    assert lib.pr_graph_create(None, None, C.byref(out)) == 1
    csr = prgb._Csr(-1, 0, None, None, 1)
    assert lib.pr_graph_create(C.byref(csr), None, C.byref(out)) == 1
    csr = prgb._Csr(5, 1 << 31, None, None, 1)
    assert lib.pr_graph_create(C.byref(csr), None, C.byref(out)) == 1
    assert lib.pr_partition_create(None, 0, None, C.byref(out)) == 1
    assert lib.pr_solve(None, 0.85, None, 1e-10, None, None, None, None) == 1
    assert lib.pr_global_power(None, 0.85, None, 1e-10, None, None, None, None) == 1
    r = C.c_double()
    assert lib.pr_residual_l1(None, 0.85, None, None, C.byref(r), None) == 1
    lib.pr_graph_destroy(None)
    lib.pr_partition_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(prgb, "_lib", None)
    monkeypatch.setattr(prgb, "_LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        prgb.load_library()


def test_newer_entry_points_reject_null_arguments_on_host(lib):
    from oracle import mpnn as ref
    assert lib.pr_mpnn_param_count() == ref.N_PARAMS == 9409
    assert lib.pr_mpnn_create(C.c_uint64(1), None, None) == 1
    buf = (C.c_float * ref.N_PARAMS)()
    assert lib.pr_mpnn_get_params(None, buf, ref.N_PARAMS) == 1
    assert lib.pr_mpnn_set_params(None, buf, ref.N_PARAMS) == 1
    assert lib.pr_mpnn_predict(None, None, 0.85, None, None, None, None, None) == 1
    assert lib.pr_mpnn_loss_grad(None, None, 0.85, None, None, None, None, None) == 1
    assert lib.pr_mpnn_train_step(None, None, 0.85, None, None, C.c_float(1e-3), None, None) == 1
    lib.pr_mpnn_destroy(None)
    assert lib.pr_partition_set_shape(None, 256, 4, 1) == 1
    assert lib.pr_partition_tune(None, 0.85, None, 1e-10, None, None, None, None, None) == 1
    assert lib.pr_launch_count() >= 0


def test_last_device_error_records_and_clears(lib):
    lib.pr_last_device_error()  # start clean
    assert lib.pr_last_device_error() == 0
    out = C.c_void_p()
    assert lib.pr_graph_create(None, None, C.byref(out)) == 1
    assert lib.pr_mpnn_param_count() > 0  # a call that cannot fail leaves it alone
    assert lib.pr_last_device_error() == 1
    assert lib.pr_last_device_error() == 0  # reading cleared it
    assert lib.pr_partition_set_shape(None, 256, 4, 1) == 1
    assert lib.pr_solve(None, 0.85, None, 1e-10, None, None, None, None) == 1
    assert lib.pr_last_device_error() == 1
