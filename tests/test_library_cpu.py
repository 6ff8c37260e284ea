"""Host-side checks of the C ABI library (no GPU needed).

The library must build for sm_103a, load, export every function that
include/splitsolve.h declares, and fail cleanly (no abort) without a device.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

import __graft_entry__
import paper_1812_01396_gb300 as ss

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ss.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "splitsolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(ss_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for f in ("ss_create", "ss_set_hamiltonian", "ss_self_energy", "ss_solve", "ss_transmission",
              "ss_destroy", "ss_last_error", "ss_config_default"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", ss.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_build_targets_sm_103a_only():
    from paper_1812_01396_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_default_values(lib):
    cfg = ss.ss_config_default()
    assert cfg.s_b_max == 512 and cfg.n_b_max == 64 and cfg.precision == ss.SS_FP64
    assert cfg.eta == 1e-10 and cfg.decim_tol == 1e-14 and cfg.decim_max_iter == 100


def test_create_rejects_bad_arguments_without_device(lib):
    h = C.c_void_p()
    assert lib.ss_create(None, None) == ss.SS_ERR_ARG
    cfg = ss.ss_config_default()
    cfg.s_b_max = 0
    assert lib.ss_create(C.byref(h), C.byref(cfg)) == ss.SS_ERR_ARG
    assert h.value is None
    assert lib.ss_destroy(None) == ss.SS_OK
    assert isinstance(lib.ss_last_error(None), bytes)


@pytest.mark.parametrize("field,value", [
    ("partitions", 0), ("partitions", 9), ("lu_lookahead", 2), ("lu_lookahead", -1),
])
def test_create_rejects_bad_options_before_touching_a_device(lib, field, value):
    """Option checks run on the host before any CUDA call, and each names the
    field in the error text."""
    h = C.c_void_p()
    cfg = ss.ss_config_default()
    setattr(cfg, field, value)
    assert lib.ss_create(C.byref(h), C.byref(cfg)) == ss.SS_ERR_ARG
    assert h.value is None
    assert field.encode() in lib.ss_last_error(None)


def test_config_defaults_of_the_options(lib):
    cfg = ss.ss_config_default()
    assert (cfg.partitions, cfg.memory_lean, cfg.hermitian_sweeps, cfg.obc) == (1, 0, 0, ss.SS_OBC_DECIMATION)
    assert (cfg.tournament_pivoting, cfg.lu_lookahead, cfg.use_graphs) == (0, 0, 1)


def test_create_reports_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    cfg = ss.ss_config_default()
    rc = lib.ss_create(C.byref(h), C.byref(cfg))
    assert rc == ss.SS_ERR_CUDA
    assert h.value is None
    assert b"device" in lib.ss_last_error(None).lower()


def test_caroli_entry_points_reject_host_tensors_before_any_launch(lib):
    """CPU tensors (or anything not a CUDA tensor) are refused by the binding
    with ValueError, so no kernel can be handed a host pointer."""
    import torch
    a = torch.zeros((2, 4, 4), dtype=torch.complex128)
    T = torch.zeros(2, dtype=torch.float64)
    for fn in (ss.ss_caroli_transmission, ss.ss_caroli_transmission_noalloc):
        with pytest.raises(ValueError):
            fn(a, a, a, T)
