"""The C-ABI library loads and exports every entry point declared in
include/cs_b300.h; argument checks that precede any CUDA call behave as the
header states.  CPU only (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2609_35619_b300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cs_b300.h")).read()
    return sorted(set(re.findall(r"^CS_API[^(]*?\b(cs_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = _declared()
    assert "cs_query" in names and "cs_query_grad" in names and "cs_scene_create" in names
    assert len(names) >= 12


def test_library_exports_every_declared_symbol():
    lib = abi.load()
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in the header but not exported"
    assert set(abi.symbols()) >= set(_declared())


def test_exported_symbols_match_header_exactly():
    """No undeclared cs_* symbol leaks out of the library (hidden visibility)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r"\bT (cs_\w+)", out)))
    assert exported == _declared()


def test_params_defaults():
    p = abi.cs_params()
    assert abi.cs_params_init(p) == abi.CS_OK
    assert (p.gamma, p.d_max, p.s_min, p.tau) == (5.0, 1.0, 1.0, pytest.approx(0.05))
    assert p.eps == pytest.approx(1e-6) and p.k_thr == 0 and p.mode == abi.CS_METRIC_MEAN_COST
    assert p.group_size == 0 and p.host_io == 0 and not p.stream


def test_argument_errors_without_device():
    lib = abi.load()
    # bad handles
    assert abi.cs_query(None, 0, None, 1, 1.0, None, None, None) == abi.CS_ERR_BAD_HANDLE
    assert abi.cs_query_grad(None, 0, None, 1, 1.0, None, None, None) == abi.CS_ERR_BAD_HANDLE
    assert abi.cs_query_fwd_grad(None, 0, None, 1, 1.0, None, None, None, None, None) == abi.CS_ERR_BAD_HANDLE
    assert abi.cs_sync(None, 0) == abi.CS_ERR_BAD_HANDLE
    assert abi.cs_scene_destroy(None) == abi.CS_OK  # NULL is a no-op
    # scene description checks
    out = ctypes.c_void_p()
    d = abi.cs_scene_desc()
    d.n = -1
    assert abi.cs_scene_create(d, 0, out) == abi.CS_ERR_INVALID_ARG
    assert "n out of range" in abi.cs_last_error()
    d.n = 10
    assert abi.cs_scene_create(d, 0, out) == abi.CS_ERR_INVALID_ARG  # missing arrays
    d.means = d.scales = d.quats = 1
    d.tier_quantile = 2.0
    assert abi.cs_scene_create(d, 0, out) == abi.CS_ERR_INVALID_ARG
    # pose chain checks
    assert abi.cs_pose_spheres(None, 4, None, 8, -1.0, None, 0) == abi.CS_ERR_INVALID_ARG
    assert abi.cs_pose_spheres(None, 0, None, 8, 1.0, None, 0) == abi.CS_OK
    assert abi.cs_params_init.__name__ and lib.cs_params_init(None) == abi.CS_ERR_INVALID_ARG


def test_tile_configs_and_version():
    ids = abi.cs_tile_configs()
    assert len(ids) >= 2 and len(set(ids)) == len(ids) and 0 not in ids
    assert "sm_103a" in abi.cs_version()


def test_binding_marshals_numpy_and_rejects_strided():
    a = np.zeros((4, 4), np.float32)
    assert abi.ptr(a) == a.ctypes.data
    with pytest.raises(ValueError):
        abi.ptr(a[:, ::2])
    assert abi.ptr(None) is None
