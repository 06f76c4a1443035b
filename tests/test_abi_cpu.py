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


def _scene_file_header(**kw):
    """A scene file header (magic, version, counts, layout, blob offsets) in
    the 192-byte layout cs_scene_load reads; one chunk, one Gaussian."""
    f = dict(magic=b"CSB300SC", version=1, header_bytes=192, n_input=1, n_kept=1, n_grid=1, n_large=0,
             n_invalid=0, blob_bytes=2820, app_bytes=0, nchunks=1, large_chunk0=1, n_gauss=1,
             nnodes=(1, 1, 1), floats=(0.1, 0.0, 1e-6, 0, 0, 0, 1, 1, 1),
             off_chead=1280, off_nodes=(1536, 1792, 2048), off_smax=2304, off_index=2560, off_slot=2816)
    f.update(kw)
    import struct
    return struct.pack("<8sII7q6i9f4x7q", f["magic"], f["version"], f["header_bytes"], f["n_input"], f["n_kept"],
                       f["n_grid"], f["n_large"], f["n_invalid"], f["blob_bytes"], f["app_bytes"], f["nchunks"],
                       f["large_chunk0"], f["n_gauss"], *f["nnodes"], *f["floats"], f["off_chead"], *f["off_nodes"],
                       f["off_smax"], f["off_index"], f["off_slot"])


def test_scene_file_checks_without_device(tmp_path):
    """cs_scene_load validates a file before it touches the device: missing
    file, wrong magic or version, an inconsistent layout, a truncated blob and
    a slot index out of range are CS_ERR_INVALID_ARG with *out NULL."""
    assert len(_scene_file_header()) == 192
    out = ctypes.c_void_p()
    assert abi.cs_scene_save(None, str(tmp_path / "x"), None) == abi.CS_ERR_BAD_HANDLE
    assert abi.cs_scene_load(None, None, out) == abi.CS_ERR_INVALID_ARG
    assert abi.cs_scene_load(str(tmp_path / "missing"), None, out) == abi.CS_ERR_INVALID_ARG
    blob = bytearray(2820)
    cases = {
        "magic": _scene_file_header(magic=b"CSB300XX") + bytes(blob),
        "another format version": _scene_file_header(version=2) + bytes(blob),
        "short header": _scene_file_header()[:100],
        "inconsistent layout": _scene_file_header(nnodes=(2, 1, 1)) + bytes(blob),
        "inconsistent layout ": _scene_file_header(off_slot=2817) + bytes(blob),
        "inconsistent layout  ": _scene_file_header(n_grid=0) + bytes(blob),
        "truncated": _scene_file_header() + bytes(blob[:-1]),
    }
    slot_bad = bytearray(blob)
    slot_bad[2816:2820] = (32).to_bytes(4, "little")  # one chunk has slots 0..31
    cases["slot index"] = _scene_file_header() + bytes(slot_bad)
    for why, data in cases.items():
        p = tmp_path / "f.csscene"
        p.write_bytes(data)
        assert abi.cs_scene_load(str(p), None, out) == abi.CS_ERR_INVALID_ARG, why
        assert not out
        assert why.strip() in abi.cs_last_error(), (why, abi.cs_last_error())
