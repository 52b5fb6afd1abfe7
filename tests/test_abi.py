"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/sl.h declares; the Python binding mirrors them by name."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sl_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1606_06117_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for s in ("sl_advect", "sl_advect_multi", "sl_advect_host", "sl_batch_create", "sl_batch_step",
              "sl_norms", "sl_courant_max", "sl_device_status", "sl_autotune", "sl_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b[TW] (sl_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_build_targets_sm_103a():
    from paper_1606_06117_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_library_loads_and_binding_mirrors_header(libpath):
    from paper_1606_06117_gb300 import _lib
    lib = _lib.load(libpath)
    assert lib.sl_version() >= 10000
    assert sorted(_lib.EXPORTS) == declared_symbols()
    for s in declared_symbols():
        assert callable(getattr(_lib, s))


def test_binding_refuses_missing_library(tmp_path):
    from paper_1606_06117_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_wide_workspace_sizes_without_a_gpu(libpath):
    """sl_advect_wide_workspace only does arithmetic on its arguments: the
    number of intermediate fields per scheme (CIR 0, FEC 1, BEC 2, CEC 3 in 2D
    and 4 in 3D), each rounded up to 256 bytes, and the argument errors."""
    from paper_1606_06117_gb300 import _lib
    _lib.load(libpath)
    field32 = (10 * 12 * 14 * 4 + 255) // 256 * 256
    for scheme, count in ((_lib.CIR, 0), (_lib.FEC, 1), (_lib.BEC, 2), (_lib.CEC, 4)):
        assert _lib.sl_advect_wide_workspace(3, [10, 12, 14], scheme, _lib.F32) == count * field32
    assert _lib.sl_advect_wide_workspace(2, [33, 7, 1], _lib.CEC, _lib.F64) == 3 * ((33 * 7 * 8 + 255) // 256 * 256)
    with pytest.raises(_lib.SLError, match="SL_ERR_UNSUPPORTED"):
        _lib.sl_advect_wide_workspace(3, [8, 8, 8], _lib.CEC, _lib.F32_D64)
    with pytest.raises(_lib.SLError, match="SL_ERR_ARG"):
        _lib.sl_advect_wide_workspace(3, [8, 8, 8], 7, _lib.F32)
    with pytest.raises(_lib.SLError, match="SL_ERR_ARG"):
        _lib.sl_advect_wide_workspace(2, [8, 8, 2], _lib.CIR, _lib.F32)


def test_wide_step_argument_checks_without_a_gpu(libpath):
    """sl_advect_wide validates its arguments before any CUDA call, so the
    host logic runs here with addresses that are never dereferenced."""
    from paper_1606_06117_gb300 import _lib
    _lib.load(libpath)
    dims = [8, 8, 8]
    sp = [1.0, 1.0, 1.0]
    fb = 8 * 8 * 8 * 4
    inp, out, vel = 0x100000, 0x200000, 0x300000
    need = _lib.sl_advect_wide_workspace(3, dims, _lib.CEC, _lib.F32)
    ws = 0x400000
    cases = [
        ((out, 0, vel, 3, dims, sp, 0.1, _lib.CEC, _lib.F32, 0, ws, need), "SL_ERR_ARG"),          # NULL input
        ((out, inp, vel, 3, dims, sp, 0.1, _lib.CEC, _lib.F32, 0, ws, need - 1), "SL_ERR_ARG"),  # small workspace
        ((out, inp, vel, 3, dims, sp, 0.1, _lib.CEC, _lib.F32, 0, 0, need), "SL_ERR_ARG"),       # NULL workspace
        ((out, inp, vel, 3, dims, sp, 0.1, _lib.CEC, _lib.F32, 0, ws + 16, need), "SL_ERR_ARG"),  # misaligned
        ((inp + fb // 2, inp, vel, 3, dims, sp, 0.1, _lib.CEC, _lib.F32, 0, ws, need), "SL_ERR_ALIAS"),
        ((out, inp, vel, 3, dims, sp, 0.1, _lib.CEC, _lib.F32, 0, vel + 256, need), "SL_ERR_ALIAS"),
        ((out, inp, vel, 2, [8, 70000, 1], sp, 0.1, _lib.CIR, _lib.F32, 0, 0, 0), "SL_ERR_UNSUPPORTED"),
        ((out, inp, vel, 3, dims, [1.0, 0.0, 1.0], 0.1, _lib.CEC, _lib.F32, 0, ws, need), "SL_ERR_ARG"),
    ]
    for args, code in cases:
        with pytest.raises(_lib.SLError, match=code):
            _lib.sl_advect_wide(*args)
