"""The C ABI library builds, loads and exports every entry point include/qtraj.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qtraj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qtraj_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2107_06147_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(libpath):
    names = _declared()
    assert "qtraj_create" in names and "qtraj_evolve" in names and len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (qtraj_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_library_loads_and_prototypes_cover_the_header(libpath):
    from paper_2107_06147_gb300 import qtraj
    lib = qtraj.load()
    for n in _declared():
        assert hasattr(lib, n)
        assert n in qtraj._PROTOS, f"binding lacks a prototype for {n}"
    # no device work: error reporting and argument checks run on the host
    h = ctypes.c_void_p()
    p = qtraj.Config(N=100).params()
    st = lib.qtraj_create(100, 20.0, 0.001, 4.65, ctypes.byref(p), ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"power of two" in lib.qtraj_last_error(None)
    p = qtraj.Config(precision=qtraj.FP32, form=qtraj.PLAIN).params()
    assert lib.qtraj_create(512, 20.0, 0.001, 4.65, ctypes.byref(p), ctypes.byref(h)) == 1
    assert lib.qtraj_workspace_bytes(None, 10) == 0
    assert lib.qtraj_philox4x32_10(None, None, -1, None, None) == 1
    assert lib.qtraj_period_draws(None, None, 5, None, None) == 1
    assert b"null buffer" in lib.qtraj_last_error(None)


def test_record_layouts_agree():
    import oracle
    from paper_2107_06147_gb300 import qtraj
    assert qtraj.OBS_DTYPE.itemsize == 192
    assert oracle.OBS_DTYPE.names == qtraj.OBS_DTYPE.names
    assert ctypes.sizeof(qtraj.Params) == 80 and ctypes.sizeof(qtraj.Medium) == 56
