"""The C-ABI library builds, loads and exports every entry point include/*.h declares.

No GPU is needed: only argument checks that fail before any CUDA call are exercised.
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2212_08058_gb300 import build
    return build.build()


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
        names |= set(re.findall(r"\b(sfseg_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sfseg_\w+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_every_declaration(libpath):
    from paper_2212_08058_gb300 import sfseg
    assert _declared() <= set(sfseg.SIGNATURES)
    L = sfseg.lib(libpath)
    for name in _declared():
        assert hasattr(L, name)


def test_argument_checks_without_gpu(libpath):
    from paper_2212_08058_gb300 import sfseg
    L = sfseg.lib(libpath)
    assert L.sfseg_version() >= 100
    h = ctypes.c_void_p()
    assert L.sfseg_create(None, 1, 2, 2, 2, ctypes.byref(h)) == 1           # INVALID_ARG
    bad_alpha = sfseg.Params(0.0, 0.1)
    assert L.sfseg_create(ctypes.byref(bad_alpha), 1, 2, 2, 2, ctypes.byref(h)) == 1
    assert b"alpha" in L.sfseg_last_error()
    ok = sfseg.Params(1.0, 0.1)
    assert L.sfseg_create(ctypes.byref(ok), 1, 0, 2, 2, ctypes.byref(h)) == 2  # SHAPE: empty
    assert L.sfseg_create(ctypes.byref(ok), 0, 1, 2, 2, ctypes.byref(h)) == 1  # C < 1
    assert L.sfseg_create(ctypes.byref(ok), 1, 2048, 2048, 1024, ctypes.byref(h)) == 2  # >= 2^31
    assert L.sfseg_destroy(None) == 0
    nb = sfseg.neighborhood((1, 3, 3))
    assert L.sfseg_power_iterate(None, None, 0, None, 0.0, ctypes.byref(nb), 1, 0, None, 1, 0, None, None) == 1
    # the other entry points refuse a null handle before touching the GPU
    assert L.sfseg_soft_binarize(None, ctypes.byref(nb), 1, 1.0, 0.5, None, None, None) == 1
    assert L.sfseg_set_features_sf(None, None, 0, 1, None, 0.0, None, 0, None, 0.0, None) == 1
    assert L.sfseg_coarse_start(None, ctypes.byref(nb), 2, 1e-4, 10, 10, None, None, None) == 1
    assert L.sfseg_selftest_wait(None, 10, None) == 1
    o = ctypes.c_void_p()
    assert L.sfseg_online_create(ctypes.byref(ok), 1, 0, 8, 8, ctypes.byref(o)) == 1     # q < 1
    assert L.sfseg_online_push(None, None, 0, None, 0.0, ctypes.byref(nb), 1, 0, 0, None, None) == 1
    assert L.sfseg_online_destroy(None) == 0
    # the network's launch-shape report: nothing launched yet on this thread, bad kernel index
    f, r, c = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int(-1)
    assert L.sfseg_net_launch_shape(0, ctypes.byref(f), ctypes.byref(r), ctypes.byref(c)) == 0
    assert (f.value, r.value, c.value) == (0, 0, 0)
    assert L.sfseg_net_launch_shape(2, ctypes.byref(f), ctypes.byref(r), ctypes.byref(c)) == 1
    assert L.sfseg_net_launch_shape(1, None, ctypes.byref(r), ctypes.byref(c)) == 1


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    """No fallback: a missing library is an error, not a slower path."""
    from paper_2212_08058_gb300 import sfseg
    monkeypatch.setattr(sfseg, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        sfseg.lib(str(tmp_path / "nope.so"))
