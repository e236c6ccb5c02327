"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"HD_API\s+[\w\s\*]+?\b(hd_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2101_07464_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("hd_create", "hd_apply", "hd_reset", "hd_destroy", "hd_set_options", "hd_probe"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hd_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert getattr(lib, n) is not None


def test_library_exports_nothing_undeclared(libpath):
    """Every hd_* symbol the library exports is declared (and documented) in include/*.h."""
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hd_\w+)", out))
    extra = sorted(exported - set(_declared()))
    assert not extra, extra


def test_binding_loads_and_maps_status_strings(libpath):
    import paper_2101_07464_gb300 as hd
    L = hd.lib()
    assert L.hd_status_string(0) == b"HD_OK"
    assert b"TMAX" in L.hd_status_string(3)


def test_argument_errors_need_no_gpu(libpath):
    import paper_2101_07464_gb300 as hd
    L = hd.lib()
    h = ctypes.c_void_p()
    # invalid arguments are rejected before any device work
    assert L.hd_create(7, 4, 4, 2, 0, 0, ctypes.byref(h)) == hd.binding.HD_ERR_ARG
    assert L.hd_create(hd.HD_HAAR, 4, 5, 2, 0, 0, ctypes.byref(h)) == hd.binding.HD_ERR_DIM
    assert L.hd_create(hd.HD_HAAR, 4, 4, 5, 0, 0, ctypes.byref(h)) == hd.binding.HD_ERR_TMAX
    assert L.hd_create(hd.HD_GINIBRE, 3, 6, 4, 0, 0, ctypes.byref(h)) == hd.binding.HD_ERR_TMAX
    assert L.hd_create(hd.HD_GINIBRE, 0, 6, 1, 0, 0, ctypes.byref(h)) == hd.binding.HD_ERR_DIM
    assert L.hd_apply(None, None, 0, None) == hd.binding.HD_ERR_ARG
    assert L.hd_reset(None, 0) == hd.binding.HD_ERR_ARG
    L.hd_destroy(None)


def test_tuning_entry_points_reject_null_state_without_gpu(libpath):
    import paper_2101_07464_gb300 as hd
    L = hd.lib()
    words = (ctypes.c_int32 * hd.binding.HD_TUNE_WORDS)()
    cnt = ctypes.c_int32()
    ARG = hd.binding.HD_ERR_ARG
    assert L.hd_autotune(None, None, None, None, 1) == ARG
    assert L.hd_get_tuning(None, words, hd.binding.HD_TUNE_WORDS) == ARG
    assert L.hd_set_tuning(None, words, hd.binding.HD_TUNE_WORDS) == ARG
    assert L.hd_get_map_options(None, ctypes.byref(cnt), None) == ARG


def test_tuning_word_count_matches_header():
    """[version, split option] + (warps, stages) for 6 sweep kernels x 11 column ranges."""
    import paper_2101_07464_gb300 as hd
    txt = open(os.path.join(ROOT, "include", "hd.h")).read()
    m = re.search(r"#define HD_TUNE_WORDS (\d+)", txt)
    assert m and int(m.group(1)) == hd.binding.HD_TUNE_WORDS == 2 + 2 * 6 * 11


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libhd.so every entry point raises instead of computing."""
    import paper_2101_07464_gb300 as hd
    monkeypatch.setattr(hd.binding, "_LIB", None)
    monkeypatch.setattr(hd.binding._build, "LIB", str(tmp_path / "libhd.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hd.lib()
    with pytest.raises(RuntimeError, match="not built"):
        hd.hd_create("haar", 8, 8, 2, 0, "f64")
