"""The C-ABI library builds, loads and exports every symbol include/zncc.h declares; host-side
argument checks answer without touching a GPU. CPU only."""

import ctypes
import os
import re

import pytest

from paper_2212_00476_gb300 import build as zbuild
from paper_2212_00476_gb300 import zncc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "zncc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\**\s+\**(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    zbuild.build()
    return zncc.lib()


def test_header_parsed():
    names = _declared_functions()
    for must in ["zncc_create", "zncc_cost_volume", "dt_aggregate", "wta_disparity", "zncc_run",
                 "zncc_run_host", "zncc_window_stats"]:
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    declared = _declared_functions()
    bound = {name for name, _, _ in zncc.SIGNATURES}
    assert set(declared) == bound, (set(declared) ^ bound)
    for name in declared:
        assert hasattr(lib, name), name


def test_create_rejects_bad_arguments_without_gpu(lib):
    h = ctypes.c_void_p()
    cases = [((0, 10, 4, 9), zncc.ZNCC_EINVAL), ((10, 0, 4, 9), zncc.ZNCC_EINVAL),
             ((10, 10, 0, 9), zncc.ZNCC_EINVAL), ((10, 10, 4, 8), zncc.ZNCC_EINVAL),
             ((10, 10, 4, 1), zncc.ZNCC_EINVAL), ((10, 10, 4, 17), zncc.ZNCC_EINVAL),
             ((3073, 10, 4, 9), zncc.ZNCC_EUNSUPPORTED), ((10, 4097, 4, 9), zncc.ZNCC_EUNSUPPORTED),
             ((10, 10, 2000, 9), zncc.ZNCC_EUNSUPPORTED)]
    for args, want in cases:
        st = lib.zncc_create(*args, ctypes.byref(h))
        assert st == want, (args, st)
        assert h.value is None
        assert lib.zncc_last_error(None).decode() != ""
    assert lib.zncc_create(10, 10, 4, 9, None) == zncc.ZNCC_EINVAL


def test_null_context_and_status_strings(lib):
    assert lib.zncc_destroy(None) == zncc.ZNCC_EINVAL
    assert lib.zncc_set_stream(None, None) == zncc.ZNCC_EINVAL
    assert lib.zncc_volume_bytes(None, 0) == 0
    assert lib.zncc_run(None, None, None, 0, 1.0, 1.0, 0, 0, None) == zncc.ZNCC_EINVAL
    for s, name in enumerate(zncc.STATUS_NAMES):
        assert lib.zncc_status_string(s).decode() == name


def test_header_constants_match_the_binding():
    """Every enumerator include/zncc.h gives a value (status codes, storage types, tuning keys)
    has a constant of the same name and value in the Python binding."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "zncc.h")).read(), flags=re.S)
    pairs = re.findall(r"\b(ZNCC_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)
    tune = [n for n, _ in pairs if n.startswith("ZNCC_TUNE_")]
    assert "ZNCC_TUNE_AHAT_JOIN" in tune and len(tune) >= 12
    for name, value in pairs:
        assert hasattr(zncc, name), name
        assert getattr(zncc, name) == int(value), (name, getattr(zncc, name), value)
