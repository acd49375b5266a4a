"""The C-ABI library loads and exports every entry point include/ara.h declares (CPU only)."""

import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ara.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ARA_API\s+[\w\s\*]+?\b(ara_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libara():
    from paper_1310_2274_b300 import build

    path = build.build()
    return C.CDLL(path), path


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ara_create_yet", "ara_add_elt", "ara_add_layer", "ara_run",
                 "ara_risk_measures", "ara_create", "ara_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(libara):
    lib, path = libara
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # and nothing but the C ABI is exported (hidden visibility elsewhere)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    assert {s for s in exported if s.startswith("ara_")} == set(declared_symbols())


def test_status_strings(libara):
    lib, _ = libara
    lib.ara_status_string.restype = C.c_char_p
    assert lib.ara_status_string(0) == b"ok"
    assert lib.ara_status_string(5) == b"inversion did not converge"
    assert lib.ara_status_string(99) == b"unknown status"


def test_create_without_device_reports_no_device(libara):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib, _ = libara
    h = C.c_void_p()
    assert lib.ara_create(None, C.byref(h)) == 7  # ARA_ERR_NO_DEVICE
    assert not h.value


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1310_2274_b300 as P

    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(ImportError):
        P.lib()


def test_binding_constants_match_the_header():
    """The binding's option values and thresholds are the header's #defines."""
    import paper_1310_2274_b300 as ara

    text = open(HEADER).read()
    defs = {m.group(1): m.group(2) for m in re.finditer(r"#define\s+ARA_(\w+)\s+([\d.]+)\b", text)}
    pairs = {"OPT_SCHEDULE": ara.OPT_SCHEDULE, "SCHED_BAND": ara.SCHED_BAND,
             "SCHED_TRIAL": ara.SCHED_TRIAL, "SCHED_AUTO": ara.SCHED_AUTO,
             "OPT_TABLES": ara.OPT_TABLES, "TABLES_EAGER": ara.TABLES_EAGER,
             "TABLES_ON_DEMAND": ara.TABLES_ON_DEMAND, "OPT_BAND_WIDTH": ara.OPT_BAND_WIDTH,
             "OPT_STREAM_CHUNK": ara.OPT_STREAM_CHUNK, "TABLE_BUY_HITS": ara.TABLE_BUY_HITS,
             "BAND_BUY_PASSES": ara.BAND_BUY_PASSES}
    for name, value in pairs.items():
        assert float(defs[name]) == float(value), name
