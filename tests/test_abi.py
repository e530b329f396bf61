"""The C-ABI library loads and exports every entry point declared in include/tns.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tns.h")
LIB = os.path.join(ROOT, "paper_2305_05581_gb300", "libtns.so")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(tns_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared()
    for n in ["tns_create", "tns_destroy", "tns_load_integrals", "tns_mps_init", "tns_build_env",
              "tns_psi_layout", "tns_heff_apply", "tns_sweep", "tns_last_error", "tns_davidson"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2305_05581_gb300.binding import SYMBOLS
    assert sorted("tns_" + s for s in SYMBOLS) == declared()


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    rc = lib.tns_create(ctypes.byref(h), 0, None)
    assert rc == -6 and not h.value
