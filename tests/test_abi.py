"""The C-ABI library builds, loads and exports every symbol include/xs.h declares (CPU only, no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_24807_gb300 import build
    path = build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as e:  # CUDA runtime libraries absent on this host
        pytest.skip(f"cannot load libxs.so here: {e}")


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "xs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("xs_create", "xs_destroy", "xs_set_params", "xs_ground_state", "xs_excited",
                     "xs_get_amplitudes", "xs_apply", "xs_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2505_24807_gb300 import xs
    for n in declared_symbols():
        assert hasattr(xs, n), n


def test_null_context_is_rejected_without_a_gpu(lib):
    lib.xs_destroy.argtypes = [ctypes.c_void_p]
    assert lib.xs_destroy(None) == 0
    lib.xs_last_error.restype = ctypes.c_char_p
    lib.xs_last_error.argtypes = [ctypes.c_void_p]
    assert lib.xs_last_error(None) == b"null context"
