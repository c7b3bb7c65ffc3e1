"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/ups.h (no GPU needed: nothing here calls into a kernel)."""
import ctypes
import os
import re

import pytest

from paper_2505_22335_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ups.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ups_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB_PATH)


def test_header_matches_binding_exports():
    assert declared_symbols() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_and_defaults_without_gpu(lib):
    L = binding.load()
    assert b"sm_103a" in L.ups_version()
    cfg = binding.Config()
    L.ups_config_default(ctypes.byref(cfg))
    assert cfg.n_feat == 16 and cfg.k == 10 and cfg.hidden == 32
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.alpha_max - 0.99) < 1e-7


def test_create_fails_loudly_without_a_device(lib):
    """No silent CPU fallback: creating a context without a usable GPU is an error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = binding.load()
    h = ctypes.c_void_p()
    st = L.ups_create(None, 0, ctypes.byref(h))
    assert st != binding.UPS_OK
    assert L.ups_last_error(None)
    with pytest.raises(binding.UpsError):
        binding.Renderer()


def test_bad_config_rejected(lib):
    L = binding.load()
    cfg = binding.Config()
    L.ups_config_default(ctypes.byref(cfg))
    cfg.n_feat = 7
    h = ctypes.c_void_p()
    assert L.ups_create(ctypes.byref(cfg), 0, ctypes.byref(h)) == 2
    assert b"n_feat" in L.ups_last_error(None)
