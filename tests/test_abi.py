"""The C-ABI library builds, loads and exports every symbol include/nfmimo.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "nfmimo.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nfm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("nfm_set_geometry", "nfm_forward", "nfm_adjoint", "nfm_spgm_epoch", "nfm_power_iteration"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2509_00774_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_boundary():
    from paper_2509_00774_gb300 import nfmimo
    lib = nfmimo.load_library()
    for n in _declared():
        assert getattr(lib, n).argtypes is not None or n == "nfm_destroy", n
    ctx_methods = {m for m in dir(nfmimo.Context) if not m.startswith("_")}
    batch_methods = {m for m in dir(nfmimo.Batch) if not m.startswith("_")}
    for n in _declared():
        short = n[len("nfm_"):]
        if short in ("create", "destroy", "last_error", "batch_create", "batch_destroy", "batch_last_error"):
            continue
        if short.startswith("batch_"):
            assert short[len("batch_"):] in batch_methods, short
        else:
            assert short in ctx_methods, short


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2509_00774_gb300 import nfmimo
    lib = nfmimo.load_library()
    h = ctypes.c_void_p()
    rc = lib.nfm_create(ctypes.byref(h), 0, None)
    assert rc != 0 and not h.value
    assert lib.nfm_last_error(None)
