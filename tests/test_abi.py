"""The C-ABI library loads and exports every entry point include/fastlsq.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fastlsq.h")).read()
    return sorted(set(re.findall(r"FASTLSQ_API\s+[\w\s\*]*?\b(fastlsq_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_10541_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("fastlsq_assemble", "fastlsq_lstsq", "fastlsq_newton", "fastlsq_backward"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2602_10541_gb300 import fastlsq as fl
    assert set(_declared()) <= set(fl._SIGNATURES)


def test_binding_signatures_match_header_arity():
    """Every binding passes as many arguments as the header's declaration takes."""
    from paper_2602_10541_gb300 import fastlsq as fl
    src = open(os.path.join(ROOT, "include", "fastlsq.h")).read()
    for name, params in re.findall(r"FASTLSQ_API\s+[\w\s\*]*?\b(fastlsq_\w+)\s*\(([^)]*)\)", src):
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(fl._SIGNATURES[name]) == n, (name, n, len(fl._SIGNATURES[name]))


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2602_10541_gb300 import _build
    from paper_2602_10541_gb300 import fastlsq as fl
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fl, "_lib", None)
    with pytest.raises(RuntimeError):
        fl.load()


def test_create_fails_cleanly_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    rc = lib.fastlsq_create(ctypes.byref(h), 0, None)
    assert rc < 0 and not h.value
