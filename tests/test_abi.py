"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/frpca.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(frpca_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1810_06825_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_entry_points():
    names = _declared()
    for required in ("frpca_create", "frpca_run", "frpca_destroy", "frpca_last_error", "frpca_spmm", "frpca_lu",
                     "frpca_gram", "frpca_eig", "frpca_eigsvd", "frpca_gaussian", "frpca_get_transpose"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    cdll, path = lib
    missing = [n for n in sorted(_declared()) if not hasattr(cdll, n)]
    assert not missing, f"not exported: {missing}"
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (frpca_\w+)", out))
    assert _declared() <= exported


def test_python_binding_names_match_header():
    import paper_1810_06825_gb300 as frpca
    for name in _declared():
        assert hasattr(frpca, name), name
    assert set(frpca.EXPORTED) <= _declared()


def test_last_error_without_handle_is_safe(lib):
    import paper_1810_06825_gb300 as frpca
    assert isinstance(frpca.frpca_last_error(None), str)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_1810_06825_gb300 as frpca
    monkeypatch.setattr(frpca, "_lib", None)
    monkeypatch.setattr(frpca, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        frpca.library()
