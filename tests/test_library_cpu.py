"""CPU-side checks of the CUDA library: it builds for sm_103a, loads without a
GPU, and exports every entry point that include/nbgpu.h declares.  No compute
call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:NB_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**(nb_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["nb_fit", "nb_score_group", "nb_model_counts", "nb_model_free",
                     "nb_last_error"]:
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    import paper_1905_13746_gb300 as nb
    path = nb.build()
    assert os.path.exists(path)
    handle = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(handle, n)]
    assert not missing, f"declared but not exported: {missing}"
    lib = nb.lib()
    assert lib.nb_version().decode().startswith("nbgpu")
    for name in nb.EXPORTED:
        assert name in _declared(), f"binding names {name} but the header does not declare it"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1905_13746_gb300 as nb
    monkeypatch.setattr(nb, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nb, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nb.lib()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1905_13746_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "nb_oracle" not in text, fn
