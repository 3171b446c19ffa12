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


def test_group_fallback_host_logic_matches_the_oracle():
    # nb_group_fallback is host code (no GPU needed): the small-group rule of
    # Sec. 4 against the oracle, on the paper's own list and random cases
    import numpy as np

    import paper_1905_13746_gb300 as nb
    from oracle import groupwise as ogw
    cc = np.full((100, 2), 30)
    cc[[4, 7, 60, 64, 96, 97, 99]] = (5, 40)
    assert nb.group_fallback(cc).tolist() == ogw.group_models(cc).tolist()
    rng = np.random.default_rng(3)
    for _ in range(200):
        nb_ = int(rng.integers(1, 40))
        C = int(rng.integers(2, 4))
        cc = rng.integers(0, 12, size=(nb_, C))
        mf = int(rng.integers(0, 8))
        try:
            ref = ogw.group_models(cc, mf).tolist()
        except ValueError:
            with pytest.raises(nb.NbError):
                nb.group_fallback(cc, mf)
            continue
        assert nb.group_fallback(cc, mf).tolist() == ref


def test_groupwise_arguments_rejected_before_any_device_work():
    import paper_1905_13746_gb300 as nb
    lib = nb.lib()
    # invalid shapes fail with NB_EINVAL and a message, without touching a GPU
    assert lib.nb_route(None, -1, 5120, 100, None, 100, None, 2, None, None, None, None, None,
                        0, None, None) == nb.NB_EINVAL
    assert b"nb_route" in lib.nb_last_error()
    assert lib.nb_gather(None, nb.NB_U16, 16, 16, 1, 1, None, None, 1, None, 1, None, 16, None,
                         None) == nb.NB_EINVAL
    assert lib.nb_select_features(None, 0, 1, 0, None, None) == nb.NB_EINVAL
    assert lib.nb_route_workspace(10000, 100) >= 100 * 8


def test_label_and_size_tensors_checked_before_the_call():
    # the library reads labels as int32 and sizes as int64: any other tensor
    # is refused in the binding instead of being misread
    import torch

    import paper_1905_13746_gb300 as nb
    nb._labels(torch.zeros(4, dtype=torch.int32), 4)
    for bad in (torch.zeros(4, dtype=torch.int64), torch.zeros(5, dtype=torch.int32),
                torch.zeros((2, 2), dtype=torch.int32), torch.zeros(8, dtype=torch.int32)[::2]):
        with pytest.raises(TypeError):
            nb._labels(bad, 4)
    nb._sizes(torch.zeros(3, dtype=torch.int64), 3)
    for bad in (torch.zeros(3, dtype=torch.int32), torch.zeros(2, dtype=torch.int64)):
        with pytest.raises(TypeError):
            nb._sizes(bad, 3)


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference times the FP64 oracle on the host cores (no GPU)
    # and prints one JSON line carrying the same metric as the GPU arm
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-fit-rows", "2000", "--ref-score-rows", "4000",
                          "--n", "20000"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "files/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["warmup"] >= 3 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] and d["metric"]
