"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every symbol include/sonar.h declares, and its struct layouts match the
binding's.  No compute calls (there is no GPU here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_01074_gb300.build import build
    from paper_2503_01074_gb300 import sonar
    build()
    return sonar.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sonar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sonar_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2503_01074_gb300 import sonar
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
    assert sorted(sonar.exported_symbols()) == names


def test_only_api_symbols_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2503_01074_gb300",
                                                                     "libsonar.so")],
                         capture_output=True, text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if l.strip()]
    leaked = [s for s in syms if s.startswith("cuda") or s.startswith("cu")]
    assert not leaked, leaked[:10]


def test_struct_layouts():
    from paper_2503_01074_gb300 import sonar
    assert C.sizeof(sonar.Sensor) == 80
    assert C.sizeof(sonar.Params) == 32
    assert C.sizeof(sonar.Outputs) == 48
    assert C.sizeof(sonar.BatchItem) == 136
    assert sonar.BatchItem.seed.offset == 96
    assert C.sizeof(sonar.BatchOutputs) == 40
    assert sonar.HIT_DTYPE.itemsize == 16


def test_version_and_no_device_behaviour(lib):
    assert b"sm_103a" in lib.sonar_version()
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.sonar_create(0, C.byref(h)) != 0          # no device: an error, not a crash
    assert lib.sonar_destroy(None) == 0
    assert lib.sonar_last_error(None) == b""


def test_product_path_has_no_cpu_fallback(tmp_path, monkeypatch):
    from paper_2503_01074_gb300 import sonar
    monkeypatch.setattr(sonar, "_LIB", None)
    with pytest.raises(ImportError):
        sonar.load_library(str(tmp_path / "missing.so"))
    # the package never imports the oracle
    pkg = os.path.join(ROOT, "paper_2503_01074_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, flags=re.M), f
