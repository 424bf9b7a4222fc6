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


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/sonar.h compiles as C99 (no C++ in the boundary) and a C program
    links against libsonar.so and calls it (only calls that need no GPU: the
    version string and argument errors)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "sonar.h"
int main(void) {
    const char* v = sonar_version();
    if (!v || strncmp(v, "libsonar", 8) != 0) return 1;
    if (sonar_create(0, NULL) != SONAR_ERR_ARG) return 2;          /* NULL out */
    if (sonar_check(NULL, NULL) != SONAR_ERR_ARG) return 3;        /* NULL context */
    if (sonar_philox(NULL, NULL, 0, 0, NULL, NULL) != SONAR_ERR_ARG) return 4;
    if (sizeof(sonar_hit) != 16) return 5;
    puts(v);
    return 0;
}
''')
    exe = tmp_path / "abi"
    libdir = os.path.join(ROOT, "paper_2503_01074_gb300")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lsonar", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("libsonar")
