"""CPU-side checks of the CUDA library: it builds, loads and exports every
entry point that include/ declares.  No device work is done here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpe_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2301_08275_gb300 as gpe
    return gpe.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        for name in _declared(header):
            assert name in exported, "%s declared in %s but not exported" % (name, header)


def test_library_loads_and_binding_names_match(libpath):
    import paper_2301_08275_gb300 as gpe
    L = gpe.lib()
    for name in _declared("gpe.h"):
        assert hasattr(L, name)
        assert hasattr(gpe, name), "binding lacks %s" % name
    assert gpe.lib().gpe_last_error() is not None


def test_binding_raises_without_library(tmp_path, monkeypatch):
    import paper_2301_08275_gb300 as gpe
    monkeypatch.setattr(gpe, "_lib", None)
    monkeypatch.setattr(gpe, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        gpe.lib()


def test_desc_layout_matches_header():
    """The ctypes struct mirrors gpe_plan_desc field for field (offsets from a C compile)."""
    import paper_2301_08275_gb300 as gpe
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "gpe.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(gpe_plan_desc),
    offsetof(gpe_plan_desc, ndim), offsetof(gpe_plan_desc, n), offsetof(gpe_plan_desc, lo),
    offsetof(gpe_plan_desc, len), offsetof(gpe_plan_desc, g), offsetof(gpe_plan_desc, dt),
    offsetof(gpe_plan_desc, gamma), offsetof(gpe_plan_desc, prec), offsetof(gpe_plan_desc, batch),
    offsetof(gpe_plan_desc, g_each), offsetof(gpe_plan_desc, gamma_each), offsetof(gpe_plan_desc, V_host));
  return 0; }
'''
    d = "/tmp/gpe_desc_check_%d" % os.getpid()
    os.makedirs(d, exist_ok=True)
    open(os.path.join(d, "c.c"), "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), os.path.join(d, "c.c"), "-o",
                    os.path.join(d, "c")], check=True)
    vals = [int(v) for v in subprocess.run([os.path.join(d, "c")], capture_output=True, text=True,
                                           check=True).stdout.split()]
    D = gpe.gpe_plan_desc
    py = [ctypes.sizeof(D)] + [getattr(D, f).offset for f in
                               ("ndim", "n", "lo", "len", "g", "dt", "gamma", "prec", "batch", "g_each",
                                "gamma_each", "V_host")]
    assert vals == py


def test_product_path_does_not_touch_the_oracle():
    """The library sources and binding never name the oracle package."""
    pkg = os.path.join(ROOT, "paper_2301_08275_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle." not in text, f
