"""Host-side checks of the CUDA library that need no GPU: it builds, loads,
and exports every entry point include/vsbpp.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "vsbpp.h")).read()
    return sorted(set(re.findall(r"\b(vsbpp_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_binding_agree():
    from paper_1602_08735_gb300 import native
    assert sorted(native.EXPORTS) == declared_symbols()


def test_library_builds_and_exports_everything():
    from paper_1602_08735_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vsbpp_[a-z_0-9]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"not exported: {missing}"


def test_library_loads_without_gpu():
    from paper_1602_08735_gb300 import native
    lib = native.load()
    assert lib.vsbpp_version() == 10100
    assert native.strerror(-2).startswith("an item is heavier")
