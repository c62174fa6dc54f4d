"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/rgmres.h declares; without a GPU its calls fail loudly (no CPU
fallback).  No compute runs here."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(rgm_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1807_09467_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rgm_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = declared - exported
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_1807_09467_gb300 import _lib
    assert _declared() == set(_lib.EXPORTED)


def test_loads_and_fails_loudly_without_gpu(libpath):
    import torch
    import paper_1807_09467_gb300 as rg
    from paper_1807_09467_gb300 import _lib
    L = _lib.load()
    assert L.rgm_status_string(-3) == b"CUDA error"
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rg.RgmError) as e:
        rg.Solver(100)
    assert e.value.code == _lib.RGM_E_CUDA
