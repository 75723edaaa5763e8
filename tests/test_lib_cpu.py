"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/fc.h declares (no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess

import pytest

import paper_1804_04640_gb300 as fc
from paper_1804_04640_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fc_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return fc.load_library()


def test_builds_for_sm103a(lib):
    assert os.path.exists(_build.LIB)
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fc_[a-z_0-9]+)", out))
    assert declared <= exported, declared - exported
    assert declared == set(fc.EXPORTS)
    for name in declared:
        assert hasattr(lib, name)


def test_error_path_without_gpu(lib):
    """Argument errors are reported before any device work."""
    import numpy as np
    with pytest.raises(fc.FcError) as e:
        fc.fc_load(np.zeros((2, 4), dtype=np.uint8), [0, 2])
    assert e.value.code == fc.FC_ERR_ARG
    assert "arity" in fc.fc_last_error()
