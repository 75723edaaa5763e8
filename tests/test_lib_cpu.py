"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/fc.h declares (no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess

import numpy as np
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


def test_binding_table_offsets_match_products():
    """The binding's packed table offsets (the product of the arities of each
    list, back to back; an empty list is the one-cell table) for lists with
    empty ones anywhere, at the end included, and ids the library would
    reject counted as arity 1."""
    rng = np.random.default_rng(5)
    ar = rng.integers(1, 41, size=9)
    for trial in range(200):
        lists = []
        for _ in range(int(rng.integers(1, 12))):
            k = int(rng.integers(0, 4))
            lists.append([int(x) for x in rng.choice(9, size=k, replace=False)])
        if trial % 3 == 0:
            lists.append([])
        if trial % 7 == 0:
            lists.insert(0, [])
        off, flat = fc.pack_lists(lists)
        got = fc._table_offsets(ar, off, flat)
        want = np.concatenate([[0], np.cumsum([int(np.prod([ar[v] for v in q])) for q in lists])])
        assert np.array_equal(got, want), lists
    off, flat = fc.pack_lists([[0, 99], [], [-3]])
    assert fc._table_offsets(ar, off, flat).tolist() == [0, int(ar[0]), int(ar[0]) + 1, int(ar[0]) + 2]
