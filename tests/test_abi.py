"""The C-ABI library loads without a GPU and exports every entry point that
include/hpfmm.h declares; host-side argument checks need no GPU either."""
import os
import re
import subprocess

import pytest

import paper_2507_21913_gb300 as hp
from paper_2507_21913_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(hpfmm_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def library():
    _build.build()
    return hp.lib()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("hpfmm_create", "hpfmm_eval", "hpfmm_destroy", "hpfmm_direct",
              "hpfmm_status_string", "hpfmm_last_error", "hpfmm_get_order"):
        assert n in names


def test_library_exports_every_declared_symbol(library):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hpfmm_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing
    for n in _declared():
        assert hasattr(library, n)


def test_status_strings_and_version(library):
    assert hp.hpfmm_version().startswith("hpfmm")
    for s in range(6):
        assert library.hpfmm_status_string(s)


def test_create_rejects_bad_arguments_without_gpu(library):
    import numpy as np
    x = np.array([0.1, 0.2]); y = np.array([0.3, 0.4])
    with pytest.raises(hp.HpfmmError) as e:
        hp.hpfmm_create(x, y, kappa=-1.0)
    assert e.value.status == hp.HPFMM_EINVAL
    with pytest.raises(hp.HpfmmError) as e:
        hp.hpfmm_create(x, y, kappa=1.0 - 0.5j)
    assert e.value.status == hp.HPFMM_EINVAL
    with pytest.raises(hp.HpfmmError) as e:
        hp.hpfmm_create(x, y, kappa=1.0, p=0)
    assert e.value.status == hp.HPFMM_EINVAL
