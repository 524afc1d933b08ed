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


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "hpfmm.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("hpfmm_options size %zu\n", sizeof(hpfmm_options));
  F(hpfmm_options, prec); F(hpfmm_options, tau_fp64); F(hpfmm_options, levels);
  F(hpfmm_options, subtree_levels); F(hpfmm_options, m2l_mode); F(hpfmm_options, adaptive);
  F(hpfmm_options, async_update); F(hpfmm_options, reserved); F(hpfmm_options, root_x0); F(hpfmm_options, root_side);
  printf("hpfmm_plan_info size %zu\n", sizeof(hpfmm_plan_info));
  F(hpfmm_plan_info, n); F(hpfmm_plan_info, levels); F(hpfmm_plan_info, p);
  F(hpfmm_plan_info, prec); F(hpfmm_plan_info, x0); F(hpfmm_plan_info, side);
  F(hpfmm_plan_info, workspace_bytes);
  printf("hpfmm_tuning size %zu\n", sizeof(hpfmm_tuning));
  F(hpfmm_tuning, p); F(hpfmm_tuning, levels); F(hpfmm_tuning, subtree_levels);
  F(hpfmm_tuning, met); F(hpfmm_tuning, mean_leaf); F(hpfmm_tuning, est_rel_err);
  F(hpfmm_tuning, ms_per_eval); F(hpfmm_tuning, nsample);
  printf("hpfmm_alu_peaks size %zu\n", sizeof(hpfmm_alu_peaks));
  F(hpfmm_alu_peaks, sms); F(hpfmm_alu_peaks, mufu_ops_per_s);
  F(hpfmm_alu_peaks, ffma_flops_per_s); F(hpfmm_alu_peaks, dfma_flops_per_s);
  F(hpfmm_alu_peaks, mufu_mhz); F(hpfmm_alu_peaks, ffma_mhz); F(hpfmm_alu_peaks, dfma_mhz);
  F(hpfmm_alu_peaks, mufu_per_clk_sm); F(hpfmm_alu_peaks, ffma_flops_per_clk_sm);
  F(hpfmm_alu_peaks, dfma_flops_per_clk_sm);
  return 0;
}
"""


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the option, plan-info and tuning structs have the
    C compiler's sizes and field offsets for include/hpfmm.h."""
    import ctypes
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    c = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        t, f, v = line.split()
        c[(t, f)] = int(v)
    for cname, py in (("hpfmm_options", hp.Options), ("hpfmm_plan_info", hp.PlanInfo),
                      ("hpfmm_tuning", hp.Tuning), ("hpfmm_alu_peaks", hp.AluPeaks)):
        assert ctypes.sizeof(py) == c[(cname, "size")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == c[(cname, f)], (cname, f)


def test_adaptive_option_checks_without_gpu(library):
    """Argument checks of the adaptive tree come before any device work."""
    import numpy as np
    x = np.array([0.1, 0.2]); y = np.array([0.3, 0.4])
    with pytest.raises(hp.HpfmmError) as e:
        hp.hpfmm_create(x, y, prec="fp64", adaptive=True)
    assert e.value.status == hp.HPFMM_EUNSUPPORTED
    with pytest.raises(hp.HpfmmError) as e:
        hp.hpfmm_create(x, y, prec="fp32", levels=14, adaptive=True)
    assert e.value.status == hp.HPFMM_EINVAL
    with pytest.raises(hp.HpfmmError) as e:
        hp.hpfmm_create(x, y, prec="fp32", p=32, adaptive=True)
    assert e.value.status == hp.HPFMM_EUNSUPPORTED
    opt = hp.Options()
    library.hpfmm_default_options(__import__("ctypes").byref(opt))
    assert opt.adaptive == 0 and opt.async_update == 0 and list(opt.reserved) == [0]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library every entry point raises."""
    import numpy as np
    monkeypatch.setattr(hp, "_LIB", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent" / "libhpfmm.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hp.lib()
    with pytest.raises(RuntimeError, match="not built"):
        hp.hpfmm_create(np.zeros(4), np.ones(4), kappa=1.0, p=8)
