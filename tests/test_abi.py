"""The C ABI library loads on a machine without a GPU, exports every function that
include/imin.h declares, and the binding's struct layouts match the header
(sizes and field offsets printed by a C program compiled against the header)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from conftest import ROOT
from paper_2405_12871_gb300 import _lib

HEADER = os.path.join(ROOT, "include", "imin.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(imin_[a-z_]+)\s*\(", text)))


def test_header_declares_binding_exports():
    assert sorted(_lib.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True,
                         text=True)
    if out.returncode == 0:
        syms = set(line.split()[-1] for line in out.stdout.splitlines() if line.strip())
        for name in _declared():
            assert name in syms, name


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "imin.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("imin_sample_opts size %zu\n", sizeof(imin_sample_opts));
  printf("imin_sample_out size %zu\n", sizeof(imin_sample_out));
  printf("imin_solve_opts size %zu\n", sizeof(imin_solve_opts));
  printf("imin_result size %zu\n", sizeof(imin_result));
  printf("imin_query size %zu\n", sizeof(imin_query));
  F(imin_query, opts); F(imin_query, delta);
  F(imin_sample_opts, first_sample); F(imin_sample_opts, mode);
  F(imin_sample_out, world_spread); F(imin_sample_out, nonempty_lrr);
  F(imin_solve_opts, fixed_theta); F(imin_solve_opts, variant);
  F(imin_result, nVs); F(imin_result, I_hat); F(imin_result, I_after); F(imin_result, n_spread);
  F(imin_result, n_final); F(imin_result, worlds_sampled); F(imin_result, ms_stage);
  F(imin_result, kernel_ms); F(imin_result, kernel_launches);
  F(imin_result, final_kernel_ms); F(imin_result, final_launches);
  return 0;
}
"""


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    lines = subprocess.check_output([str(exe)], text=True).split("\n")
    m = {"imin_sample_opts": _lib.SampleOpts, "imin_sample_out": _lib.SampleOut,
         "imin_solve_opts": _lib.SolveOpts, "imin_result": _lib.Result,
         "imin_query": _lib.Query}
    n = 0
    for line in lines:
        if not line.strip():
            continue
        t, f, v = line.split()
        if f == "size":
            assert C.sizeof(m[t]) == int(v), t
        else:
            assert getattr(m[t], f).offset == int(v), (t, f)
        n += 1
    assert n == 24


def test_no_gpu_reports_device_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(_lib.IminError) as e:
        _lib.imin_create(0)
    assert e.value.code in (_lib.IMIN_EDEVICE, _lib.IMIN_EINVAL)
