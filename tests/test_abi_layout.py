"""The Python binding's ctypes structures have the C layout of include/hdivsp.h.

A plain C program compiled against the header prints sizeof and offsetof of every
field of every structure the binding mirrors; each must equal the ctypes value, so
that a field added, removed or reordered on one side only cannot pass unnoticed."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2304_12387_gb300 as hd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "hd_problem_desc": hd.ProblemDesc,
    "hd_solve_opts": hd.SolveOpts,
    "hd_solve_info": hd.SolveInfo,
    "hd_gmres_opts": hd.GmresOpts,
    "hd_train_opts": hd.TrainOpts,
    "hd_train_info": hd.TrainInfo,
    "hd_slab": hd.Slab,
    "hd_massinv_desc": hd.MassInvDesc,
    "hd_rad_desc": hd.RadDesc,
    "hd_rad_info": hd.RadInfo,
}


def test_ctypes_structures_match_the_c_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hdivsp.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[s, f] = int(v)
    for cname, cls in STRUCTS.items():
        assert got[cname, "sizeof"] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[cname, f] == getattr(cls, f).offset, (cname, f)
