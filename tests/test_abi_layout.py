"""The ctypes structures of the binding have the C header's layout (no GPU needed).

A small C program, compiled with the host C compiler against include/hom.h, prints sizeof and
offsetof of every field of the ABI structures; each must equal its ctypes counterpart.  A field
added to one side only (an option, a result value) shifts every later field and fails here.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1712_05145_gb300 import hom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [("hom_options", hom.hom_options), ("hom_solve_info", hom.hom_solve_info),
           ("hom_kernel_stat", hom.hom_kernel_stat), ("hom_request", hom.hom_request),
           ("hom_result", hom.hom_result)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hom.h"', "int main(void) {"]
    for name, cls in STRUCTS:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    layout = {}
    for line in out.splitlines():
        a, b, v = line.split()
        layout[(a, b)] = int(v)
    return layout


@pytest.mark.parametrize("name,cls", STRUCTS, ids=[s[0] for s in STRUCTS])
def test_struct_layout_matches_header(c_layout, name, cls):
    assert ctypes.sizeof(cls) == c_layout[(name, "size")], name
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(name, field)], (name, field)


def test_every_option_field_is_bound(c_layout):
    """hom_options ends where the binding's last field ends: no header field is missing."""
    last = hom.hom_options._fields_[-1][0]
    end = getattr(hom.hom_options, last).offset + getattr(hom.hom_options, last).size
    size = c_layout[("hom_options", "size")]
    assert size - end < 8, (end, size)   # at most tail padding
