"""The Python binding's ctypes structures against the C headers: a small C program (built with the
host compiler) prints sizeof and every field's offset of the C ABI structs, which must equal the
ctypes layout field by field -- so an appended or reordered field in either cannot drift silently."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))

PAIRS = [("Desc", "qtx_rgf_desc"), ("Inputs", "qtx_rgf_inputs"), ("Outputs", "qtx_rgf_outputs"),
         ("WInputs", "qtx_w_inputs"), ("WOutputs", "qtx_w_outputs")]


def _c_layout(tmp_path, q):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qtx_rgf.h"', '#include "qtx_kernels.h"',
             "int main(void) {"]
    for py, c in PAIRS:
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(q, py)._fields_:
            lines.append(f'  printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_ctypes_structs_match_the_headers(tmp_path):
    import paper_2606_25595_gb300 as q
    c = _c_layout(tmp_path, q)
    for py, _ in PAIRS:
        S = getattr(q, py)
        assert c[(py, "size")] == ctypes.sizeof(S), py
        for name, _ in S._fields_:
            assert c[(py, name)] == getattr(S, name).offset, (py, name)
