"""The ctypes mirrors of the C-ABI structs have the C sizes (no GPU needed).

A C compiler reports each struct's size from include/diter.h; a field added to or
missing from a Python mirror changes its size and fails here.
"""
import ctypes
import os
import subprocess
import tempfile

import pytest

from paper_1202_6158_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["di_stats", "di_solve_opts", "di_sweep_record", "di_profile", "di_tune_result", "di_batch_tune_result",
           "di_completion", "di_server_graph_stats"]


def c_sizes():
    src = '#include <stdio.h>\n#include "diter.h"\nint main(void) {\n' + "".join(
        f'    printf("{s} %zu\\n", sizeof({s}));\n' for s in STRUCTS) + "    return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "sizes.c"), os.path.join(d, "sizes")
        open(c, "w").write(src)
        r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no C compiler: " + r.stderr[:200])
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_ctypes_mirrors_match_c_sizes():
    sizes = c_sizes()
    for s in STRUCTS:
        assert ctypes.sizeof(getattr(_lib, s)) == sizes[s], s
