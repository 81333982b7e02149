"""The DI_DEBUG build (libditer_debug.so) on the GPU.

Its sweep kernels check the indices they compute (scan list appends against their
warp's region, the push's list positions and node ids, pushed-to columns and pull
link endpoints against [0, n)) and report a failed check as DI_EKERNEL.  Here the
debug build runs in a child process (DI_LIB_VARIANT=debug): its self-test records
one failure from a kernel that touches no memory and must see it reported, and
solves of several graph families, in both precisions and both sweep directions,
must pass every check and agree with the oracle as the release build does.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import graphgen as gg
import oracle
import paper_1202_6158_gb300 as di
from paper_1202_6158_gb300 import build
build.build(debug=True)
out = {"debug_build": di.di_debug_build()}
out["selftest"] = [list(di.di_debug_selftest()) for _ in range(2)]
D = 0.85
cases = {"uniform": gg.uniform_graph(3000, 12, seed=3), "zipf_hubs": gg.zipf_graph(1 << 14, kmax=5000, seed=2),
         "rmat": gg.rmat_graph(12, 16, seed=4)}
res = {}
for name, g in cases.items():
    V = gg.uniform_v(g.n)
    ref = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-13, mode="sweep")
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        for direction in (0, 1):
            H, st = G.solve(1e-13, direction=direction)
            res[f"{name}/fp64/{direction}"] = [float(np.abs(H - ref.H).sum()), st["sweeps"], ref.sweeps,
                                              st["edges_pushed"], ref.edges]
            H, st = G.solve(1e-10, prec=di.DI_FP32_MIXED, direction=direction)
            res[f"{name}/fp32/{direction}"] = [float(np.abs(H - ref.H).sum()), st["bound"]]
        seeds = gg.seed_set(g.n, 1, 8, 9, 0)
        Hq, stq = G.query(seeds, 1e-10)
        Vq = np.zeros(g.n)
        np.add.at(Vq, seeds, 1.0 / len(seeds))
        rq = oracle.diter(g.n, g.row_ptr, g.col_idx, D, Vq, 1e-13, mode="sweep")
        res[f"{name}/query"] = [float(np.abs(Hq - rq.H).sum()), stq["bound"]]
out["solves"] = res
print("JSON" + json.dumps(out))
"""


def test_debug_build_checks_pass_and_report():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, DI_LIB_VARIANT="debug")
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("JSON")]
    assert p.returncode == 0 and lines, p.stdout[-2000:] + p.stderr[-4000:]
    out = json.loads(lines[-1][4:])
    assert out["debug_build"] is True
    word = (99 << 48) | 12345
    # reported every time, and cleared after each report (the solves below see no failure)
    assert out["selftest"] == [[6, word], [6, word]]
    for key, v in out["solves"].items():
        if "/fp64/" in key:
            err, sweeps, osweeps, edges, oedges = v
            assert err <= 1e-12 and sweeps == osweeps and edges == oedges, (key, v)
        else:
            err, bound = v
            assert err <= bound + 1e-12 + (2e-6 if "/fp32/" in key else 0.0), (key, v)
