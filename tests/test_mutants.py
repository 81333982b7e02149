"""Plant plausible mistakes in copies of the oracle and check the pins catch each.

Each mutant is oracle.c with one textual change (a dropped term, a wrong sign,
a transposed operand, a wrong degree), compiled with gcc into a temporary
library.  A battery of the pins of test_oracle_pins.py must fail for every
mutant and pass for the unmodified source.  Everything runs on the CPU.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import ge
from tests import graphs

D = 0.85

MUTANTS = {
    "push_drops_d": ("F[col_idx[e]] += sent * p * d;", "F[col_idx[e]] += sent * p;"),
    "dangling_keeps_mass": ("        *R -= fabs(sent);\n", "        *R -= fabs(sent) * (1.0 - d);\n"),
    "history_not_updated": ("    H[i] += sent;\n    F[i] = 0.0;", "    F[i] = 0.0;"),
    "residual_wrong_factor": ("        *R -= fabs(sent) * (1.0 - d);\n    }", "        *R -= fabs(sent) * d;\n    }"),
    "degree_off_by_one": ("double p = 1.0 / (double)(end - beg);", "double p = 1.0 / (double)(end - beg + 1);"),
    "power_transposed": ("Y[col_idx[e]] += d * p * X[i];", "Y[i] += d * p * X[col_idx[e]];"),
    "sweep_reads_after_push": ("                sent[k] = F[i];\n                H[i] += sent[k];\n                F[i] = 0.0;\n",
                               "                sent[k] = F[i];\n                H[i] += sent[k];\n"),
    "sweep_skips_dangling": ("                    R -= fabs(sent[k]);\n", "                    R -= 0.0;\n"),
    "init_wrong_scale": ("F[i] = (1.0 - d) * V[i];", "F[i] = V[i];"),
    "transpose_order": ("in_src[fill[col_idx[e]]++] = i;", "in_src[fill[col_idx[e]]++] = col_idx[e];"),
    "update_wrong_sign": ("F[ci_old[e]] -= H[i] * p * d;", "F[ci_old[e]] += H[i] * p * d;"),
    "update_drops_d": ("F[ci_new[e]] += H[i] * p * d;", "F[ci_new[e]] += H[i] * p;"),
    "signed_fluid_never_selected": ("if (!wsel) return fabs(f) > T;", "if (!wsel) return f > T;"),
    "op_argmax_ignores_weight": ("return wsel ? fabs(F[i]) * (double)wsel[i] : fabs(F[i]);", "return fabs(F[i]);"),
    "op_sweep_ignores_scale": ("float t = (float)(T * wscale);", "float t = (float)T;"),
    "op_threshold_raised": ("else if (wsel) T = fmin(T, beta * R / (double)n);", "else if (wsel) T = beta * R / (double)n;"),
    "outdeg_off_by_one": ("outdeg[i] = row_ptr[i + 1] - row_ptr[i];", "outdeg[i] = row_ptr[i + 1] - row_ptr[i] - 1;"),
    "outdeg_next_row": ("outdeg[i] = row_ptr[i + 1] - row_ptr[i];",
                        "outdeg[i] = row_ptr[i + (i + 1 < n ? 2 : 1)] - row_ptr[i + (i + 1 < n ? 1 : 0)];"),
}


def _battery(lib):
    """True when every pin holds for the library `lib`."""
    rng = np.random.default_rng(77)
    n = 40
    rp, ci = graphs.random_graph(n, 0.2, 6, rng)
    V = graphs.random_v(n, rng)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    P = ge.transition_matrix(n, rp, ci)
    ok = True
    for mode in ["per", "sweep", "thresh"]:
        r = oracle.diter(n, rp, ci, D, V, 1e-10, mode=mode, max_pushes=200000, lib=lib)
        ok &= bool(r.converged)
        ok &= bool(np.abs(X - r.H).sum() <= r.l1F / (1 - D) + 1e-14)
        ok &= bool(abs(r.R - r.l1F) < 1e-14)
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode=mode, max_pushes=30, lib=lib)
        ok &= bool(np.abs(r.H + r.F - (1 - D) * V - D * P @ r.H).max() < 1e-15)
        # within a sweep (or fewer than N picks) R is the decremented value of ALGO-REF
        ok &= bool(abs(r.R - r.l1F) < 1e-15)
    # graph update (Section 3.2): F_0' = F + d(P'-P)H, then continue on P' with signed fluid
    rp2, ci2 = graphs.modify(n, rp, ci, np.random.default_rng(5))
    X2 = ge.pagerank_dense(n, rp2, ci2, D, V)
    P2 = ge.transition_matrix(n, rp2, ci2)
    r0 = oracle.diter(n, rp, ci, D, V, 1e-3, mode="sweep", max_pushes=200000, lib=lib)
    Fi = oracle.update(n, rp, ci, rp2, ci2, D, r0.F, r0.H, lib=lib)
    ok &= bool(np.abs(r0.H + Fi - (1 - D) * V - D * P2 @ r0.H).max() < 1e-15)
    for mode in ["sweep", "max"]:
        r1 = oracle.solve_update(n, rp, ci, rp2, ci2, D, r0.F, r0.H, 1e-10, mode=mode, max_pushes=200000, lib=lib)
        ok &= bool(r1.converged and np.abs(X2 - r1.H).sum() <= r1.l1F / (1 - D) + 1e-13)
        ok &= bool(r1.R >= r1.l1F - 1e-15)
    # ALGO-OP / OP2 (Section 4.3): first argmax pick, first weighted sweep, convergence
    F0 = (1 - D) * V
    rph, cih = graphs.hub_graph(80, 3, np.random.default_rng(0))
    Vh = graphs.random_v(80, np.random.default_rng(1))
    for sel in ("op", "op2"):
        tr = np.zeros((100000, 3))
        r = oracle.diter(80, rph, cih, D, Vh, 1e-10, mode="sweep", max_pushes=400000, lib=lib, select=sel, trace=tr)
        ok &= bool(r.converged and np.all(np.diff(tr[:r.sweeps, 0]) <= 0))
        w, wscale = oracle.selection_weights(n, rp, ci, sel)
        i_star = int(np.argmax(np.abs(F0) * w.astype(np.float64)))
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode="max", max_pushes=1, lib=lib, select=sel)
        ok &= np.flatnonzero(r.H).tolist() == [i_star]
        S1 = np.flatnonzero(np.float32(np.abs(F0)) * w > np.float32(0.5 * (1 - D) / n * wscale))
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode="sweep", max_pushes=1, lib=lib, select=sel)
        ok &= np.flatnonzero(r.H).tolist() == S1.tolist()
        r = oracle.diter(n, rp, ci, D, V, 1e-10, mode="sweep", max_pushes=200000, lib=lib, select=sel)
        ok &= bool(r.converged and np.abs(X - r.H).sum() <= r.l1F / (1 - D) + 1e-14)
    Xp, it, delta, conv = oracle.power(n, rp, ci, D, V, 1e-11, lib=lib)
    ok &= bool(conv and np.abs(X - Xp).sum() <= 1e-11)
    in_ptr, in_src = oracle.transpose(n, rp, ci, lib=lib)
    want = [i for _j, i in sorted((int(j), i) for i in range(n) for j in ci[rp[i]:rp[i + 1]])]
    ok &= in_src.tolist() == want
    # out-degrees against a count of the sources in an edge list
    edges = [(int(i), int(j)) for i, j in np.random.default_rng(9).integers(0, 30, (120, 2))] + [(29, 29)]
    rpe, _cie = graphs.csr(30, edges)
    ok &= oracle.outdeg(30, rpe, lib=lib).tolist() == [sum(1 for i, _j in edges if i == k) for k in range(30)]
    return ok


def _compile(src_text, tmp_path, name):
    src = tmp_path / f"{name}.c"
    src.write_text(src_text)
    out = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(out), str(src),
                    "-lm"], check=True)
    return oracle.load(str(out))


def test_unmodified_oracle_passes_battery():
    assert _battery(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    text = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    lib = _compile(text.replace(old, new), tmp_path, name)
    assert not _battery(lib), f"mutant {name} survived the pins"
