"""Graph update (Section 3.2) and ALGO-OP / ALGO-OP2 selection (Section 4.3) on the GPU.

Update: a solve on P stopped at some bound continues on the updated graph P'
from F_0' = F + d(P'-P)H (signed fluid).  Its result must be within its bound
of the solution of X = dP'X + (1-d)V (Gaussian elimination, or the oracle run
on P' to 1e-13), and within the sum of the bounds of the oracle's own update
run.  Right after the injection the device state satisfies H + F = F_0 + dP'H.

Selection: DI_SELECT_OP / _OP2 threshold sweeps against the oracle's weighted
snapshot sweeps.  Both take the selection decision in FP32 from the same
weights, so the sweep and elementary-step counts agree; H within 1e-12 at
bound 1e-13.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import ge
from tests import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.85


@pytest.fixture(scope="module")
def di():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_6158_gb300 as di
    di.load()
    return di


def sparse_P(n, rp, ci):
    import scipy.sparse as sp
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    return sp.csr_matrix((1.0 / deg[src], (ci, src)), shape=(n, n))


def update_cases():
    rng = np.random.default_rng(31)
    out = {}
    rp, ci = graphs.random_graph(1500, 0.15, 8, rng)
    out["random_1500"] = (1500, rp, ci) + graphs.modify(1500, rp, ci, rng)
    g = gg.rmat_graph(12, 16, seed=3)
    out["rmat_12"] = (g.n, g.row_ptr, g.col_idx) + graphs.modify(g.n, g.row_ptr, g.col_idx, rng, drop=0.05,
                                                                   add=0.05)
    g = gg.zipf_graph(1 << 14, kmax=5000, seed=2)
    out["zipf_2e14"] = (g.n, g.row_ptr, g.col_idx) + graphs.modify(g.n, g.row_ptr, g.col_idx, rng, drop=0.02,
                                                                     add=0.02)
    return out


CASES = update_cases()


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tol0", [1e-2, 1e-6])
def test_update_reaches_new_fixed_point(di, name, tol0, direction):
    n, rp, ci, rp2, ci2 = CASES[name]
    V = gg.uniform_v(n)
    with di.DiGraph(n, rp, ci, D) as Go, di.DiGraph(n, rp2, ci2, D) as Gn:
        Go.solve(tol0)
        H, st = Gn.update_from(Go, 1e-12, direction=direction)
        F, H2 = Gn.state()
    assert np.array_equal(H, H2)
    assert st["converged"] == 1 and st["bound"] <= 1e-12
    if n <= 1500:
        X2 = ge.pagerank_dense(n, rp2, ci2, D, V)
        assert np.abs(X2 - H).sum() <= st["bound"] + 1e-13
    else:
        r = oracle.diter(n, rp2, ci2, D, V, 1e-13, mode="sweep")
        assert np.abs(r.H - H).sum() <= st["bound"] + r.l1F / (1 - D) + 1e-12
    # the oracle's own update from its own stopping point on P
    r0 = oracle.diter(n, rp, ci, D, V, tol0, mode="sweep")
    r1 = oracle.solve_update(n, rp, ci, rp2, ci2, D, r0.F, r0.H, 1e-12)
    assert np.abs(r1.H - H).sum() <= st["bound"] + r1.l1F / (1 - D) + 1e-12


@pytest.mark.parametrize("direction", [0, 1])
def test_injection_keeps_theorem1_for_new_graph(di, direction):
    n, rp, ci, rp2, ci2 = CASES["zipf_2e14"]
    F0 = (1 - D) * gg.uniform_v(n)
    P2 = sparse_P(n, rp2, ci2)
    with di.DiGraph(n, rp, ci, D) as Go, di.DiGraph(n, rp2, ci2, D) as Gn:
        Go.solve(1e-3)
        for k in (1, 3, 10):
            H, st = Gn.update_from(Go, 1e-14, max_sweeps=k, allow_unconverged=True, direction=direction)
            F, H2 = Gn.state()
            assert st["sweeps"] == k
            if k == 1:
                assert (F < 0).any(), "the injection should leave negative fluid on this graph"
            resid = H2 + F - F0 - D * (P2 @ H2)
            assert np.abs(resid).max() <= 1e-15
            assert st["R"] >= st["l1_F"] * (1 - 1e-12)   # R stays an upper bound on |F|_1


def test_same_graph_continues_the_solve(di):
    n, rp, ci, _, _ = CASES["rmat_12"]
    V = gg.uniform_v(n)
    with di.DiGraph(n, rp, ci, D) as G:
        G.solve(1e-3)
        H, st = G.update_from(G, 1e-12)
    r = oracle.diter(n, rp, ci, D, V, 1e-13, mode="sweep")
    assert np.abs(r.H - H).sum() <= st["bound"] + 1e-12


def test_chained_updates(di):
    n, rp, ci, rp2, ci2 = CASES["random_1500"]
    rng = np.random.default_rng(77)
    rp3, ci3 = graphs.modify(n, rp2, ci2, rng)
    X3 = ge.pagerank_dense(n, rp3, ci3, D, gg.uniform_v(n))
    with di.DiGraph(n, rp, ci, D) as G1, di.DiGraph(n, rp2, ci2, D) as G2, di.DiGraph(n, rp3, ci3, D) as G3:
        G1.solve(1e-2)
        G2.update_from(G1, 1e-4)
        H, st = G3.update_from(G2, 1e-12)
    assert np.abs(X3 - H).sum() <= st["bound"] + 1e-13


def test_update_rejects_mismatches(di):
    n, rp, ci, rp2, ci2 = CASES["random_1500"]
    rpx, cix = graphs.random_graph(n + 1, 0.1, 4, np.random.default_rng(1))
    with di.DiGraph(n, rp, ci, D) as Go, di.DiGraph(n, rp2, ci2, D) as Gn, \
            di.DiGraph(n + 1, rpx, cix, D) as Gx, di.DiGraph(n, rp2, ci2, 0.5) as Gd:
        with pytest.raises(di.DiError, match="no FP64"):
            Gn.update_from(Go, 1e-8)
        Go.solve(1e-3, prec=di.DI_FP32_MIXED)
        with pytest.raises(di.DiError, match="no FP64"):
            Gn.update_from(Go, 1e-8)
        Go.solve(1e-3)
        with pytest.raises(di.DiError, match="same nodes"):
            Gx.update_from(Go, 1e-8)
        with pytest.raises(di.DiError, match="same d"):
            Gd.update_from(Go, 1e-8)


# ------------------------------------------------------------ ALGO-OP / OP2

SEL_CASES = {
    "random_1025": (1025,) + graphs.random_graph(1025, 0.1, 12, np.random.default_rng(7)),
    "rmat_12": (lambda g: (g.n, g.row_ptr, g.col_idx))(gg.rmat_graph(12, 16, seed=3)),
    "zipf_2e14": (lambda g: (g.n, g.row_ptr, g.col_idx))(gg.zipf_graph(1 << 14, kmax=5000, seed=2)),
}


@pytest.mark.parametrize("name", sorted(SEL_CASES))
@pytest.mark.parametrize("sel", ["op", "op2"])
def test_weighted_sweeps_match_oracle(di, name, sel):
    n, rp, ci = SEL_CASES[name]
    V = gg.uniform_v(n)
    with di.DiGraph(n, rp, ci, D) as G:
        H, st = G.solve(1e-13, select=sel)
    r = oracle.diter(n, rp, ci, D, V, 1e-13, mode="sweep", select=sel)
    assert st["converged"] == 1 and st["bound"] <= 1e-13
    assert np.abs(H - r.H).sum() <= 1e-12
    assert st["sweeps"] == r.sweeps
    assert st["edges_pushed"] == r.edges


@pytest.mark.parametrize("sel", ["op", "op2"])
def test_weighted_sweeps_against_elimination(di, sel):
    rng = np.random.default_rng(55)
    n = 250
    rp, ci = graphs.random_graph(n, 0.15, 9, rng)
    V = graphs.random_v(n, rng)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    with di.DiGraph(n, rp, ci, D, V=V) as G:
        H, st = G.solve(1e-12, select=sel)
        H32, st32 = G.solve(1e-9, select=sel, prec=di.DI_FP32_MIXED)
    assert np.abs(X - H).sum() <= st["bound"] + 1e-14
    assert np.all(H <= X + 1e-15)
    assert np.abs(X - H32).sum() <= st32["bound"] + 2e-6


def test_weighted_update(di):
    n, rp, ci, rp2, ci2 = CASES["random_1500"]
    X2 = ge.pagerank_dense(n, rp2, ci2, D, gg.uniform_v(n))
    with di.DiGraph(n, rp, ci, D) as Go, di.DiGraph(n, rp2, ci2, D) as Gn:
        Go.solve(1e-3, select="op")
        H, st = Gn.update_from(Go, 1e-12, select="op2")
    assert np.abs(X2 - H).sum() <= st["bound"] + 1e-13


def test_select_is_validated(di):
    n, rp, ci = SEL_CASES["random_1025"]
    with di.DiGraph(n, rp, ci, D) as G:
        with pytest.raises(di.DiError, match="select"):
            G.solve(1e-6, select=3)


# ------------------------------------------------------------------ autotuner

def test_autotune_picks_a_valid_fastest_candidate(di):
    n, rp, ci = SEL_CASES["zipf_2e14"]
    V = gg.uniform_v(n)
    with di.DiGraph(n, rp, ci, D) as G:
        best, tried = G.autotune(1e-10)
        # 90 combinations of beta, rule, grid and direction, then 4 more class cutoffs
        assert len(tried) == 94
        assert best["ms"] == min(t["ms"] for t in tried if t["ms"] >= 0)
        assert {t["select"] for t in tried} == {0, 1, 2}
        assert {t["push_ctas_per_sm"] for t in tried} == {2, 4, 8}
        assert {t["direction"] for t in tried} == {0, 1}
        assert {(t["cut1"], t["cut2"]) for t in tried} == {(8, 1024), (4, 1024), (8, 256), (8, 4096), (4, 256)}
        assert all(t["ms"] >= 0 for t in tried)  # every candidate converged
        # the winning cutoffs stay on the graph: its classes are the oracle's bins for them
        ex = G.export()
        assert list(ex["cuts"][:2]) == [best["cut1"], best["cut2"]]
        bin_of, _, _ = oracle.bins(n, *relabel_rp(n, rp, ex["perm"]), [0, best["cut1"], best["cut2"]])
        assert np.array_equal(ex["bin_of"], bin_of)
        # the tuned settings give a correct solve
        H, st = G.solve(1e-12, beta=best["beta"], select=best["select"], direction=best["direction"])
    r = oracle.diter(n, rp, ci, D, V, 1e-13, mode="sweep")
    assert np.abs(H - r.H).sum() <= st["bound"] + 1e-12


def relabel_rp(n, rp, perm):
    """(n, row pointers) of the CSR in the numbering perm (row r = input row perm[r])."""
    deg = np.diff(rp)[np.asarray(perm)]
    return (np.concatenate([[0], np.cumsum(deg)]).astype(np.int32),)


@pytest.mark.parametrize("k", [8, 64])
def test_autotune_batch_keeps_the_fastest_valid_candidate(di, k):
    """di_autotune_batch: every candidate batch converges, the fastest is kept and stays set on
    the graph, and a batch run with the tuned settings matches the oracle query by query
    within max(bound) + 2e-6 (FP32 fluid rows)."""
    g = gg.rmat_graph(13, 16, seed=5)
    seeds = gg.seed_sets(g.n, k, 1, 16, seed=9)
    tol = 1e-6
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        best, tried = G.autotune_batch(seeds, tol)
        ok = [t for t in tried if t["ms"] >= 0]
        assert len(ok) == len(tried) >= 12
        assert all(t["max_bound"] <= tol for t in tried)
        assert best["ms"] == min(t["ms"] for t in ok)
        assert {t["pull_share"] for t in tried} == {2, 4, 8, 16}
        assert {t["push_ctas_per_sm"] for t in tried} == {2, 4, 8}
        assert {t["beta"] for t in tried} == {0.25, 0.5, 1.0}
        widths = {t["lanes"] for t in tried}
        assert widths == ({k, 2 * k} if k < 64 else {64})
        ex = G.export()
        assert list(ex["cuts"][:2]) == [best["cut1"], best["cut2"]]
        H, st_q, st_all = G.query_batch(seeds, tol)
        assert st_all["converged"] == 1
    for q in (0, k // 2, k - 1):
        V = np.zeros(g.n)
        np.add.at(V, np.asarray(seeds[q]), 1.0 / len(seeds[q]))
        r = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-12, mode="sweep")
        assert np.abs(H[q] - r.H).sum() <= max(st_q[q]["bound"], r.l1F / (1 - D)) + 2e-6
