"""Batched personalized queries (di_query_batch) against the oracle, one query at a time.

Each query q has its own V_q (uniform, or weighted, over its seeds).  The oracle
solves it alone in FP64 to bound 1e-12; the batch uses FP32 fluid rows with FP64
histories, so the bar is |H_q - X_q|_1 <= bound_q + 2e-6 (Theorem 2 plus the FP32
fluid rounding).  A query gives the same answer alone and inside a full batch,
within the sum of the two bounds plus the same FP32 allowance.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.85
FP32_ALLOW = 2e-6


@pytest.fixture(scope="module")
def di():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_6158_gb300 as di
    di.load()
    return di


@pytest.fixture(scope="module")
def graphs():
    return {"rmat12": gg.rmat_graph(12, 16, seed=3), "zipf14": gg.zipf_graph(1 << 14, kmax=5000, seed=2)}


def v_of(n, seeds, w=None):
    V = np.zeros(n)
    ww = np.ones(len(seeds)) if w is None else np.asarray(w, float)
    np.add.at(V, np.asarray(seeds), ww / ww.sum())
    return V


@pytest.mark.parametrize("name", ["rmat12", "zipf14"])
def test_batch_of_64_against_oracle(di, graphs, name):
    g = graphs[name]
    seeds = gg.seed_sets(g.n, 64, 1, 32, seed=21)
    tol = 1e-6
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        H, st_q, st_all = G.query_batch(seeds, tol)
    assert st_all["converged"] == 1
    for q in (0, 1, 17, 40, 63):
        r = oracle.diter(g.n, g.row_ptr, g.col_idx, D, v_of(g.n, seeds[q]), 1e-12, mode="sweep")
        assert st_q[q]["converged"] and st_q[q]["bound"] <= tol
        assert np.abs(H[q] - r.H).sum() <= st_q[q]["bound"] + FP32_ALLOW
        assert np.all(H[q] >= 0)


def test_weighted_seeds(di, graphs):
    g = graphs["rmat12"]
    seeds = gg.seed_sets(g.n, 5, 2, 10, seed=4)
    weights = [np.arange(1, len(s) + 1, dtype=float) for s in seeds]
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        H, st_q, _ = G.query_batch(seeds, 1e-7, weights=weights)
    for q in range(5):
        r = oracle.diter(g.n, g.row_ptr, g.col_idx, D, v_of(g.n, seeds[q], weights[q]), 1e-12, mode="sweep")
        assert np.abs(H[q] - r.H).sum() <= st_q[q]["bound"] + FP32_ALLOW


def test_alone_equals_in_the_mix(di, graphs):
    g = graphs["zipf14"]
    seeds = gg.seed_sets(g.n, 64, 1, 32, seed=8)
    tol = 1e-6
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        Hmix, st_mix, _ = G.query_batch(seeds, tol)
        for q in (3, 30, 60):
            Ha, st_a, _ = G.query_batch([seeds[q]], tol)
            assert np.abs(Ha[0] - Hmix[q]).sum() <= st_a[0]["bound"] + st_mix[q]["bound"] + 2 * FP32_ALLOW


def test_batch_agrees_with_single_queries(di, graphs):
    g = graphs["rmat12"]
    seeds = gg.seed_sets(g.n, 8, 1, 32, seed=9)
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        Hb, st_b, _ = G.query_batch(seeds, 1e-7)
        for q in range(8):
            Hs, st_s = G.query(seeds[q], 1e-9)
            assert np.abs(Hb[q] - Hs).sum() <= st_b[q]["bound"] + st_s["bound"] + FP32_ALLOW


def test_device_output_and_limits(di, graphs):
    g = graphs["rmat12"]
    seeds = gg.seed_sets(g.n, 3, 1, 4, seed=10)
    dev = torch.device("cuda")
    H = torch.empty((3, g.n), dtype=torch.float64, device=dev)
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        G.query_batch(seeds, 1e-6, H_out=H)
        torch.cuda.synchronize()
        Hh, _, _ = G.query_batch(seeds, 1e-6)
        assert np.abs(H.cpu().numpy() - Hh).sum() <= 1e-5
        with pytest.raises(di.DiError):
            G.query_batch([], 1e-6)
        with pytest.raises(di.DiError, match="64"):
            G.query_batch([[1]] * 65, 1e-6)
        with pytest.raises(di.DiError, match="seed"):
            G.query_batch([[g.n + 1]], 1e-6)
        with pytest.raises(di.DiError, match="at least one seed"):
            G.query_batch([[1], []], 1e-6)


def test_profiled_batch_matches_the_captured_loop(di, graphs):
    """profile=1 launches the same sweep kernels from the host with events: the same answers
    within the bounds, one profiled sweep per loop sweep, positive kernel times."""
    g = graphs["rmat12"]
    seeds = gg.seed_sets(g.n, 64, 1, 32, seed=23)
    tol = 1e-6
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        H, st_q, st_all = G.query_batch(seeds, tol)
        Hp, st_qp, st_allp = G.query_batch(seeds, tol, profile=1)
    prof = st_allp["profile"]
    assert "profile" not in st_all
    assert st_allp["converged"] == 1 and all(s["bound"] <= tol for s in st_qp)
    assert prof["sweeps"] == st_allp["sweeps"]
    assert 0 <= prof["pull_sweeps"] <= prof["sweeps"]
    assert prof["scan_ms"] > 0 and prof["push_ms"] > 0 and prof["finalize_ms"] > 0
    for q in range(64):
        assert np.abs(H[q] - Hp[q]).sum() <= st_q[q]["bound"] + st_qp[q]["bound"] + 2 * FP32_ALLOW
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        with pytest.raises(di.DiError, match="profile"):
            di.di_query_batch_ex(G.handle, seeds[:2], tol, np.empty((2, g.n)), profile=2)
