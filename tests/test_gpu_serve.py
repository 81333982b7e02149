"""Continuous batching (di_server_*) on the GPU.

Queries on several graphs go through the server's lanes, which are refilled
mid-flight.  Every query is checked against the same query run alone
(di_query_batch with one query): both results are under-approximations of the
same X_q with |X_q - H|_1 <= bound (Theorem 2), so they differ by at most the
sum of the two bounds plus the FP32 fluid rounding.  A sample is also checked
against the FP64 oracle solved alone to bound 1e-12.
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
    return [gg.rmat_graph(10, 16, seed=5), gg.rmat_graph(12, 16, seed=6), gg.zipf_graph(1 << 14, kmax=5000, seed=7)]


def v_of(n, seeds, w=None):
    V = np.zeros(n)
    ww = np.ones(len(seeds)) if w is None else np.asarray(w, float)
    np.add.at(V, np.asarray(seeds), ww / ww.sum())
    return V


def run_stream(di, srv, reqs, burst=7):
    """Submit the requests in bursts with polls in between; returns {ticket: completion}."""
    done = {}
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(srv.submit(r["graph"], r["seeds"], r["tol"], r["out"], r.get("w")))
        if i % burst == burst - 1:
            for c in srv.poll(0.0):
                done[c["ticket"]] = c
    for c in srv.drain(300.0):
        done[c["ticket"]] = c
    return tickets, done


def test_mixed_stream_equals_alone(di, graphs):
    Gs = [di.DiGraph(g.n, g.row_ptr, g.col_idx, D) for g in graphs]
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(150):
        gi = int(rng.integers(0, 3))
        g = graphs[gi]
        seeds = gg.seed_set(g.n, 1, 16, 31 + gi, i)
        tol = float(rng.choice([1e-5, 1e-6, 1e-7]))
        kind = i % 3  # pageable numpy, pinned host tensor, device tensor
        if kind == 0:
            out = np.full(g.n, -1.0)
        elif kind == 1:
            out = torch.full((g.n,), -1.0, dtype=torch.float64).pin_memory()
        else:
            out = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
        reqs.append({"graph": gi, "seeds": seeds, "tol": tol, "out": out})
    with di.DiServer(Gs, round_sweeps=8) as srv:
        assert srv.lanes() == [64, 64, 64]
        tickets, done = run_stream(di, srv, reqs)
    assert len(done) == len(reqs)
    for i, (t, r) in enumerate(zip(tickets, reqs)):
        c = done[t]
        g = graphs[r["graph"]]
        assert c["graph"] == r["graph"] and c["status"] == 0
        assert c["bound"] <= r["tol"]
        assert c["t_submit"] <= c["t_admit"] <= c["t_done"]
        H = r["out"].cpu().numpy() if hasattr(r["out"], "cpu") else r["out"]
        assert np.all(H >= 0)
        Ha, st_a, _ = Gs[r["graph"]].query_batch([r["seeds"]], r["tol"])
        assert np.abs(Ha[0] - H).sum() <= c["bound"] + st_a[0]["bound"] + 2 * FP32_ALLOW
        if i % 15 == 0:
            x = oracle.diter(g.n, g.row_ptr, g.col_idx, D, v_of(g.n, r["seeds"]), 1e-12, mode="sweep")
            assert np.abs(H - x.H).sum() <= c["bound"] + FP32_ALLOW
    for G in Gs:
        G.close()


def test_lanes_refill_under_a_small_budget(di, graphs):
    g = graphs[1]
    G = di.DiGraph(g.n, g.row_ptr, g.col_idx, D)
    lane_bytes = 16 * g.n + 4 * 1024 * 8   # fluid rows may be padded by up to a few scan chunks
    budget = 12 * lane_bytes + 64 * g.n
    with di.DiServer([G], mem_budget=budget, round_sweeps=4) as srv:
        K = srv.lanes()[0]
        assert K in (8, 16)
        reqs = [{"graph": 0, "seeds": gg.seed_set(g.n, 1, 8, 77, i), "tol": 1e-6, "out": np.empty(g.n)}
                for i in range(5 * K)]
        tickets, done = run_stream(di, srv, reqs, burst=3 * K)
        st = srv.stats(0)
    assert st["lanes"] == K and st["admitted"] == st["completed"] == len(reqs)
    assert st["rounds"] >= 1 and st["sweeps"] >= max(c["sweeps"] for c in done.values())
    assert st["edges_pushed"] > 0 and st["device_ms"] > 0
    lanes_used = [done[t]["lane"] for t in tickets]
    assert all(0 <= q < K for q in lanes_used)
    assert len(done) == len(reqs)
    # every lane served several queries one after another
    assert max(np.bincount(lanes_used)) >= 2
    for t, r in zip(tickets, reqs):
        Ha, st_a, _ = G.query_batch([r["seeds"]], 1e-6)
        assert np.abs(Ha[0] - r["out"]).sum() <= done[t]["bound"] + st_a[0]["bound"] + 2 * FP32_ALLOW
    G.close()


def test_cancel_queued_and_running_queries(di, graphs):
    g = graphs[1]
    G = di.DiGraph(g.n, g.row_ptr, g.col_idx, D)
    lane_bytes = 16 * g.n + 4 * 1024 * 8
    budget = 12 * lane_bytes + 64 * g.n
    with di.DiServer([G], mem_budget=budget, round_sweeps=4) as srv:
        K = srv.lanes()[0]
        reqs = [{"graph": 0, "seeds": gg.seed_set(g.n, 1, 8, 78, i), "tol": 1e-7, "out": np.full(g.n, -7.0)}
                for i in range(3 * K)]
        tickets = [srv.submit(0, r["seeds"], r["tol"], r["out"]) for r in reqs]
        srv.poll(0.0)  # the first K queries take the lanes and their first round starts
        assert srv.pending() == (2 * K, K)
        gone = {1, K + 2, 2 * K + 5}  # one running, two queued
        for i in sorted(gone):
            assert srv.cancel(tickets[i])
        assert srv.pending()[0] == 2 * K - 2
        assert not srv.cancel(tickets[1])      # already withdrawn
        assert not srv.cancel(10 ** 12)        # never issued
        done = {c["ticket"]: c for c in srv.drain(120.0)}
        assert not srv.cancel(tickets[0])      # finished
        st = srv.stats(0)
    assert set(done) == {t for i, t in enumerate(tickets) if i not in gone}
    assert st["cancelled"] == 3 and st["admitted"] == 3 * K - 2 and st["completed"] == 3 * K - 3
    for i in gone:
        assert np.all(reqs[i]["out"] == -7.0)  # never written
    # every lane was reused after the cancelled one was cleared: later queries are unaffected
    for i, (t, r) in enumerate(zip(tickets, reqs)):
        if i in gone:
            continue
        Ha, st_a, _ = G.query_batch([r["seeds"]], r["tol"])
        assert done[t]["status"] == 0
        assert np.abs(Ha[0] - r["out"]).sum() <= done[t]["bound"] + st_a[0]["bound"] + 2 * FP32_ALLOW
    G.close()


def test_weighted_query_and_dropped_output(di, graphs):
    g = graphs[0]
    G = di.DiGraph(g.n, g.row_ptr, g.col_idx, D)
    seeds = gg.seed_set(g.n, 3, 9, 90, 0)
    w = np.arange(1, len(seeds) + 1, dtype=float)
    H = np.empty(g.n)
    with di.DiServer([G]) as srv:
        t1 = srv.submit(0, seeds, 1e-7, H, w=w)
        t2 = srv.submit(0, seeds, 1e-7)  # no output buffer: result dropped, completion still reported
        done = {c["ticket"]: c for c in srv.drain(60.0)}
    assert set(done) == {t1, t2}
    x = oracle.diter(g.n, g.row_ptr, g.col_idx, D, v_of(g.n, seeds, w), 1e-12, mode="sweep")
    assert np.abs(H - x.H).sum() <= done[t1]["bound"] + FP32_ALLOW
    G.close()


def test_sweep_limit_reports_not_converged(di, graphs):
    g = graphs[2]
    G = di.DiGraph(g.n, g.row_ptr, g.col_idx, D)
    seeds = gg.seed_set(g.n, 4, 4, 5, 0)
    H = np.empty(g.n)
    with di.DiServer([G], lane_sweeps=2) as srv:
        t = srv.submit(0, seeds, 1e-12, H)
        done = {c["ticket"]: c for c in srv.drain(60.0)}
    c = done[t]
    assert c["status"] == di.DI_ENOTCONVERGED and c["sweeps"] == 2 and c["bound"] > 1e-12
    x = oracle.diter(g.n, g.row_ptr, g.col_idx, D, v_of(g.n, seeds), 1e-12, mode="sweep")
    assert np.abs(H - x.H).sum() <= c["bound"] + FP32_ALLOW
    G.close()


def test_invalid_requests(di, graphs):
    g = graphs[0]
    G = di.DiGraph(g.n, g.row_ptr, g.col_idx, D)
    with di.DiServer([G]) as srv:
        with pytest.raises(di.DiError, match="graph index"):
            srv.submit(1, [0], 1e-6)
        with pytest.raises(di.DiError, match="at least one seed"):
            srv.submit(0, [], 1e-6)
        with pytest.raises(di.DiError, match="seed id"):
            srv.submit(0, [g.n], 1e-6)
        with pytest.raises(di.DiError, match="weights"):
            srv.submit(0, [0, 1], 1e-6, w=[1.0, -1.0])
        with pytest.raises(di.DiError, match="tol"):
            srv.submit(0, [0], 0.0)
        assert srv.pending() == (0, 0)
    with pytest.raises(di.DiError) as e:
        di.DiServer([G], mem_budget=1)
    assert e.value.status == di.DI_ENOMEM
    G.close()
