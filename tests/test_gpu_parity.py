"""Parity of the CUDA path (through the C ABI) with the oracle, on seeded synthetic graphs.

Bars (written in each test):
  * CSR-derived structures (out-degrees, in-link lists, degree bins): bit-exact.
  * FP64 D-iteration vs the oracle's snapshot sweeps with the same threshold
    schedule: |H_gpu - H_oracle|_1 <= 1e-12 when both run to bound <= 1e-13,
    and <= max(bounds) + 1e-12 at looser targets (both under-approximate X,
    Theorem 2).  The sweep count and the elementary-step count agree exactly.
  * FP32-mixed D-iteration: |H - H_oracle|_1 <= 2e-6.
  * Power iteration: same number of products and |X - X_oracle|_1 <= 1e-12.
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
BETA = 0.5


@pytest.fixture(scope="module")
def di():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_6158_gb300 as di
    di.load()
    return di


def case_graphs():
    rng = np.random.default_rng(7)
    out = {}
    g = gg.uniform_graph(10000, 20, seed=1)
    out["uniform_1e4"] = (g.n, g.row_ptr, g.col_idx)
    g = gg.zipf_graph(1 << 14, kmax=5000, seed=2)
    out["zipf_2e14_hubs"] = (g.n, g.row_ptr, g.col_idx)
    g = gg.rmat_graph(12, 16, seed=3)
    out["rmat_12"] = (g.n, g.row_ptr, g.col_idx)
    rp, ci = graphs.star(3000)
    out["star_3000"] = (3001, rp, ci)
    rp, ci = graphs.csr(5000, [(i, 4999) for i in range(4999)] + [(4999, 0)])
    out["in_hub_5000"] = (5000, rp, ci)
    rp, ci = graphs.random_graph(1025, 0.1, 12, rng)
    out["random_1025_multi"] = (1025, rp, ci)
    rp, ci = graphs.complete(50)
    out["complete_50"] = (50, rp, ci)
    out["empty_7"] = (7, np.zeros(8, np.int32), np.zeros(0, np.int32))
    # in-degree ties at the hot-target cutoff spread over many id blocks: 100 targets with 50
    # in-links, then 2858 (every 7th id) with exactly 40; the 156 lowest of those are hot
    n = 20011
    tgt = [(j, 50) for j in range(3, n, 197)][:100]
    taken = {j for j, _ in tgt}
    tgt += [(j, 40) for j in range(0, n, 7) if j not in taken]
    edges = [(int(src), j) for j, c in tgt for src in rng.choice(n, c, replace=False)]
    rp, ci = graphs.csr(n, edges)
    out["ties_20011"] = (n, rp, ci)
    return out


CASES = case_graphs()


# ------------------------------------------------------------- graph ingest

def relabel(n, rp, ci, perm):
    """The CSR in the numbering perm (row r = input row perm[r], targets mapped, order kept)."""
    new_of = np.empty(n, np.int64)
    new_of[perm] = np.arange(n)
    deg = np.diff(rp)[perm]
    rp2 = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    ci2 = np.concatenate([new_of[ci[rp[i]:rp[i + 1]]] for i in perm] or [np.zeros(0, np.int64)]).astype(np.int32)
    return rp2, ci2


def expected_hot(n, ci):
    """Top-256 in-degree (at least 32), largest first, ties by lower id."""
    indeg = np.bincount(ci, minlength=n)
    order = np.lexsort((np.arange(n), -indeg))[:256]
    return order[indeg[order] >= 32]


@pytest.mark.parametrize("name", sorted(CASES))
def test_derived_structures_bit_exact(di, name):
    """Internal numbering (hot targets first, then input order), degrees, in-link lists, bins."""
    n, rp, ci = CASES[name]
    with di.DiGraph(n, rp, ci, D) as g:
        ex = g.export()
    c1, c2, ic1, ic2 = ex["cuts"].tolist()
    hot = expected_hot(n, ci)
    rest = np.setdiff1d(np.arange(n), hot)
    perm = np.concatenate([hot, rest]).astype(np.int32)
    assert np.array_equal(ex["perm"], perm)
    rp, ci = relabel(n, rp, ci, perm)
    assert np.array_equal(ex["outdeg"], oracle.outdeg(n, rp))
    in_ptr, in_src = oracle.transpose(n, rp, ci)
    assert np.array_equal(ex["in_ptr"], in_ptr)
    assert np.array_equal(ex["in_src"], in_src)
    bin_of, _, _ = oracle.bins(n, rp, [0, c1, c2])
    assert np.array_equal(ex["bin_of"], bin_of)
    in_bin_of, _, _ = oracle.bins(n, in_ptr, [ic1, ic2])
    assert np.array_equal(ex["in_bin_of"], in_bin_of)


def test_host_and_device_inputs_build_the_same_graph(di):
    """A host col_idx is copied in pieces overlapped with the in-degree count; a device one is
    copied whole: the derived structures are the same."""
    n, rp, ci = CASES["zipf_2e14_hubs"]
    with di.DiGraph(n, rp, ci, D) as gh, \
            di.DiGraph(n, torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), D) as gd:
        eh, ed = gh.export(), gd.export()
        assert np.array_equal(gh.hot_targets(), gd.hot_targets())
    for k in eh:
        assert np.array_equal(eh[k], ed[k]), k


@pytest.mark.parametrize("name", sorted(CASES))
def test_hot_targets_bit_exact(di, name):
    """The push's shared-memory targets: top-256 in-degree (>= 32), ties by lower id."""
    n, rp, ci = CASES[name]
    with di.DiGraph(n, rp, ci, D) as g:
        hot = g.hot_targets()
    assert np.array_equal(hot, expected_hot(n, ci))


# ------------------------------------------------------------ D-iteration

def _solve(di, n, rp, ci, tol, V=None, **kw):
    with di.DiGraph(n, rp, ci, D, V=V) as g:
        H, st = g.solve(tol, beta=kw.pop("beta", BETA), **kw)
        F, H2 = g.state()
        tr = g.trace() if kw.get("trace") else None
    assert np.array_equal(H, H2)
    return H, F, st, tr


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_tight_parity_with_oracle_sweeps(di, name, direction):
    """Both to bound <= 1e-13: |H_gpu - H_oracle|_1 <= 1e-12, same sweeps and elementary steps.
    direction=1 pulls along the in-links on dense sweeps: the same diffusion of the same sets;
    direction=2 does the same after pausing the loop to build the in-link CSR."""
    n, rp, ci = CASES[name]
    V = gg.uniform_v(n)
    tol = 1e-13
    H, F, st, _ = _solve(di, n, rp, ci, tol, direction=direction)
    r = oracle.diter(n, rp, ci, D, V, tol, mode="sweep", beta=BETA)
    assert st["converged"] == 1 and st["bound"] <= tol
    assert abs(st["l1_F"] - np.abs(F).sum()) <= 1e-15 + 1e-12 * st["l1_F"]
    assert np.abs(H - r.H).sum() <= 1e-12
    assert st["sweeps"] == r.sweeps
    assert st["edges_pushed"] == r.edges
    assert st["sources_pushed"] == r.pushes
    assert np.all(F >= 0) and np.all(H >= 0)


def test_config1_target_and_order_independence(di):
    """Uniform-degree graph, d=0.85, V=1/N, stop at |F|_1 < 1e-10: within bounds of every oracle order."""
    n, rp, ci = CASES["uniform_1e4"]
    V = gg.uniform_v(n)
    tol = 1e-10 / (1 - D)
    H, F, st, _ = _solve(di, n, rp, ci, tol)
    assert st["l1_F"] < 1e-10
    for mode in ["sweep", "thresh", "per", "rand"]:
        r = oracle.diter(n, rp, ci, D, V, tol, mode=mode, beta=BETA, seed=5)
        assert np.abs(H - r.H).sum() <= max(st["bound"], r.l1F / (1 - D)) + 1e-12, mode


@pytest.mark.parametrize("seed", range(4))
def test_against_gaussian_elimination(di, seed):
    """Small graphs with multi-edges, self-loops, dangling nodes: |X - H|_1 <= bound, 0 <= H <= X."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 300))
    rp, ci = graphs.random_graph(n, 0.15, 9, rng)
    V = graphs.random_v(n, rng)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    H, F, st, _ = _solve(di, n, rp, ci, 1e-12, V=V)
    assert np.abs(X - H).sum() <= st["bound"] + 1e-14
    assert np.all(H <= X + 1e-15)


@pytest.mark.parametrize("d", [0.01, 0.5, 0.99])
def test_damping_extremes_against_elimination(di, d):
    """d near 0 (almost no diffusion: H is close to (1-d)V after a sweep or two) and d near 1
    (about ln(1e-12)/ln(d) sweeps): |X - H|_1 <= bound and 0 <= H <= X against dense
    elimination, for both sweep directions."""
    rng = np.random.default_rng(77)
    n = 300
    rp, ci = graphs.random_graph(n, 0.1, 12, rng)
    V = graphs.random_v(n, rng)
    X = ge.pagerank_dense(n, rp, ci, d, V)
    for direction in (0, 1):
        with di.DiGraph(n, rp, ci, d, V=V) as g:
            H, st = g.solve(1e-12, beta=BETA, direction=direction)
        assert st["converged"] == 1
        assert np.abs(X - H).sum() <= st["bound"] + 1e-14
        assert np.all(H >= 0) and np.all(H <= X + 1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 1023, 1024, 1025, 4097, 70001])
def test_ragged_sizes(di, n):
    rng = np.random.default_rng(n)
    rp, ci = graphs.random_graph(n, 0.1, 6, rng)
    V = gg.uniform_v(n)
    H, F, st, _ = _solve(di, n, rp, ci, 1e-13)
    r = oracle.diter(n, rp, ci, D, V, 1e-13, mode="sweep", beta=BETA)
    assert np.abs(H - r.H).sum() <= 1e-12
    assert st["sweeps"] == r.sweeps


@pytest.mark.parametrize("direction", [0, 1])
def test_theorem1_on_device_state(di, direction):
    """After k sweeps the device state satisfies H + F = F_0 + dPH (Theorem 1), for both directions."""
    import scipy.sparse as sp
    n, rp, ci = CASES["zipf_2e14_hubs"]
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    P = sp.csr_matrix((1.0 / deg[src], (ci, src)), shape=(n, n))
    F0 = (1 - D) * gg.uniform_v(n)
    for k in [1, 2, 5, 20]:
        H, F, st, _ = _solve(di, n, rp, ci, 1e-14, max_sweeps=k, allow_unconverged=True, direction=direction)
        assert st["sweeps"] == k
        resid = H + F - F0 - D * (P @ H)
        assert np.abs(resid).max() <= 1e-15
        r = oracle.diter(n, rp, ci, D, gg.uniform_v(n), 0.0, mode="sweep", beta=BETA, max_pushes=st["sources_pushed"])
        assert np.abs(H - r.H).sum() <= 1e-13
        assert np.abs(F - r.F).sum() <= 1e-13


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_trace_records(di, direction):
    n, rp, ci = CASES["rmat_12"]
    H, F, st, tr = _solve(di, n, rp, ci, 1e-10, trace=1, direction=direction)
    assert len(tr) == st["sweeps"]
    # the first two sweeps push; with direction=1 a sweep pulls exactly when the two before it
    # each diffused at least half of the out-links (dense sweeps, as on this R-MAT graph)
    nnz = len(ci)
    dense = [2 * t["edges"] >= nnz for t in tr]
    assert tr[0]["pull"] == 0 and tr[1]["pull"] == 0
    for k in range(2, len(tr)):
        assert tr[k]["pull"] == (1 if direction and dense[k - 1] and dense[k - 2] else 0)
    assert (sum(t["pull"] for t in tr) > 0) == bool(direction)
    assert sum(t["edges"] for t in tr) == st["edges_pushed"]
    assert all(tr[k + 1]["l1_F"] <= tr[k]["l1_F"] * (1 + 1e-12) for k in range(len(tr) - 1))
    assert tr[-1]["R"] <= 1e-10 * (1 - D)


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_profiled_solve_counts_pull_sweeps(di, direction):
    """profile=1 launches the sweep kernels from the host with events; it counts one sweep per
    loop sweep and, of those, the ones the trace records as pulls, and diffuses the same sets."""
    n, rp, ci = CASES["rmat_12"]
    with di.DiGraph(n, rp, ci, D) as g:
        H0, st0 = g.solve(1e-10, beta=BETA, direction=direction)
        H, st = g.solve(1e-10, beta=BETA, trace=1, profile=1, direction=direction)
        tr = g.trace()
        prof = g.profile()
    assert prof["sweeps"] == st["sweeps"] == st0["sweeps"] == len(tr)
    assert prof["pull_sweeps"] == sum(t["pull"] for t in tr)
    assert (prof["pull_sweeps"] > 0) == bool(direction)
    assert prof["scan_ms"] > 0 and prof["push_ms"] > 0 and prof["finalize_ms"] > 0
    assert st["edges_pushed"] == st0["edges_pushed"]
    assert np.abs(H - H0).sum() <= 1e-13


@pytest.mark.parametrize("direction", [0, 1])
def test_fp32_mixed_precision(di, direction):
    """FP32 fluid and pushes, FP64 H and residual: |H - H_oracle|_1 <= 2e-6."""
    for name in ["uniform_1e4", "zipf_2e14_hubs", "rmat_12"]:
        n, rp, ci = CASES[name]
        V = gg.uniform_v(n)
        H, F, st, _ = _solve(di, n, rp, ci, 1e-7, prec=di.DI_FP32_MIXED, direction=direction)
        r = oracle.diter(n, rp, ci, D, V, 1e-12, mode="sweep", beta=BETA)
        assert np.abs(H - r.H).sum() <= 2e-6, name
        assert st["bound"] <= 1e-7 * (1 + 1e-6)


def test_normalized_output(di):
    n, rp, ci = CASES["uniform_1e4"]
    with di.DiGraph(n, rp, ci, D) as g:
        H, st = g.solve(1e-10, normalize=1)
        Hr, _ = g.solve(1e-10)
    assert abs(H.sum() - 1.0) < 1e-13
    assert np.allclose(H, Hr / Hr.sum(), rtol=1e-14, atol=0)


def test_personalized_query(di):
    n, rp, ci = CASES["rmat_12"]
    seeds = gg.seed_set(n, 1, 32, seed=11, q=0)
    V = np.zeros(n)
    V[seeds] = 1.0 / len(seeds)
    with di.DiGraph(n, rp, ci, D) as g:
        H, st = g.query(seeds, 1e-12)
        w = np.arange(1, len(seeds) + 1, dtype=np.float64)
        Hw, stw = g.query(seeds, 1e-12, w=w)
    r = oracle.diter(n, rp, ci, D, V, 1e-12, mode="sweep", beta=BETA)
    assert np.abs(H - r.H).sum() <= max(st["bound"], r.l1F / (1 - D)) + 1e-12
    Vw = np.zeros(n)
    Vw[seeds] = w / w.sum()
    rw = oracle.diter(n, rp, ci, D, Vw, 1e-12, mode="sweep", beta=BETA)
    assert np.abs(Hw - rw.H).sum() <= max(stw["bound"], rw.l1F / (1 - D)) + 1e-12


def test_explicit_v(di):
    n, rp, ci = CASES["zipf_2e14_hubs"]
    rng = np.random.default_rng(3)
    V = graphs.random_v(n, rng)
    H, F, st, _ = _solve(di, n, rp, ci, 1e-13, V=V)
    r = oracle.diter(n, rp, ci, D, V, 1e-13, mode="sweep", beta=BETA)
    assert np.abs(H - r.H).sum() <= 1e-12


def test_device_buffers(di):
    n, rp, ci = CASES["rmat_12"]
    dev = torch.device("cuda")
    rp_t = torch.from_numpy(rp).to(dev)
    ci_t = torch.from_numpy(ci).to(dev)
    H_t = torch.empty(n, dtype=torch.float64, device=dev)
    with di.DiGraph(n, rp_t, ci_t, D) as g:
        g.solve(1e-12, H_out=H_t)
        torch.cuda.synchronize()
        H_host, _ = g.solve(1e-12)
    assert np.abs(H_t.cpu().numpy() - H_host).sum() <= 1e-13


def test_limits_report_not_converged(di):
    n, rp, ci = CASES["uniform_1e4"]
    with di.DiGraph(n, rp, ci, D) as g:
        H = np.empty(n)
        rc, st = di.di_solve_ex(g.handle, H, 1e-12, max_edge_pushes=50000, allow_unconverged=True)
        assert rc == di.DI_ENOTCONVERGED and not st["converged"]
        assert st["edges_pushed"] >= 50000 and st["bound"] > 1e-12
        rc, st2 = di.di_solve_ex(g.handle, H, 1e-12, max_sweeps=3, allow_unconverged=True)
        assert rc == di.DI_ENOTCONVERGED and st2["sweeps"] == 3
        with pytest.raises(di.DiError):
            g.solve(1e-12, max_sweeps=3)
        # a target met at the start needs no sweep (the while-test of ALGO-REF comes first)
        _, st3 = g.solve(1.0)
        assert st3["sweeps"] == 0 and st3["converged"]


def test_invalid_inputs(di):
    n, rp, ci = CASES["rmat_12"]
    bad = ci.copy()
    bad[5] = n
    with pytest.raises(di.DiError, match="col_idx"):
        di.DiGraph(n, rp, bad, D)
    # a host col_idx is copied and counted in pieces: an error in the last piece, and from
    # device memory (one piece)
    bad = ci.copy()
    bad[-1] = -1
    with pytest.raises(di.DiError, match="col_idx"):
        di.DiGraph(n, rp, bad, D)
    with pytest.raises(di.DiError, match="col_idx"):
        di.DiGraph(n, torch.from_numpy(rp).cuda(), torch.from_numpy(bad).cuda(), D)
    rp2 = rp.copy()
    rp2[10], rp2[11] = rp2[11], rp2[10] - 1
    with pytest.raises(di.DiError):
        di.DiGraph(n, rp2, ci, D)
    V = gg.uniform_v(n)
    V[0] = -V[0]
    with pytest.raises(di.DiError, match="negative"):
        di.DiGraph(n, rp, ci, D, V=V)
    V = gg.uniform_v(n) * 1.01
    with pytest.raises(di.DiError, match="normalized"):
        di.DiGraph(n, rp, ci, D, V=V)
    with pytest.raises(di.DiError):
        di.DiGraph(n, rp, ci, 1.0)
    with di.DiGraph(n, rp, ci, D) as g:
        with pytest.raises(di.DiError):
            g.solve(0.0)
        with pytest.raises(di.DiError, match="seed"):
            g.query([n + 3], 1e-6)


# --------------------------------------------------------- power iteration

@pytest.mark.parametrize("name", ["uniform_1e4", "zipf_2e14_hubs", "rmat_12", "in_hub_5000", "star_3000", "empty_7"])
def test_power_iteration_matches_oracle(di, name):
    n, rp, ci = CASES[name]
    V = gg.uniform_v(n)
    tol = 1e-12
    with di.DiGraph(n, rp, ci, D) as g:
        X, st = g.power(tol)
    Xo, it, delta, ok = oracle.power(n, rp, ci, D, V, tol)
    assert ok and st["converged"]
    if st["sweeps"] != it:
        # The stop rule compares |X_k - X_{k-1}|_1 with tol (1-d)/d, and at tol = 1e-12 that
        # difference is a sum of cancellations of entries near |X|_inf: a product's rounding
        # moves it by about sqrt(L) eps |X|_inf, and the two summation orders decide
        # differently only inside that band.  A stop one product apart is right only if the
        # oracle's difference at the earlier product lies within a few times that of the threshold.
        assert abs(st["sweeps"] - it) == 1
        _, k, dk, _ = oracle.power(n, rp, ci, D, V, tol, max_iter=min(st["sweeps"], it))
        thr = tol * (1 - D) / D
        noise = np.sqrt(len(ci)) * np.finfo(np.float64).eps * np.abs(Xo).max()
        assert abs(dk - thr) <= 4 * noise
    assert np.abs(X - Xo).sum() <= 1e-12
    assert st["edges_pushed"] == st["sweeps"] * len(ci)


def test_power_and_diter_agree(di):
    n, rp, ci = CASES["zipf_2e14_hubs"]
    with di.DiGraph(n, rp, ci, D) as g:
        X, stp = g.power(1e-11)
        H, std = g.solve(1e-11)
    assert np.abs(X - H).sum() <= 2e-11


def test_bounded_wait_gives_up(di):
    """The scan's bounded wait, on an mbarrier that nothing completes, gives up in every CTA
    and returns; the context stays usable."""
    assert di.di_selftest_wait(64, 8) == 8
    with pytest.raises(di.DiError):
        di.di_selftest_wait(0, 8)
    n, rp, ci = CASES["uniform_1e4"]
    H, F, st, _ = _solve(di, n, rp, ci, 1e-10)
    assert st["converged"] == 1


@pytest.mark.parametrize("family", ["uniform", "zipf_hubs"])
def test_scan_wait_watchdog_keeps_results_valid(di, family):
    """With one poll per bulk-copy wait (a watchdog far shorter than a DRAM load) every solve
    either converges to the oracle's answer or stops with DI_ETIMEOUT; a wait that ran out
    leaves the graph and the context usable.  The Zipf graph has rows above 1024 out-links,
    whose chunks the push stages with bulk copies behind the same bounded waits."""
    if family == "uniform":
        g = gg.uniform_graph(1 << 18, 20, seed=5)
    else:
        g = gg.zipf_graph(1 << 16, kmax=20000, seed=5)
        assert int(np.diff(g.row_ptr).max()) > 2 * 2048
    V = gg.uniform_v(g.n)
    r = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-10, mode="sweep", beta=BETA)
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as G:
        for _ in range(3):
            try:
                H, st = G.solve(1e-10, beta=BETA, scan_wait_polls=1)
                assert np.abs(H - r.H).sum() <= max(st["bound"], r.l1F / (1 - D)) + 1e-12
            except di.DiError as e:
                assert e.status == di.DI_ETIMEOUT
        with pytest.raises(di.DiError):
            G.solve(1e-8, beta=BETA, scan_wait_polls=-1)
        H, st = G.solve(1e-10, beta=BETA)
    assert st["converged"] == 1
    assert np.abs(H - r.H).sum() <= max(st["bound"], r.l1F / (1 - D)) + 1e-12


def test_many_hub_rows(di):
    """2500 nodes with 1100 out-links each (all above the 1024-link cutoff): every sweep cuts
    thousands of hub rows into chunks spread over the CTAs.  Same sweeps, elementary steps and
    H as the oracle."""
    rng = np.random.default_rng(12)
    n = 4000
    edges = [(i, int(j)) for i in range(2500) for j in rng.choice(n, 1100, replace=False)]
    rp, ci = graphs.csr(n, edges)
    V = gg.uniform_v(n)
    tol = 1e-10
    H, F, st, tr = _solve(di, n, rp, ci, tol, trace=1)
    r = oracle.diter(n, rp, ci, D, V, tol, mode="sweep", beta=BETA)
    assert st["converged"] == 1
    assert tr[0]["pushed"] == 2500
    assert st["sweeps"] == r.sweeps and st["edges_pushed"] == r.edges
    assert np.abs(H - r.H).sum() <= max(st["bound"], r.l1F / (1 - D)) + 1e-12


def test_giant_hub_row(di):
    """A row of 270,000 out-links: more than 253 chunks of 1024, so its chunks are longer than
    a staging buffer and the push reads them directly.  FP64 and FP32-mixed, both directions,
    and a batch of queries seeded on the hub, against the oracle."""
    rng = np.random.default_rng(21)
    n = 300000
    rp0, ci0 = graphs.random_graph(n, 0.2, 6, rng)
    hub = rng.choice(np.arange(1, n), 270000, replace=False).astype(np.int32)
    deg = np.diff(rp0)
    deg[0] = len(hub)
    rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    ci = np.concatenate([hub, ci0[rp0[1]:]]).astype(np.int32)
    V = gg.uniform_v(n)
    tol = 1e-11
    r = oracle.diter(n, rp, ci, D, V, tol, mode="sweep", beta=BETA)
    with di.DiGraph(n, rp, ci, D) as g:
        for prec, ptol, allow in ((di.DI_FP64, tol, 1e-12), (di.DI_FP32_MIXED, 1e-7, 2e-6)):
            for direction in (0, 1):
                H, st = g.solve(ptol, beta=BETA, prec=prec, direction=direction)
                assert st["converged"] == 1
                if prec == di.DI_FP64:
                    assert st["sweeps"] == r.sweeps and st["edges_pushed"] == r.edges
                assert np.abs(H - r.H).sum() <= max(st["bound"], r.l1F / (1 - D)) + allow
        seeds = [[0], [0, 5, 9], [17]]
        Hb, stq, sta = g.query_batch(seeds, 1e-8)
    assert sta["converged"] == 1
    for q, sd in enumerate(seeds):
        Vq = np.zeros(n)
        Vq[sd] = 1.0 / len(sd)
        rq = oracle.diter(n, rp, ci, D, Vq, 1e-12, mode="sweep", beta=BETA)
        assert np.abs(Hb[q] - rq.H).sum() <= stq[q]["bound"] + 2e-6
