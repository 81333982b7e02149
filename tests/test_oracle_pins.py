"""Pins of the oracle to the paper and to mathematics (CPU only).

Each test ties an oracle function to something other than itself: a closed
form, exact rational elimination, a library solver, Theorems 1 and 2, the
Lemma of Section 3.1, monotonicity, order independence or brute force.
test_mutants.py checks that plausible mistakes planted in copies of the oracle
fail these pins.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import ge
from tests import graphs

D = 0.85
ALL_MODES = ["per", "rand", "max", "thresh", "sweep"]


def _rand_case(seed, n=40, p_dang=0.2, max_deg=6):
    rng = np.random.default_rng(seed)
    rp, ci = graphs.random_graph(n, p_dang, max_deg, rng)
    V = graphs.random_v(n, rng)
    return n, rp, ci, V


# --------------------------------------------------------------- elimination

@pytest.mark.parametrize("seed", range(6))
def test_ge_matches_exact_rational(seed):
    """FP64 elimination == exact rational elimination (Section 2.1 fixed point) to rounding."""
    rng = np.random.default_rng(100 + seed)
    n = 9
    rp, ci = graphs.random_graph(n, 0.25, 4, rng)
    Vq = [Fraction(int(x), 1) for x in rng.integers(1, 9, n)]
    s = sum(Vq)
    Vq = [v / s for v in Vq]
    d = Fraction(17, 20)
    exact = ge.solve_exact(n, rp, ci, d, Vq)
    approx = ge.pagerank_dense(n, rp, ci, float(d), np.array([float(v) for v in Vq]))
    # the exact solution satisfies X = dPX + (1-d)V exactly, edge by edge
    for r in range(n):
        inflow = sum(exact[i] * Fraction(1, int(rp[i + 1] - rp[i]))
                     for i in range(n) for e in range(rp[i], rp[i + 1]) if ci[e] == r)
        assert exact[r] == d * inflow + (1 - d) * Vq[r]
    assert np.max(np.abs(approx - np.array([float(x) for x in exact]))) < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_ge_matches_library_solver(seed):
    n, rp, ci, V = _rand_case(seed, n=150)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    P = ge.transition_matrix(n, rp, ci)
    Xlib = np.linalg.solve(np.eye(n) - D * P, (1 - D) * V)
    assert np.abs(X - Xlib).sum() < 1e-13


def test_closed_forms():
    n = 12
    rng = np.random.default_rng(5)
    V = graphs.random_v(n, rng)
    # chain 0->1->...->n-1: X_k = (1-d) sum_{m<=k} d^{k-m} V_m
    rp, ci = graphs.chain(n)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    want = np.array([(1 - D) * sum(D ** (k - m) * V[m] for m in range(k + 1)) for k in range(n)])
    assert np.allclose(X, want, rtol=0, atol=1e-15)
    # cycle: X_k = (1-d)/(1-d^n) sum_{m<n} d^m V_{k-m mod n}
    rp, ci = graphs.cycle(n)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    want = np.array([(1 - D) / (1 - D ** n) * sum(D ** m * V[(k - m) % n] for m in range(n)) for k in range(n)])
    assert np.allclose(X, want, rtol=0, atol=1e-15)
    # star 0 -> 1..m: X_0 = (1-d)V_0, X_leaf = (1-d)V_leaf + d X_0/m
    m = n - 1
    rp, ci = graphs.star(m)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    assert abs(X[0] - (1 - D) * V[0]) < 1e-16
    assert np.allclose(X[1:], (1 - D) * V[1:] + D * X[0] / m, rtol=0, atol=1e-16)
    # complete graph with V uniform: X = 1/n
    rp, ci = graphs.complete(n)
    X = ge.pagerank_dense(n, rp, ci, D, np.full(n, 1.0 / n))
    assert np.allclose(X, 1.0 / n, rtol=0, atol=1e-15)
    # isolated (all dangling): X = (1-d)V
    rp = np.zeros(n + 1, np.int32)
    X = ge.pagerank_dense(n, rp, np.zeros(0, np.int32), D, V)
    assert np.allclose(X, (1 - D) * V, rtol=0, atol=0)


# ----------------------------------------------------------- D-iteration

@pytest.mark.parametrize("mode", ALL_MODES)
@pytest.mark.parametrize("seed", range(3))
def test_diter_reaches_fixed_point_within_bound(mode, seed):
    """0 <= H <= X and |X - H|_1 <= |F|_1/(1-d) (Theorem 2 with dangling nodes, Section 3.3)."""
    n, rp, ci, V = _rand_case(seed)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    tol = 1e-11
    r = oracle.diter(n, rp, ci, D, V, tol, mode=mode, seed=seed)
    assert r.converged and r.R / (1 - D) <= tol
    bound = r.l1F / (1 - D)
    assert bound <= tol * (1 + 1e-9) + 1e-15
    err = np.abs(X - r.H).sum()
    assert err <= bound + 1e-14
    assert np.all(r.H >= 0) and np.all(r.H <= X + 1e-15)
    assert np.all(r.F >= 0)


def test_error_identity_is_equality_without_dangling():
    """Eq. (SL): |S_inf - H_n|_1 = |F_n|_1/(1-d) when every column of P sums to one."""
    rng = np.random.default_rng(9)
    n = 30
    rp, ci = graphs.random_graph(n, 0.0, 5, rng)
    V = graphs.random_v(n, rng)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    for mode in ALL_MODES:
        r = oracle.diter(n, rp, ci, D, V, 1e-3, mode=mode, seed=3)
        lhs = np.abs(X - r.H).sum()
        assert abs(lhs - r.l1F / (1 - D)) < 1e-13


@pytest.mark.parametrize("mode", ALL_MODES)
def test_theorem1_invariant_along_the_run(mode):
    """H_n + F_n = F_0 + dPH_n after every prefix of the run (Theorem 1)."""
    n, rp, ci, V = _rand_case(11, n=25)
    P = ge.transition_matrix(n, rp, ci)
    F0 = (1 - D) * V
    for k in [0, 1, 2, 3, 5, 8, 13, 40, 100, 400]:
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode=mode, seed=4, max_pushes=k)
        resid = r.H + r.F - F0 - D * P @ r.H
        assert np.max(np.abs(resid)) < 1e-15, (mode, k)


@pytest.mark.parametrize("mode", ALL_MODES)
def test_theorem2_identity(mode):
    """S_inf - H_n = (I - dP)^{-1} F_n (Theorem 2), with the inverse applied by elimination."""
    n, rp, ci, V = _rand_case(12, n=30)
    P = ge.transition_matrix(n, rp, ci)
    M = np.eye(n) - D * P
    X = ge.solve_no_pivot(M, (1 - D) * V)
    for k in [1, 7, 50]:
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode=mode, seed=2, max_pushes=k)
        assert np.abs((X - r.H) - ge.solve_no_pivot(M, r.F)).max() < 1e-15


def test_lemma_argmax_contraction():
    """ALGO-MAX: |F_n| <= |F_{n-1}| (1 - (1-d)/N) at every step (Lemma, Section 3.1)."""
    n, rp, ci, V = _rand_case(13, n=20)
    prev = None
    for k in range(0, 120):
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode="max", max_pushes=k)
        if prev is not None:
            assert r.l1F <= prev * (1 - (1 - D) / n) + 1e-16
        prev = r.l1F


@pytest.mark.parametrize("mode", ALL_MODES)
def test_monotone_fluid_and_history(mode):
    """F >= 0, |F|_1 non-increasing and H non-decreasing (Section 2.2), R == recomputed |F|_1."""
    n, rp, ci, V = _rand_case(14, n=30)
    prevF, prevH = None, None
    for k in range(0, 200, 7):
        r = oracle.diter(n, rp, ci, D, V, 0.0, mode=mode, seed=1, max_pushes=k)
        assert np.all(r.F >= 0)
        assert abs(r.R - r.l1F) < 1e-15
        if prevF is not None:
            assert r.l1F <= prevF + 1e-17
            assert np.all(r.H >= prevH)
        prevF, prevH = r.l1F, r.H.copy()


def test_order_independence():
    """Every order reaches the same X (Section 1, Section 2.2): pairwise within the bounds."""
    n, rp, ci, V = _rand_case(15, n=60)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    res = [oracle.diter(n, rp, ci, D, V, 1e-6, mode=m, seed=s) for m in ALL_MODES for s in (1, 2)]
    for a in res:
        assert np.abs(X - a.H).sum() <= a.l1F / (1 - D) + 1e-14
        for b in res:
            assert np.abs(a.H - b.H).sum() <= max(a.l1F, b.l1F) / (1 - D) + 1e-14


def test_dangling_only_graph_single_sweep():
    """With no links every diffusion just drains fluid: H = (1-d)V = X after one sweep."""
    n = 16
    V = graphs.random_v(n, np.random.default_rng(1))
    r = oracle.diter(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), D, V, 1e-14, mode="sweep", beta=0.0)
    assert r.sweeps == 1 and r.edges == 0 and r.pushes == n
    assert np.array_equal(r.H, (1 - D) * V)


def test_counting_rules():
    """Elementary steps = out-links used; zero-fluid PER picks are skipped uncounted (Section 4.2)."""
    rp, ci = graphs.star(5)
    n = 6
    V = np.zeros(n)
    V[0] = 1.0
    r = oracle.diter(n, rp, ci, D, V, 0.0, mode="per", max_pushes=1)
    assert r.pushes == 1 and r.edges == 5 and r.picks == 1
    r = oracle.diter(n, rp, ci, D, V, 0.0, mode="per", max_pushes=3)
    assert r.pushes == 3 and r.edges == 5 and r.picks == 3
    # the chain's fluid sits only at the head: PER skips the empty nodes uncounted
    rp, ci = graphs.chain(6)
    r = oracle.diter(6, rp, ci, D, V, 0.0, mode="per", max_pushes=2)
    assert r.pushes == 2 and r.picks == 2
    V2 = np.zeros(6)
    V2[5] = 1.0
    r = oracle.diter(6, rp, ci, D, V2, 0.0, mode="per", max_pushes=1)
    assert r.picks == 6 and r.pushes == 1 and r.edges == 0


def test_sweep_resume_is_bitwise_continuation():
    """Checkpoint/resume: the state (F, H, R) is complete (Theorem 1), so two calls == one."""
    n, rp, ci, V = _rand_case(16, n=80)
    whole = oracle.diter(n, rp, ci, D, V, 1e-12, mode="sweep")
    F, H, R = oracle.init(n, D, V)
    first = oracle.run(n, rp, ci, D, F, H, R, 1e-12, mode="sweep", max_pushes=50)
    assert not first.converged
    second = oracle.run(n, rp, ci, D, F, H, first.R, 1e-12, mode="sweep")
    assert np.array_equal(second.H, whole.H) and np.array_equal(second.F, whole.F)
    assert first.edges + second.edges == whole.edges


def test_max_push_cap_reports_not_converged():
    n, rp, ci, V = _rand_case(17)
    r = oracle.diter(n, rp, ci, D, V, 1e-12, mode="sweep", max_pushes=5)
    assert not r.converged and r.R / (1 - D) > 1e-12


# ------------------------------------------------------------ power iteration

def test_power_partial_sums():
    """From X_0 = 0, n products give S_{n-1} = sum_{k<n} (dP)^k (1-d)V (Section 2.2)."""
    n, rp, ci, V = _rand_case(18, n=30)
    P = ge.transition_matrix(n, rp, ci)
    for iters in [1, 2, 5, 17]:
        X, it, delta, ok = oracle.power(n, rp, ci, D, V, 0.0, max_iter=iters)
        assert it == iters and not ok
        S = np.zeros(n)
        term = (1 - D) * V
        for _ in range(iters):
            S += term
            term = D * P @ term
        assert np.abs(X - S).max() < 1e-16


def test_power_converges_to_fixed_point():
    """MAT-ITER stop rule |X_n - X_{n-1}| d/(1-d) < tol bounds |X - X_n|_1 (contraction by d)."""
    n, rp, ci, V = _rand_case(19, n=100)
    X = ge.pagerank_dense(n, rp, ci, D, V)
    tol = 1e-10
    Xp, it, delta, ok = oracle.power(n, rp, ci, D, V, tol)
    assert ok and delta * D / (1 - D) < tol
    assert np.abs(X - Xp).sum() <= tol + 1e-15


# ------------------------------------------------------ transpose and bins

def outdeg_case(seed):
    """A multigraph given as an edge list (self-loops and repeated links kept, some rows empty,
    the last row non-empty) and its CSR; the out-degrees are counted from the list itself."""
    rng = np.random.default_rng(seed)
    n = 60
    edges = [(int(rng.integers(0, n - 10)), int(rng.integers(0, n))) for _ in range(250)]  # rows 50..58 empty
    edges += [(n - 1, 0), (n - 1, n - 1), (n - 1, n - 1), (3, 3)]
    rp, ci = graphs.csr(n, edges)
    return n, rp, edges


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_outdeg_brute_force(seed):
    """#out_i (Section 2.1: column i of P holds 1/#out_i on each listed link) is the number of
    times i appears as a source in the edge list, multi-edges and self-loops included."""
    n, rp, edges = outdeg_case(seed)
    want = [sum(1 for i, _j in edges if i == k) for k in range(n)]
    got = oracle.outdeg(n, rp)
    assert got.tolist() == want
    assert 0 in want and int(got.sum()) == len(edges)


def test_outdeg_edge_cases():
    assert oracle.outdeg(1, np.array([0, 0], np.int32)).tolist() == [0]
    assert oracle.outdeg(3, np.array([0, 2, 2, 5], np.int32)).tolist() == [2, 0, 3]


def test_transpose_brute_force():
    n, rp, ci, _ = _rand_case(20, n=70)
    in_ptr, in_src = oracle.transpose(n, rp, ci)
    edges = sorted((int(j), i) for i in range(n) for j in ci[rp[i]:rp[i + 1]])
    want_ptr = np.zeros(n + 1, np.int64)
    for j, _i in edges:
        want_ptr[j + 1] += 1
    assert np.array_equal(in_ptr, np.cumsum(want_ptr))
    assert in_src.tolist() == [i for _j, i in edges]


def test_bins_brute_force():
    n, rp, ci, _ = _rand_case(21, n=200, max_deg=40)
    cuts = [0, 3, 17]
    bin_of, bin_ptr, bin_ids = oracle.bins(n, rp, cuts)
    deg = np.diff(rp)
    want = [sum(int(dg > c) for c in cuts) for dg in deg]
    assert bin_of.tolist() == want
    for b in range(len(cuts) + 1):
        ids = bin_ids[bin_ptr[b]:bin_ptr[b + 1]].tolist()
        assert ids == [i for i in range(n) if want[i] == b]


# ------------------------------------------------- graph update (Section 3.2)

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("tol0", [1e-1, 1e-3, 1e-6])
def test_update_reaches_the_updated_fixed_point(seed, tol0):
    """A run on P stopped at bound tol0, continued on P' from F_0' = F + d(P'-P)H, ends
    within its bound of the solution of X = dP'X + (1-d)V (the theorem after Theorem 3)."""
    rng = np.random.default_rng(seed)
    n = 60
    rp, ci = graphs.random_graph(n, 0.15, 6, rng)
    rp2, ci2 = graphs.modify(n, rp, ci, rng)
    V = graphs.random_v(n, rng)
    X2 = ge.pagerank_dense(n, rp2, ci2, D, V)
    r0 = oracle.diter(n, rp, ci, D, V, tol0, mode="sweep")
    for mode in ("sweep", "max", "per"):
        r1 = oracle.solve_update(n, rp, ci, rp2, ci2, D, r0.F, r0.H, 1e-12, mode=mode, max_pushes=10 ** 7)
        assert r1.converged
        assert np.abs(X2 - r1.H).sum() <= r1.l1F / (1 - D) + 1e-13


def test_update_injection_keeps_theorem1_for_the_new_graph():
    """After the injection, H + F' = F_0 + dP'H: the state is a D-iteration state of P'."""
    rng = np.random.default_rng(9)
    n = 50
    rp, ci = graphs.random_graph(n, 0.2, 5, rng)
    rp2, ci2 = graphs.modify(n, rp, ci, rng)
    V = graphs.random_v(n, rng)
    r0 = oracle.diter(n, rp, ci, D, V, 1e-4, mode="sweep")
    F2 = oracle.update(n, rp, ci, rp2, ci2, D, r0.F, r0.H)
    P2 = ge.transition_matrix(n, rp2, ci2)
    assert (F2 < 0).any(), "the update should inject negative fluid somewhere"
    assert np.abs(r0.H + F2 - (1 - D) * V - D * P2 @ r0.H).max() < 1e-15
    # the signed fluid keeps moving: |F|_1 never grows along the continued run
    prev = np.abs(F2).sum()
    F, H = F2.copy(), r0.H.copy()
    for _ in range(20):
        r = oracle.run(n, rp2, ci2, D, F, H, float(np.abs(F).sum()), 0.0, mode="max", max_pushes=3)
        cur = np.abs(r.F).sum()
        assert cur <= prev * (1 + 1e-15)
        assert r.R >= cur - 1e-15        # R stays an upper bound on |F|_1
        prev = cur


def test_theorem3_update_identity():
    """Theorem 3: X' - X = (I - dP')^-1 d(P' - P) X, checked with exact rational elimination."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(4)
    n = 7
    rp, ci = graphs.random_graph(n, 0.2, 3, rng)
    rp2, ci2 = graphs.modify(n, rp, ci, rng)
    d = Fr(17, 20)
    V = [Fr(1, n)] * n
    X = ge.solve_exact(n, rp, ci, d, V)
    X2 = ge.solve_exact(n, rp2, ci2, d, V)

    def P(rp_, ci_, x):
        y = [Fr(0)] * n
        for i in range(n):
            deg = rp_[i + 1] - rp_[i]
            for e in range(rp_[i], rp_[i + 1]):
                y[ci_[e]] += x[i] / deg
        return y
    rhs = [d * (a - b) for a, b in zip(P(rp2, ci2, X), P(rp, ci, X))]
    # (I - dP') (X' - X) = d(P' - P) X
    diff = [a - b for a, b in zip(X2, X)]
    lhs = [a - d * b for a, b in zip(diff, P(rp2, ci2, diff))]
    assert lhs == rhs


def test_update_with_the_same_graph_injects_nothing():
    rng = np.random.default_rng(12)
    n = 30
    rp, ci = graphs.random_graph(n, 0.2, 4, rng)
    V = graphs.random_v(n, rng)
    r0 = oracle.diter(n, rp, ci, D, V, 1e-3, mode="sweep")
    F2 = oracle.update(n, rp, ci, rp, ci, D, r0.F, r0.H)
    assert np.abs(F2 - r0.F).max() < 1e-17


# ---------------------------------------------- ALGO-OP / ALGO-OP2 (Section 4.3)

def test_selection_weights_by_hand():
    rp, ci = graphs.star(4)               # 0 -> 1..4; leaves dangling
    w, wscale = oracle.selection_weights(5, rp, ci, "op")
    # centre: #in 0, #out 4 -> 1/5; leaves: #in 1, #out 0 -> 1/2
    assert w.tolist() == [np.float32(1 / 5), np.float32(0.5), np.float32(0.5), np.float32(0.5), np.float32(0.5)]
    assert wscale == 0.25                 # mean 0.44 -> 2^-2
    w2, wscale2 = oracle.selection_weights(5, rp, ci, "op2")
    assert w2.tolist() == [np.float32(0.2), 1.0, 1.0, 1.0, 1.0]
    assert wscale2 == 0.5                 # mean 0.84 -> 2^-1


@pytest.mark.parametrize("sel", ["op", "op2"])
def test_op_argmax_and_first_sweep(sel):
    rng = np.random.default_rng(21)
    n = 40
    rp, ci = graphs.random_graph(n, 0.2, 8, rng)
    V = graphs.random_v(n, rng)
    F0 = (1 - D) * V
    w, wscale = oracle.selection_weights(n, rp, ci, sel)
    i_star = int(np.argmax(F0 * w.astype(np.float64)))
    assert i_star != int(np.argmax(F0)), "the weights should change the first choice on this graph"
    r = oracle.diter(n, rp, ci, D, V, 0.0, mode="max", max_pushes=1, select=sel)
    assert np.flatnonzero(r.H).tolist() == [i_star]
    S1 = np.flatnonzero(np.float32(F0) * w > np.float32(0.5 * (1 - D) / n * wscale))
    r = oracle.diter(n, rp, ci, D, V, 0.0, mode="sweep", max_pushes=1, select=sel)
    assert np.flatnonzero(r.H).tolist() == S1.tolist()


@pytest.mark.parametrize("sel", ["op", "op2"])
@pytest.mark.parametrize("mode", ["max", "sweep", "thresh"])
def test_op_orders_reach_the_fixed_point(sel, mode):
    """Any choice of the sequence converges to X (Section 2.2); ALGO-OP is one such choice."""
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        n = 50
        rp, ci = graphs.random_graph(n, 0.15, 6, rng)
        V = graphs.random_v(n, rng)
        X = ge.pagerank_dense(n, rp, ci, D, V)
        r = oracle.diter(n, rp, ci, D, V, 1e-12, mode=mode, select=sel, max_pushes=10 ** 7)
        assert r.converged
        assert np.abs(X - r.H).sum() <= r.l1F / (1 - D) + 1e-13
        assert np.all(r.H <= X + 1e-15)


@pytest.mark.parametrize("sel", [None, "op", "op2"])
def test_threshold_schedule(sel):
    """T_0 = beta R_0/N; after an empty sweep T/2; after a non-empty one beta R/N, or with weights
    min(T, beta R/N) (never raised).  The sweep's set is {i : |F_i| > T} or, weighted,
    {i : (float)|F_i| w_i > (float)(T wscale)}; checked on the recorded (T, R, count) of every sweep."""
    rng = np.random.default_rng(0)
    n = 80
    rp, ci = graphs.hub_graph(n, 3, rng)
    V = graphs.random_v(n, rng)
    tr = np.zeros((100000, 3))
    r = oracle.diter(n, rp, ci, D, V, 1e-11, mode="sweep", select=sel, trace=tr)
    assert r.converged
    T, R, cnt = tr[:r.sweeps, 0], tr[:r.sweeps, 1], tr[:r.sweeps, 2]
    assert T[0] == 0.5 * (1 - D) / n
    for k in range(r.sweeps - 1):
        if cnt[k] == 0:
            assert T[k + 1] == T[k] / 2
        elif sel is None:
            assert T[k + 1] == 0.5 * R[k + 1] / n
        else:
            assert T[k + 1] == min(T[k], 0.5 * R[k + 1] / n)
    if sel is not None:
        assert np.all(np.diff(T) <= 0)
    if sel == "op":
        assert (cnt == 0).any(), "the ALGO-OP run should meet empty sweeps on this graph"
    # the first sweep's set, replayed from F_0
    F0 = (1 - D) * V
    if sel is None:
        S1 = np.flatnonzero(np.abs(F0) > T[0])
    else:
        w, wscale = oracle.selection_weights(n, rp, ci, sel)
        S1 = np.flatnonzero(np.float32(np.abs(F0)) * w > np.float32(T[0] * wscale))
    assert cnt[0] == len(S1)


# ------------------------------------------------ timed multi-core CPU baseline

@pytest.mark.parametrize("threads", [1, 3])
def test_power_omp_matches_power(threads):
    """The OpenMP MAT-ITER (a pull over in-links) against orc_power (a push over out-links):
    the same number of products and the same iterate to rounding, on a graph with dangling
    nodes, multi-edges and self-loops; and both against elimination."""
    n, rp, ci, V = _rand_case(31, n=300, p_dang=0.15, max_deg=9)
    in_ptr, in_src = oracle.transpose(n, rp, ci)
    deg = oracle.outdeg(n, rp)
    X, it, delta, ok = oracle.power(n, rp, ci, D, V, 1e-13)
    Xo, ito, deltao, oko, used = oracle.power_omp(n, in_ptr, in_src, deg, D, V, 1e-13, threads=threads)
    assert ok and oko and used >= 1
    assert abs(it - ito) <= 1
    assert np.abs(X - Xo).sum() <= 1e-13
    assert np.abs(ge.pagerank_dense(n, rp, ci, D, V) - Xo).sum() <= 1e-12
    # a cut at k products gives the partial series, like orc_power
    X3, _, _, _ = oracle.power(n, rp, ci, D, V, 1e-13, max_iter=3)
    Xo3, it3, _, ok3, _ = oracle.power_omp(n, in_ptr, in_src, deg, D, V, 1e-13, max_iter=3, threads=threads)
    assert it3 == 3 and not ok3 and np.abs(X3 - Xo3).max() <= 1e-15
