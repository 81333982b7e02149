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
