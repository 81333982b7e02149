"""The seeded input generators: shapes, distributions, determinism (CPU only)."""
import numpy as np

import graphgen as gg


def _rows_ok(g, self_loops_allowed=False, dups_allowed=False):
    rp, ci = g.row_ptr, g.col_idx
    assert rp[0] == 0 and rp[-1] == len(ci) and np.all(np.diff(rp) >= 0)
    assert len(ci) == 0 or (ci.min() >= 0 and ci.max() < g.n)
    for i in range(g.n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) >= (0 if dups_allowed else 1)), i
        if not self_loops_allowed:
            assert not np.any(row == i)


def test_uniform_family():
    g = gg.uniform_graph(10000, 20, seed=1)
    _rows_ok(g)
    deg = g.outdeg()
    assert deg.min() == 0 and deg.max() == 20
    # U{0..20}: mean 10, P(0) = 1/21
    assert abs(deg.mean() - 10) < 0.2
    assert abs((deg == 0).mean() - 1 / 21) < 0.01
    g2 = gg.uniform_graph(10000, 20, seed=1)
    assert np.array_equal(g.row_ptr, g2.row_ptr) and np.array_equal(g.col_idx, g2.col_idx)
    g3 = gg.uniform_graph(10000, 20, seed=2)
    assert not np.array_equal(g.col_idx[:1000], g3.col_idx[:1000])


def test_zipf_family():
    n = 1 << 16
    g = gg.zipf_graph(n, alpha=2.1, kmax=5000, dangling_frac=0.12, target_exp=0.9, seed=3)
    _rows_ok(g)
    deg = g.outdeg()
    assert (deg == 0).sum() == int(0.12 * n)
    nz = deg[deg > 0]
    assert nz.min() == 1 and nz.max() <= 5000
    # Zipf(2.1): P(1) = 1/zeta(2.1) ~ 0.641, P(2) ~ 0.149
    assert abs((nz == 1).mean() - 0.641) < 0.01
    assert abs((nz == 2).mean() - 0.149) < 0.01
    # targets skewed: the most popular node receives far more than the mean in-degree
    indeg = np.bincount(g.col_idx, minlength=n)
    assert indeg.max() > 50 * indeg.mean()


def test_rmat_family():
    g = gg.rmat_graph(12, 16, seed=5)
    _rows_ok(g, self_loops_allowed=True)
    assert g.nnz <= 16 * 4096
    graw = gg.rmat_graph(12, 16, seed=5, dedup=False)
    assert graw.nnz == 16 * 4096
    _rows_ok(graw, self_loops_allowed=True, dups_allowed=True)
    # dedup keeps exactly the distinct (src, dst) pairs
    pairs = set()
    for i in range(graw.n):
        for j in graw.col_idx[graw.row_ptr[i]:graw.row_ptr[i + 1]]:
            pairs.add((i, int(j)))
    assert len(pairs) == g.nnz
    # quadrant a=0.57 dominates: node 0 has the largest out-degree
    assert g.outdeg().argmax() == 0


def test_seed_sets():
    sets = gg.seed_sets(1000, 50, 1, 32, seed=9)
    sizes = [len(s) for s in sets]
    assert min(sizes) >= 1 and max(sizes) <= 32
    for s in sets:
        assert len(set(s.tolist())) == len(s) and s.min() >= 0 and s.max() < 1000
    assert all(np.array_equal(a, b) for a, b in zip(sets, gg.seed_sets(1000, 50, 1, 32, seed=9)))


def test_unit_draws_uniform():
    u = np.array([gg.unit_draw(1, 7, k) for k in range(20000)])
    assert 0 <= u.min() and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.01


def test_modify_is_seeded_and_keeps_row_order():
    g = gg.rmat_graph(10, 8, seed=4)
    a = gg.modify(g, 0.1, 200, seed=9)
    b = gg.modify(g, 0.1, 200, seed=9)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    kept = 0
    for i in range(g.n):
        old = g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()
        new = a.col_idx[a.row_ptr[i]:a.row_ptr[i + 1]].tolist()
        # the kept edges are a subsequence of the old row, the rest are appended extras
        it = iter(old)
        k = 0
        while k < len(new) and any(x == new[k] for x in it):
            k += 1
        kept += k
        assert all(0 <= j < g.n for j in new)
    assert a.nnz - kept <= 200 + 0 and kept <= g.nnz
    assert abs((g.nnz - kept) / g.nnz - 0.1) < 0.03
    c = gg.modify(g, 0.0, 0, seed=1)
    assert np.array_equal(c.row_ptr, g.row_ptr) and np.array_equal(c.col_idx, g.col_idx)
