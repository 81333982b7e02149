"""Small hand-made graphs (CSR of out-links) used by the tests."""
import numpy as np


def csr(n, edges):
    """CSR from an edge list [(i, j), ...] in the given order (multi-edges kept)."""
    rows = [[] for _ in range(n)]
    for i, j in edges:
        rows[i].append(j)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for i in range(n):
        row_ptr[i + 1] = row_ptr[i] + len(rows[i])
    col_idx = np.array([j for r in rows for j in r], dtype=np.int32)
    return row_ptr, col_idx


def chain(n):
    return csr(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return csr(n, [(i, (i + 1) % n) for i in range(n)])


def star(m):
    """node 0 -> 1..m, leaves dangling"""
    return csr(m + 1, [(0, k) for k in range(1, m + 1)])


def complete(n):
    return csr(n, [(i, j) for i in range(n) for j in range(n) if i != j])


def random_graph(n, p_dangling, max_deg, rng, self_loops=True, multi=True):
    edges = []
    for i in range(n):
        if rng.random() < p_dangling:
            continue
        k = int(rng.integers(1, max_deg + 1))
        for _ in range(k):
            j = int(rng.integers(0, n))
            if not self_loops and j == i:
                continue
            edges.append((i, j))
    if not multi:
        edges = sorted(set(edges))
    return csr(n, edges)


def random_v(n, rng):
    v = rng.random(n) + 0.05
    return v / v.sum()


def modify(n, row_ptr, col_idx, rng, drop=0.1, add=0.1):
    """An updated graph: each edge dropped with probability `drop`, about add*L new
    random edges, one linked node made dangling and one dangling node given links."""
    edges = [(i, int(j)) for i in range(n) for j in col_idx[row_ptr[i]:row_ptr[i + 1]]]
    keep = [e for e in edges if rng.random() >= drop]
    for _ in range(max(1, int(add * len(edges)))):
        keep.append((int(rng.integers(0, n)), int(rng.integers(0, n))))
    outdeg = np.diff(np.asarray(row_ptr))
    linked = [i for i in range(n) if outdeg[i] > 0]
    dangling = [i for i in range(n) if outdeg[i] == 0]
    if linked:
        gone = linked[int(rng.integers(0, len(linked)))]
        keep = [e for e in keep if e[0] != gone]
    if dangling:
        new = dangling[int(rng.integers(0, len(dangling)))]
        keep += [(new, int(rng.integers(0, n))) for _ in range(3)]
    return csr(n, keep)


def hub_graph(n, hubs, rng, max_deg=4):
    """A random graph plus `hubs` nodes that link to and from every other node: the ALGO-OP
    weights 1/((#in+1)(#out+1)) then span several orders of magnitude."""
    edges = []
    for h in range(hubs):
        for j in range(n):
            if j != h:
                edges.append((h, j))
                edges.append((j, h))
    rp0, ci0 = random_graph(n, 0.1, max_deg, rng)
    for i in range(n):
        for j in ci0[rp0[i]:rp0[i + 1]]:
            edges.append((i, int(j)))
    return csr(n, edges)
