"""The allocation-free power iteration, di_power_noalloc, against di_power.

di_power_noalloc exists for callers that cannot allocate device memory (services
with fixed memory pools, plug-ins in hosts that own the GPU allocator).  It keeps its work area in a static array inside
the library, so this file runs last: it must give di_power's answer whether it
runs alone in a fresh process or after every other test, and on two calls in a
row (the array keeps the previous call's contents).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 0.85
TOL = 1e-12


@pytest.fixture(scope="module")
def di():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_6158_gb300 as di
    di.load()
    return di


def in_links(n, rp, ci):
    """In-link CSR (sources ascending) with numpy."""
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    order = np.lexsort((src, ci))
    in_ptr = np.zeros(n + 1, np.int32)
    np.add.at(in_ptr, ci.astype(np.int64) + 1, 1)
    return np.cumsum(in_ptr).astype(np.int32), src[order].astype(np.int32)


@pytest.mark.parametrize("graph", ["uniform", "zipf"])
def test_noalloc_power_matches_di_power_twice(di, graph):
    if graph == "uniform":
        g = gg.uniform_graph(10000, 20, seed=1)
    else:
        g = gg.zipf_graph(50000, kmax=5000, seed=2)
    n, rp, ci = g.n, g.row_ptr, g.col_idx
    with di.DiGraph(n, rp, ci, D) as G:
        X_ref, st_ref = G.power(TOL)
    in_ptr, in_src = in_links(n, rp, ci)
    dev = torch.device("cuda")
    t_in_ptr = torch.from_numpy(in_ptr).to(dev)
    t_in_src = torch.from_numpy(in_src).to(dev)
    t_row_ptr = torch.from_numpy(rp).to(dev)
    X = torch.empty(n, dtype=torch.float64, device=dev)
    for call in range(2):
        X.fill_(-1.0)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _, st = di.di_power_noalloc(n, t_in_ptr, t_in_src, t_row_ptr, D, TOL, X)
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the module that holds the static array
            assert torch.cuda.mem_get_info()[0] == free0
        assert st["converged"] == 1
        if st["sweeps"] != st_ref["sweeps"]:
            # The two kernels sum |X_k - X_{k-1}|_1 in different orders, so a difference within
            # rounding of the stop threshold may stop one product apart; accept that only when
            # the oracle's difference at the earlier product lies in that band (about
            # sqrt(L) eps |X|_inf).
            assert abs(st["sweeps"] - st_ref["sweeps"]) == 1
            V = np.full(n, 1.0 / n)
            _, _k, dk, _ = oracle.power(n, rp, ci, D, V, TOL, max_iter=min(st["sweeps"], st_ref["sweeps"]))
            noise = np.sqrt(len(ci)) * np.finfo(np.float64).eps * np.abs(X_ref).max()
            assert abs(dk - TOL * (1 - D) / D) <= 4 * noise
        assert np.abs(X.cpu().numpy() - X_ref).sum() <= 1e-12


def test_noalloc_rejects_oversize_and_host_arrays(di):
    dev = torch.device("cuda")
    n = 65537
    in_ptr = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    X = torch.empty(n, dtype=torch.float64, device=dev)
    with pytest.raises(di.DiError, match="65536"):
        di.di_power_noalloc(n, in_ptr, torch.zeros(1, dtype=torch.int32, device=dev), in_ptr, D, TOL, X)
    host = np.zeros(11, np.int32)
    with pytest.raises(di.DiError, match="device memory"):
        di.di_power_noalloc(10, host, np.zeros(1, np.int32), host, D, TOL, np.zeros(10))
    pinned = torch.zeros(11, dtype=torch.int32).pin_memory()
    Xp = torch.zeros(10, dtype=torch.float64).pin_memory()
    with pytest.raises(di.DiError, match="device memory"):
        di.di_power_noalloc(10, pinned, torch.zeros(1, dtype=torch.int32, device=dev), pinned, D, TOL, Xp)
