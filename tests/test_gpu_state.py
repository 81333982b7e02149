"""Checkpoint and resume of a D-iteration state on the GPU (Theorem 1).

A state (F, H) saved with di_get_state after a solve stopped early is complete:
H + F = F_0 + dPH holds for it, so it can be written to disk, loaded into a new
graph handle with di_set_state and continued with di_solve_update(g, g).  The
tests check that
  * a state the oracle computed (no CUDA involved) is accepted with a deviation
    at rounding level, and continuing it reaches the oracle's full solve within
    the bound the device reports;
  * the device's own partial state, saved to a file and loaded into a second
    handle, continues to the same result as the first handle continuing itself;
  * a state that breaks Theorem 1 (one H entry moved, or a NaN), or one saved
    from a query (its F_0 is the query's), is rejected and the graph's state is
    left as it was.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

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


def cases():
    return {
        "uniform_20000": gg.uniform_graph(20000, 12, seed=5),
        "zipf_2e15": gg.zipf_graph(1 << 15, kmax=3000, seed=4),
        "rmat_14": gg.rmat_graph(14, 16, seed=6),
    }


CASES = cases()


@pytest.mark.parametrize("name", list(CASES))
def test_oracle_state_resumes_to_the_full_solve(di, name):
    g = CASES[name]
    V = gg.uniform_v(g.n)
    part = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-13, max_pushes=g.n // 2)
    assert not part.converged
    full = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-13)
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as dg:
        dev = dg.set_state(part.F, part.H, rtol=1e-9)
        assert dev <= 1e-13, dev
        F, H = dg.state()
        assert np.array_equal(F, part.F) and np.array_equal(H, part.H)
        Hd, st = dg.update_from(dg, 1e-12)
    assert st["converged"] and st["bound"] <= 1e-12
    err = float(np.abs(Hd - full.H).sum())
    assert err <= st["bound"] + full.l1F / (1 - D) + 1e-13, (err, st["bound"])


@pytest.mark.parametrize("name", list(CASES))
def test_saved_device_state_resumes_in_a_new_handle(di, name, tmp_path):
    g = CASES[name]
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as a:
        _, st0 = a.solve(1e-13, max_sweeps=4, allow_unconverged=True)
        assert not st0["converged"]
        F, H = a.state()
        np.savez(tmp_path / "state.npz", F=F, H=H)
        Ha, sta = a.update_from(a, 1e-12)
    saved = np.load(tmp_path / "state.npz")
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as b:
        dev = b.set_state(saved["F"], saved["H"], rtol=1e-9)
        assert dev <= 1e-12, dev
        Hb, stb = b.update_from(b, 1e-12)
    assert sta["converged"] and stb["converged"]
    # same state, same graph: the two runs differ only by the order of atomic additions
    assert float(np.abs(Ha - Hb).sum()) <= 1e-12
    full = oracle.diter(g.n, g.row_ptr, g.col_idx, D, gg.uniform_v(g.n), 1e-13)
    assert float(np.abs(Hb - full.H).sum()) <= stb["bound"] + full.l1F / (1 - D) + 1e-13


def test_device_inputs_are_accepted(di):
    g = CASES["uniform_20000"]
    V = gg.uniform_v(g.n)
    part = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-13, max_pushes=g.n)
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as dg:
        Fd = torch.from_numpy(part.F).cuda()
        Hd = torch.from_numpy(part.H).cuda()
        dev = dg.set_state(Fd, Hd, rtol=1e-9)
        assert dev <= 1e-13
        F, H = dg.state()
    assert np.array_equal(F, part.F) and np.array_equal(H, part.H)


def test_states_that_break_theorem_1_are_rejected(di):
    g = CASES["zipf_2e15"]
    V = gg.uniform_v(g.n)
    part = oracle.diter(g.n, g.row_ptr, g.col_idx, D, V, 1e-13, max_pushes=g.n)
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as dg:
        dg.set_state(part.F, part.H)
        keep_F, keep_H = dg.state()
        # move one history entry by 1e-6 of the state's scale (F dominates it on this graph)
        scale = float(np.max(np.abs(part.H) + np.abs(part.F) + (1 - D) * V))
        bad_H = part.H.copy()
        bad_H[int(np.argmax(part.H))] += 1e-6 * scale
        with pytest.raises(di.DiError) as e:
            dg.set_state(part.F, bad_H, rtol=1e-9)
        assert e.value.status == di.DI_EINVAL and "Theorem 1" in str(e.value)
        # a deviation is reported also for a rejected state, and a looser rtol accepts it
        dev = dg.set_state(part.F, bad_H, rtol=1.0)
        assert 1e-9 < dev < 1e-5
        dg.set_state(keep_F, keep_H)
        nan_F = part.F.copy()
        nan_F[7] = np.nan
        with pytest.raises(di.DiError) as e:
            dg.set_state(nan_F, part.H)
        assert e.value.status == di.DI_EINVAL
        F, H = dg.state()
        assert np.array_equal(F, keep_F) and np.array_equal(H, keep_H)
        # a query's state diffuses another F_0, so it does not satisfy Theorem 1 for (1-d)V
        dg.query(np.array([3, 11], np.int32), 1e-6)
        qF, qH = dg.state()
        with pytest.raises(di.DiError):
            dg.set_state(qF, qH, rtol=1e-6)


def test_argument_errors(di):
    g = CASES["uniform_20000"]
    with di.DiGraph(g.n, g.row_ptr, g.col_idx, D) as dg:
        x = np.zeros(g.n)
        for args in ((None, x, 1e-9), (x, None, 1e-9), (x, x, -1.0), (x, x, float("nan"))):
            with pytest.raises(di.DiError) as e:
                di.di_set_state(dg.handle, *args)
            assert e.value.status == di.DI_EINVAL
