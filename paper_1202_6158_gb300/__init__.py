"""D-iteration (fluid diffusion) PageRank on one GB300 GPU.

Python front end of libditer (include/diter.h).  The names follow the C ABI:
``di_graph_create``, ``di_solve``, ``di_solve_ex``, ``di_query``, ``di_power``,
``di_graph_export``, ``di_get_trace``, ``di_get_state``, ``di_set_state``, ``di_free``; the
:class:`DiGraph` class wraps a graph handle with the same calls as methods.
Arrays are numpy arrays or torch tensors, on the host or on the device.

The method is D. Hong, "Optimized on-line computation of PageRank algorithm":
fluid F_0 = (1-d)V is diffused along out-links (ALGO-REF, Section 2.2, with the
dangling-node rule of Section 3.3) in threshold sweeps (Section 4.2) until
|F|_1/(1-d), the Theorem 2 bound on |X - H|_1, meets the target.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (DI_EINVAL, DI_ENOMEM, DI_ENOTCONVERGED, DI_ETIMEOUT, DI_FP32_MIXED, DI_FP64, DI_OK, DiError, check,
                   di_batch_tune_result, di_completion, di_profile, di_server_graph_stats, di_tune_result, di_solve_opts,
                   di_stats, di_sweep_record, ptr)

__all__ = ["DiGraph", "DiError", "DI_FP64", "DI_FP32_MIXED", "DI_OK", "DI_EINVAL", "DI_ENOTCONVERGED", "DI_ETIMEOUT",
           "di_graph_create", "di_free", "di_solve", "di_solve_ex", "di_solve_update", "di_autotune", "di_autotune_batch", "di_query", "di_query_batch", "di_query_batch_ex", "di_power", "di_power_ex", "di_graph_export",
           "di_get_trace", "di_get_state", "di_set_state", "di_get_profile", "di_power_noalloc", "di_version", "di_selftest_wait", "di_debug_build", "di_debug_selftest", "load",
           "di_plan_lanes", "di_server_create", "di_server_lanes", "di_server_submit", "di_server_poll",
           "di_server_pending", "di_server_stats", "di_server_cancel", "di_server_free", "di_clock", "DiServer"]


def load():
    return _lib.load()


def di_version() -> str:
    return load().di_version().decode()


def di_debug_build() -> bool:
    """True when the loaded library is the DI_DEBUG build (device-side index checks)."""
    return bool(load().di_debug_build())


def di_debug_selftest() -> tuple:
    """Debug build: records one failed check from a kernel and reports it; returns (status, word)."""
    w = ctypes.c_uint64(0)
    rc = load().di_debug_selftest(ctypes.byref(w))
    return rc, w.value


def di_selftest_wait(polls=64, ctas=8) -> int:
    """Run the scan's bounded wait on a barrier nothing completes; returns how many CTAs gave up."""
    n = ctypes.c_int32(0)
    check(load().di_selftest_wait(int(polls), int(ctas), ctypes.byref(n)))
    return n.value


def di_graph_create(n, row_ptr, col_idx, d, V=None, stream=None) -> int:
    """Create a device graph; returns the opaque handle (an int)."""
    lib = load()
    out = ctypes.c_void_p()
    nnz = int(len(col_idx)) if col_idx is not None else 0
    if stream is None:
        stream = _lib.current_stream()
    check(lib.di_graph_create(int(n), ptr(row_ptr), ptr(col_idx) if nnz else None, nnz, float(d), ptr(V), stream,
                              ctypes.byref(out)))
    return out.value


def di_free(handle) -> None:
    if handle:
        load().di_free(handle)


def di_solve(handle, tol, H_out, max_edge_pushes=0, prec=DI_FP64, normalize=0, allow_unconverged=False):
    st = di_stats()
    ok = (DI_OK, DI_ENOTCONVERGED) if allow_unconverged else (DI_OK,)
    rc = check(load().di_solve(handle, float(tol), int(max_edge_pushes), int(prec), ptr(H_out), int(normalize),
                               ctypes.byref(st)), ok)
    return rc, st.as_dict()


def _opts(tol, beta, max_edge_pushes, max_sweeps, prec, normalize, trace, profile, select, direction=0,
          scan_wait_polls=0):
    sel = _lib.SELECT[select] if isinstance(select, str) else int(select)
    return di_solve_opts(float(tol), float(beta), int(max_edge_pushes), int(max_sweeps), int(prec), int(normalize),
                         int(trace), int(profile), sel, int(direction), int(scan_wait_polls))


def di_solve_ex(handle, H_out, tol, beta=0.5, max_edge_pushes=0, max_sweeps=0, prec=DI_FP64, normalize=0, trace=0,
                profile=0, allow_unconverged=False, select="ref", direction=0, scan_wait_polls=0):
    o = _opts(tol, beta, max_edge_pushes, max_sweeps, prec, normalize, trace, profile, select, direction,
              scan_wait_polls)
    st = di_stats()
    ok = (DI_OK, DI_ENOTCONVERGED) if allow_unconverged else (DI_OK,)
    rc = check(load().di_solve_ex(handle, ctypes.byref(o), ptr(H_out), ctypes.byref(st)), ok)
    return rc, st.as_dict()


def di_autotune(handle, tol, prec=DI_FP64, max_sweeps=0, max_edge_pushes=0):
    """Time one solve per (beta, select, direction, push CTAs per SM) candidate; returns (best, tried)."""
    o = _opts(tol, 0.5, max_edge_pushes, max_sweeps, prec, 0, 0, 0, 0)
    best = di_tune_result()
    cap = 128
    tried = (di_tune_result * cap)()
    n = ctypes.c_int32(0)
    check(load().di_autotune(handle, ctypes.byref(o), ctypes.byref(best), tried, cap, ctypes.byref(n)))
    return best.as_dict(), [tried[i].as_dict() for i in range(min(n.value, cap))]


def di_solve_update(old_handle, new_handle, H_out, tol, beta=0.5, max_edge_pushes=0, max_sweeps=0, trace=0,
                    profile=0, allow_unconverged=False, select="ref", direction=0):
    """Continue old_handle's FP64 state on the updated graph new_handle (Section 3.2)."""
    o = _opts(tol, beta, max_edge_pushes, max_sweeps, DI_FP64, 0, trace, profile, select, direction)
    st = di_stats()
    ok = (DI_OK, DI_ENOTCONVERGED) if allow_unconverged else (DI_OK,)
    rc = check(load().di_solve_update(old_handle, new_handle, ctypes.byref(o), ptr(H_out), ctypes.byref(st)), ok)
    return rc, st.as_dict()


def di_query(handle, seeds, w, tol, H_out, prec=DI_FP64):
    st = di_stats()
    check(load().di_query(handle, ptr(seeds), ptr(w), int(len(seeds)), float(tol), int(prec), ptr(H_out),
                          ctypes.byref(st)))
    return st.as_dict()


def di_query_batch(handle, seed_lists, tol, H_out, weights=None):
    """Up to 64 personalized queries at once; seed_lists is a list of seed-id arrays.

    Returns (per-query stats list, batch stats).  H_out is double[k][n] (host or device).
    """
    st_q, st_all, _ = di_query_batch_ex(handle, seed_lists, tol, H_out, weights, profile=0)
    return st_q, st_all


def _batch_arrays(seed_lists, weights):
    """seed_ptr, seeds and weights (or None) of a batch, as the C calls take them."""
    k = len(seed_lists)
    seed_ptr = np.zeros(k + 1, np.int32)
    seed_ptr[1:] = np.cumsum([len(s) for s in seed_lists])
    seeds = np.ascontiguousarray(np.concatenate([np.asarray(s, np.int32) for s in seed_lists] or
                                                [np.zeros(1, np.int32)]), dtype=np.int32)
    w = None
    if weights is not None:
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64) for x in weights]), dtype=np.float64)
    return seed_ptr, seeds, w


def di_autotune_batch(handle, seed_lists, tol, weights=None, cap=64):
    """Tune the batched loop for this batch's row width (class cutoffs, beta, dense-sweep share,
    grid, width); returns (best, tried) as dicts.  The winners stay set on the graph."""
    seed_ptr, seeds, w = _batch_arrays(seed_lists, weights)
    best = di_batch_tune_result()
    tried = (di_batch_tune_result * cap)()
    n = ctypes.c_int32(0)
    check(load().di_autotune_batch(handle, len(seed_lists), ptr(seed_ptr), ptr(seeds), ptr(w), float(tol),
                                   ctypes.byref(best), tried, cap, ctypes.byref(n)))
    return best.as_dict(), [tried[i].as_dict() for i in range(min(n.value, cap))]


def di_query_batch_ex(handle, seed_lists, tol, H_out, weights=None, profile=0):
    """di_query_batch with the profiling switch: profile=1 launches the sweep kernels from the
    host with events around them.  Returns (per-query stats, batch stats, profile dict or None).
    """
    k = len(seed_lists)
    seed_ptr, seeds, w = _batch_arrays(seed_lists, weights)
    st_q = (di_stats * max(k, 1))()
    st_all = di_stats()
    prof = di_profile()
    check(load().di_query_batch_ex(handle, k, ptr(seed_ptr), ptr(seeds), ptr(w), float(tol), int(profile),
                                   ptr(H_out), st_q, ctypes.byref(st_all), ctypes.byref(prof)))
    return [st_q[i].as_dict() for i in range(k)], st_all.as_dict(), prof.as_dict() if profile else None


def di_power(handle, tol, X_out, max_iter=0, allow_unconverged=False):
    st = di_stats()
    ok = (DI_OK, DI_ENOTCONVERGED) if allow_unconverged else (DI_OK,)
    rc = check(load().di_power(handle, float(tol), int(max_iter), ptr(X_out), ctypes.byref(st)), ok)
    return rc, st.as_dict()


def di_power_ex(handle, tol, X_out, max_iter=0, profile=0, allow_unconverged=False):
    st = di_stats()
    pm, fm = ctypes.c_double(0), ctypes.c_double(0)
    ok = (DI_OK, DI_ENOTCONVERGED) if allow_unconverged else (DI_OK,)
    rc = check(load().di_power_ex(handle, float(tol), int(max_iter), int(profile), ptr(X_out), ctypes.byref(st),
                                  ctypes.byref(pm), ctypes.byref(fm)), ok)
    d = st.as_dict()
    d["pull_ms"], d["finalize_ms"] = pm.value, fm.value
    return rc, d


def di_power_noalloc(n, in_ptr, in_src, row_ptr, d, tol, X_out, max_iter=0, stream=None, allow_unconverged=False):
    """Power iteration on caller-owned device arrays that allocates no device memory (n <= 65536).

    For callers that cannot allocate (inside a CUDA-graph capture, fixed memory
    pools, hosts that own the allocator).  All arrays must be device memory.
    """
    st = di_stats()
    if stream is None:
        stream = _lib.current_stream()
    ok = (DI_OK, DI_ENOTCONVERGED) if allow_unconverged else (DI_OK,)
    rc = check(load().di_power_noalloc(int(n), ptr(in_ptr), ptr(in_src), int(len(in_src)), ptr(row_ptr), float(d),
                                       float(tol), int(max_iter), ptr(X_out), ctypes.byref(st), stream), ok)
    return rc, st.as_dict()


def di_graph_export(handle, perm=None, outdeg=None, in_ptr=None, in_src=None, bin_of=None, in_bin_of=None, cuts=None):
    check(load().di_graph_export(handle, ptr(perm), ptr(outdeg), ptr(in_ptr), ptr(in_src), ptr(bin_of),
                                 ptr(in_bin_of), ptr(cuts)))


def di_get_trace(handle, cap=4096):
    recs = (di_sweep_record * max(cap, 1))()
    cnt = ctypes.c_int32(0)
    check(load().di_get_trace(handle, recs, int(cap), ctypes.byref(cnt)))
    k = min(cnt.value, cap)
    return [{f: getattr(recs[i], f) for f, _ in di_sweep_record._fields_} for i in range(k)]


def di_get_state(handle, F_out=None, H_out=None):
    check(load().di_get_state(handle, ptr(F_out), ptr(H_out)))


def di_set_state(handle, F_in, H_in, rtol=1e-9) -> float:
    """Load a saved (F, H) after the library's Theorem 1 check; returns the relative deviation."""
    dev = ctypes.c_double(0.0)
    check(load().di_set_state(handle, ptr(F_in), ptr(H_in), float(rtol), ctypes.byref(dev)))
    return dev.value


def di_get_profile(handle) -> dict:
    p = di_profile()
    check(load().di_get_profile(handle, ctypes.byref(p)))
    return p.as_dict()


class DiGraph:
    """A device-resident graph (CSR of out-links) with damping d and personalization V."""

    def __init__(self, n, row_ptr, col_idx, d=0.85, V=None, stream=None):
        self.n = int(n)
        self.nnz = int(len(col_idx))
        self.d = float(d)
        self.handle = di_graph_create(n, np.ascontiguousarray(row_ptr, dtype=np.int32)
                                      if isinstance(row_ptr, (list, np.ndarray)) else row_ptr,
                                      np.ascontiguousarray(col_idx, dtype=np.int32)
                                      if isinstance(col_idx, (list, np.ndarray)) else col_idx,
                                      d, V, stream)

    def close(self):
        if self.handle:
            di_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, tol, H_out=None, **kw):
        """D-iteration to |F|_1/(1-d) <= tol; returns (H, stats)."""
        H = H_out if H_out is not None else np.empty(self.n, dtype=np.float64)
        _rc, st = di_solve_ex(self.handle, H, tol, **kw)
        return H, st

    def autotune(self, tol, prec=DI_FP64, **kw):
        """Fastest (beta, select, direction, push grid) for this graph and target; the push grid stays set."""
        return di_autotune(self.handle, tol, prec, **kw)

    def update_from(self, old, tol, H_out=None, **kw):
        """Continue `old`'s last FP64 solve on this (updated) graph (Section 3.2); returns (H, stats)."""
        H = H_out if H_out is not None else np.empty(self.n, dtype=np.float64)
        _rc, st = di_solve_update(old.handle, self.handle, H, tol, **kw)
        return H, st

    def query(self, seeds, tol, w=None, H_out=None, prec=DI_FP64):
        H = H_out if H_out is not None else np.empty(self.n, dtype=np.float64)
        s = np.ascontiguousarray(seeds, dtype=np.int32) if isinstance(seeds, (list, np.ndarray)) else seeds
        ww = np.ascontiguousarray(w, dtype=np.float64) if isinstance(w, (list, np.ndarray)) else w
        st = di_query(self.handle, s, ww, tol, H, prec)
        return H, st

    def autotune_batch(self, seed_lists, tol, weights=None):
        return di_autotune_batch(self.handle, seed_lists, tol, weights)

    def query_batch(self, seed_lists, tol, H_out=None, weights=None, profile=0):
        """Personalized queries solved together; returns (H [k, n], per-query stats, batch stats).
        With profile=1 the batch stats carry the kernel split under "profile"."""
        H = H_out if H_out is not None else np.empty((len(seed_lists), self.n), dtype=np.float64)
        st_q, st_all, prof = di_query_batch_ex(self.handle, seed_lists, tol, H, weights, profile)
        if prof is not None:
            st_all["profile"] = prof
        return H, st_q, st_all

    def power(self, tol, X_out=None, max_iter=0, allow_unconverged=False, profile=0):
        X = X_out if X_out is not None else np.empty(self.n, dtype=np.float64)
        _rc, st = di_power_ex(self.handle, tol, X, max_iter, profile, allow_unconverged)
        return X, st

    def export(self):
        n, L = self.n, self.nnz
        out = {"perm": np.empty(n, np.int32), "outdeg": np.empty(n, np.int32), "in_ptr": np.empty(n + 1, np.int32),
               "in_src": np.empty(max(L, 1), np.int32), "bin_of": np.empty(n, np.int32),
               "in_bin_of": np.empty(n, np.int32), "cuts": np.empty(4, np.int32)}
        di_graph_export(self.handle, **out)
        out["in_src"] = out["in_src"][:L]
        return out

    def hot_targets(self):
        ids = np.empty(256, np.int32)
        cnt = ctypes.c_int32(0)
        check(load().di_graph_hot_targets(self.handle, ptr(ids), ctypes.byref(cnt)))
        return ids[:cnt.value].copy()

    def trace(self, cap=4096):
        return di_get_trace(self.handle, cap)

    def profile(self):
        return di_get_profile(self.handle)

    def state(self):
        F = np.empty(self.n, np.float64)
        H = np.empty(self.n, np.float64)
        di_get_state(self.handle, F, H)
        return F, H

    def set_state(self, F, H, rtol=1e-9):
        return di_set_state(self.handle, np.ascontiguousarray(F, np.float64) if isinstance(F, np.ndarray) else F,
                            np.ascontiguousarray(H, np.float64) if isinstance(H, np.ndarray) else H, rtol)


# ------------------------------------------------------------------ serving

def di_clock() -> float:
    """Seconds on the library's monotonic clock (the clock of di_completion times)."""
    return load().di_clock()


def di_plan_lanes(lane_bytes, fixed_bytes, budget) -> list:
    """Lanes per graph (64/32/16/8) under a device-memory budget (host only)."""
    lb = np.ascontiguousarray(lane_bytes, dtype=np.int64)
    fb = np.ascontiguousarray(fixed_bytes, dtype=np.int64)
    out = np.empty(len(lb), np.int32)
    check(load().di_plan_lanes(ptr(lb), ptr(fb), len(lb), int(budget), ptr(out)))
    return out.tolist()


def di_server_create(graph_handles, mem_budget=0, round_sweeps=16, lane_sweeps=100000) -> int:
    arr = (ctypes.c_void_p * len(graph_handles))(*graph_handles)
    out = ctypes.c_void_p()
    check(load().di_server_create(ctypes.cast(arr, ctypes.c_void_p), len(graph_handles), int(mem_budget),
                                  int(round_sweeps), int(lane_sweeps), ctypes.byref(out)))
    return out.value


def di_server_lanes(handle, ngraphs) -> list:
    out = np.empty(ngraphs, np.int32)
    check(load().di_server_lanes(handle, ptr(out)))
    return out.tolist()


def di_server_submit(handle, graph, seeds, tol, H_out=None, w=None) -> int:
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    t = ctypes.c_int64(0)
    check(load().di_server_submit(handle, int(graph), ptr(s), ptr(ww), len(s), float(tol), ptr(H_out),
                                  ctypes.byref(t)))
    return t.value


def di_server_poll(handle, wait_s=0.0, cap=256) -> list:
    out = (di_completion * cap)()
    n = ctypes.c_int32(0)
    check(load().di_server_poll(handle, float(wait_s), out, cap, ctypes.byref(n)))
    return [out[i].as_dict() for i in range(n.value)]


def di_server_stats(handle, graph) -> dict:
    st = di_server_graph_stats()
    check(load().di_server_stats(handle, int(graph), ctypes.byref(st)))
    return st.as_dict()


def di_server_pending(handle) -> tuple:
    q, r = ctypes.c_int64(0), ctypes.c_int64(0)
    check(load().di_server_pending(handle, ctypes.byref(q), ctypes.byref(r)))
    return q.value, r.value


def di_server_cancel(handle, ticket) -> bool:
    c = ctypes.c_int32(0)
    check(load().di_server_cancel(handle, int(ticket), ctypes.byref(c)))
    return bool(c.value)


def di_server_free(handle) -> None:
    if handle:
        load().di_server_free(handle)


class DiServer:
    """Continuous batching of personalized queries over several DiGraphs.

    ``submit`` queues a query and returns its ticket; ``poll`` advances every
    graph's lanes and returns finished queries (dicts of di_completion fields).
    The H of a query is written to the buffer given at submit (n doubles: numpy,
    pinned or CUDA tensor), or dropped when none is given.
    """

    def __init__(self, graphs, mem_budget=0, round_sweeps=16, lane_sweeps=100000):
        self.graphs = list(graphs)
        self.handle = di_server_create([g.handle for g in self.graphs], mem_budget, round_sweeps, lane_sweeps)
        self._keep = {}   # ticket -> output buffer, alive until the query completes

    def lanes(self):
        return di_server_lanes(self.handle, len(self.graphs))

    def submit(self, graph, seeds, tol, H_out=None, w=None):
        t = di_server_submit(self.handle, graph, seeds, tol, H_out, w)
        if H_out is not None:
            self._keep[t] = H_out
        return t

    def poll(self, wait_s=0.0, cap=256):
        done = di_server_poll(self.handle, wait_s, cap)
        for c in done:
            self._keep.pop(c["ticket"], None)
        return done

    def pending(self):
        return di_server_pending(self.handle)

    def cancel(self, ticket):
        """Withdraw a queued or running query; True when it was withdrawn (no completion follows)."""
        ok = di_server_cancel(self.handle, ticket)
        if ok:
            self._keep.pop(ticket, None)
        return ok

    def stats(self, graph):
        return di_server_stats(self.handle, graph)

    def drain(self, timeout_s=600.0):
        """Poll until nothing is queued or running; returns every completion seen."""
        out = []
        t_end = di_clock() + timeout_s
        while True:
            q, r = self.pending()
            if q == 0 and r == 0:
                return out
            if di_clock() > t_end:
                raise DiError(_lib.DI_ETIMEOUT, "drain timed out")
            out += self.poll(0.05)

    def close(self):
        if self.handle:
            di_server_free(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
