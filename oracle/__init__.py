"""The oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU restatement of what the CUDA path
computes, in FP64, used to check it.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
library itself never does, and the two share no code.

Contents (each function cites the passage it follows):

* :func:`diter`        -- ALGO-REF with the dangling-node rule (Sections 2.2,
  3.3) in the orders of Section 4 (PER, RAND, MAX) and threshold sweeps
  (sequential THRESH and snapshot SWEEP), in C (``oracle.c``).
* :func:`power`        -- MAT-ITER on the uncompleted P with the paper's stop rule.
* :func:`update`       -- the injection F_0' = F_n0 + d(P'-P)H_n0 of the updating
  equation (Section 3.2); :func:`run` then continues on P' (signed fluid).
* :func:`selection_weights` -- the ALGO-OP / ALGO-OP2 weights of Section 4.3,
  used by ``select="op"`` / ``"op2"`` in :func:`run` and :func:`diter`.
* :func:`transpose`, :func:`bins` -- in-link lists and degree bins.
* :func:`power_omp`    -- the same MAT-ITER on all host cores (OpenMP, ``power_omp.c``,
  a separate library): a timed CPU baseline, pinned to :func:`power` by the tests.
* :mod:`oracle.ge`     -- dense Gaussian elimination of (I - dP)X = (1-d)V in FP64
  and in exact rationals (Section 2.1's fixed point written out).

Pins that tie every function to the paper and to mathematics are in
``tests/test_oracle_*.py``.  No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

from . import ge  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

PER, RAND, MAX, THRESH, SWEEP = 0, 1, 2, 3, 4
MODES = {"per": PER, "rand": RAND, "max": MAX, "thresh": THRESH, "sweep": SWEEP}


def build(force: bool = False, out: str | None = None, defines: tuple = ()) -> str:
    """Compile ``oracle.c`` with gcc (single-threaded, -O2, no fast-math)."""
    target = out or _LIB
    if out is None and not force and not defines and os.path.exists(_LIB) \
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(target))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall",
           *[f"-D{d}" for d in defines], "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, target)
    return target


_OMP_SRC = os.path.join(_HERE, "power_omp.c")
_OMP_LIB = os.path.join(_HERE, "libpower_omp.so")
_omp = None


def build_omp(force: bool = False) -> str:
    """Compile ``power_omp.c`` with gcc and OpenMP (the timed multi-core CPU baseline)."""
    if not force and os.path.exists(_OMP_LIB) and os.path.getmtime(_OMP_LIB) >= os.path.getmtime(_OMP_SRC):
        return _OMP_LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall", "-fopenmp", "-o", tmp,
           _OMP_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OMP_LIB)
    return _OMP_LIB


def load_omp():
    global _omp
    if _omp is None:
        lib = ctypes.CDLL(build_omp())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.pomp_threads.argtypes = [ctypes.c_int]
        lib.pomp_threads.restype = ctypes.c_int
        lib.pomp_power.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_double, f64p, ctypes.c_double,
                                   ctypes.c_int64, f64p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        lib.pomp_power.restype = ctypes.c_int
        _omp = lib
    return _omp


class Stats(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("l1F", ctypes.c_double), ("pushes", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("picks", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("converged", ctypes.c_int32)]


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    f64p = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.orc_outdeg.argtypes = [ctypes.c_int32, i32p, i32p]
    lib.orc_transpose.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p]
    lib.orc_bins.argtypes = [ctypes.c_int32, i32p, ctypes.c_int32, i32p, i32p, i32p, i32p]
    lib.orc_init.argtypes = [ctypes.c_int32, ctypes.c_double, f64p, f64p, f64p]
    lib.orc_init.restype = ctypes.c_double
    lib.orc_diter.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_double, f64p, f64p, ctypes.c_double,
                              ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                              ctypes.POINTER(ctypes.c_float), ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                              ctypes.c_int64, ctypes.POINTER(Stats)]
    lib.orc_update_inject.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_double, f64p, f64p]
    lib.orc_diter.restype = ctypes.c_int
    lib.orc_power.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_double, f64p, ctypes.c_double,
                              ctypes.c_int64, f64p, i64p, f64p]
    lib.orc_power.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load the oracle library (building it if needed); ``path`` loads a variant build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(V, n):
    """V as a contiguous float64 array of exactly n entries (the C side reads n values)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.shape != (n,):
        raise ValueError(f"oracle: V must have shape ({n},), got {V.shape}")
    return V


@dataclass
class DiterResult:
    H: np.ndarray
    F: np.ndarray
    R: float
    l1F: float
    pushes: int
    edges: int
    picks: int
    sweeps: int
    converged: bool

    @property
    def bound(self) -> float:
        """|F|_1/(1-d) is computed by the caller; this is the tracked R."""
        return self.R


def init(n, d, V, lib=None):
    """ALGO-REF initialization (Section 2.2): H = 0, F = (1-d)V, R = 1-d."""
    lib = lib or load()
    V = _vec(V, n)
    F = np.empty(n, dtype=np.float64)
    H = np.empty(n, dtype=np.float64)
    R = lib.orc_init(n, d, _f64(V), _f64(F), _f64(H))
    return F, H, R


def selection_weights(n, row_ptr, col_idx, select):
    """ALGO-OP / ALGO-OP2 selection weights (Section 4.3) and the threshold scale.

    "op":  w_i = 1/((#in_i + 1)(#out_i + 1));  "op2": w_i = 1/(#out_i + 1).
    Each weight is the FP64 quotient of 1 by the integer product, rounded to FP32.
    wscale = 2^floor(log2(mean_i w_i)), the mean taken over the FP32 weights in FP64.
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    outdeg = np.diff(row_ptr)
    if select == "op":
        indeg = np.bincount(np.asarray(col_idx, dtype=np.int64), minlength=n)[:n]
        c = (indeg + 1) * (outdeg + 1)
    elif select == "op2":
        c = outdeg + 1
    else:
        raise ValueError(f"unknown selection {select}")
    w = (1.0 / c.astype(np.float64)).astype(np.float32)
    mean = float(np.sum(w.astype(np.float64))) / n
    _m, ex = np.frexp(mean)
    return np.ascontiguousarray(w), float(np.ldexp(1.0, int(ex) - 1))


def run(n, row_ptr, col_idx, d, F, H, R, tol, mode="sweep", beta=0.5, seed=0, max_pushes=1 << 62, lib=None,
        select=None, trace=None):
    """Continue D-iteration on the state (F, H, R) in place (ALGO-REF, Sections 2.2 and 3.3).

    select = "op" / "op2" chooses nodes by |F_i| w_i (Section 4.3) in the MAX and sweep orders.
    trace: a float64 array of shape (cap, 3) that receives (T, R, selected) per snapshot sweep.
    """
    lib = lib or load()
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx if len(col_idx) else np.zeros(1, np.int32))
    st = Stats()
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    wp, wscale = None, 1.0
    if select is not None and select != "ref":
        w, wscale = selection_weights(n, rp, ci[:int(rp[n])], select)
        wp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    tp, tcap = None, 0
    if trace is not None:
        assert trace.dtype == np.float64 and trace.flags["C_CONTIGUOUS"] and trace.shape[1] == 3
        tp, tcap = _f64(trace), trace.shape[0]
    rc = lib.orc_diter(n, rpp, cip, d, _f64(F), _f64(H), R, tol, m, beta, seed, max_pushes, wp, wscale, tp, tcap,
                       ctypes.byref(st))
    if rc < 0:
        raise ValueError(f"oracle: unknown mode {mode}")
    return DiterResult(H, F, st.R, st.l1F, st.pushes, st.edges, st.picks, st.sweeps, bool(st.converged))


def diter(n, row_ptr, col_idx, d, V, tol, mode="sweep", beta=0.5, seed=0, max_pushes=1 << 62, lib=None,
          select=None, trace=None):
    """D-iteration from the initial state to R/(1-d) <= tol (ALGO-REF, Sections 2.2, 3.3, 4)."""
    F, H, R = init(n, d, V, lib)
    return run(n, row_ptr, col_idx, d, F, H, R, tol, mode, beta, seed, max_pushes, lib, select, trace)


def update(n, rp_old, ci_old, rp_new, ci_new, d, F, H, lib=None):
    """F_0' = F + d(P' - P)H (Section 3.2, updating equation); returns a new array."""
    lib = lib or load()
    _a, pa = _i32(rp_old)
    _b, pb = _i32(ci_old if len(ci_old) else np.zeros(1, np.int32))
    _c, pc = _i32(rp_new)
    _e, pe = _i32(ci_new if len(ci_new) else np.zeros(1, np.int32))
    F2 = np.array(F, dtype=np.float64, copy=True)
    Hc = np.ascontiguousarray(H, dtype=np.float64)
    lib.orc_update_inject(n, pa, pb, pc, pe, d, _f64(Hc), _f64(F2))
    return F2


def solve_update(n, rp_old, ci_old, rp_new, ci_new, d, F, H, tol, mode="sweep", beta=0.5, max_pushes=1 << 62,
                 lib=None):
    """Continue a run on P (state F, H) on the updated graph P' to |F'|_1/(1-d) <= tol (Section 3.2)."""
    F2 = update(n, rp_old, ci_old, rp_new, ci_new, d, F, H, lib)
    H2 = np.array(H, dtype=np.float64, copy=True)
    R = float(np.abs(F2).sum())
    return run(n, rp_new, ci_new, d, F2, H2, R, tol, mode, beta, max_pushes=max_pushes, lib=lib)


def power(n, row_ptr, col_idx, d, V, tol, max_iter=100000, lib=None):
    """MAT-ITER from X_0 = 0 on the uncompleted P; returns (X, iterations, last |X_n - X_{n-1}|_1, ok)."""
    lib = lib or load()
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx if len(col_idx) else np.zeros(1, np.int32))
    V = _vec(V, n)
    X = np.empty(n, dtype=np.float64)
    it = ctypes.c_int64(0)
    delta = ctypes.c_double(0)
    rc = lib.orc_power(n, rpp, cip, d, _f64(V), tol, max_iter, _f64(X), ctypes.byref(it), ctypes.byref(delta))
    return X, int(it.value), float(delta.value), rc == 0


def power_omp(n, in_ptr, in_src, outdeg_, d, V, tol, max_iter=100000, threads=0):
    """MAT-ITER (Section 4) on `threads` host cores (0: all), as a pull over the in-link lists
    in_ptr/in_src with out-degrees outdeg_; returns (X, iterations, last |X_n - X_{n-1}|_1, ok,
    threads used)."""
    lib = load_omp()
    used = lib.pomp_threads(int(threads))
    ip, ipp = _i32(in_ptr)
    L = int(ip[-1])
    isrc, isp = _i32(in_src if L else np.zeros(1, np.int32))
    od, odp = _i32(outdeg_)
    V = _vec(V, n)
    X = np.empty(n, dtype=np.float64)
    it = ctypes.c_int64(0)
    delta = ctypes.c_double(0)
    rc = lib.pomp_power(n, ipp, isp, odp, d, _f64(V), tol, max_iter, _f64(X), ctypes.byref(it), ctypes.byref(delta))
    return X, int(it.value), float(delta.value), rc == 0, used


def outdeg(n, row_ptr, lib=None):
    lib = lib or load()
    rp, rpp = _i32(row_ptr)
    out = np.empty(n, dtype=np.int32)
    lib.orc_outdeg(n, rpp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


def transpose(n, row_ptr, col_idx, lib=None):
    """In-link lists: row j holds every source i of an edge i -> j, ascending."""
    lib = lib or load()
    rp, rpp = _i32(row_ptr)
    L = int(rp[-1])
    ci, cip = _i32(col_idx if L else np.zeros(1, np.int32))
    in_ptr = np.empty(n + 1, dtype=np.int32)
    in_src = np.empty(max(L, 1), dtype=np.int32)
    lib.orc_transpose(n, rpp, cip, in_ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      in_src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return in_ptr, in_src[:L]


def bins(n, row_ptr, cuts, lib=None):
    """Degree bins: bin b = number of cuts c with outdeg > c; each bin's ids ascending."""
    lib = lib or load()
    rp, rpp = _i32(row_ptr)
    cu, cup = _i32(np.asarray(cuts, dtype=np.int32))
    nb = len(cuts) + 1
    bin_of = np.empty(n, dtype=np.int32)
    bin_ptr = np.empty(nb + 1, dtype=np.int32)
    bin_ids = np.empty(max(n, 1), dtype=np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
    lib.orc_bins(n, rpp, len(cuts), cup, p(bin_of), p(bin_ptr), p(bin_ids))
    return bin_of, bin_ptr, bin_ids[:n]
