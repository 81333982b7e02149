"""ctypes binding of libditer.so: the C ABI of include/diter.h, argument marshalling only.

Every function here passes pointers and sizes to the library and converts the
status code into an exception; no step of the method runs in Python.  Arrays
may be numpy arrays (host) or torch tensors (host or CUDA); torch is used for
device memory and the current stream only.  If libditer.so is missing or cannot
be loaded the import fails with an error: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DI_LIB_VARIANT=debug loads the DI_DEBUG build (device-side index checks) instead
LIB_PATH = os.path.join(HERE, "libditer_debug.so" if os.environ.get("DI_LIB_VARIANT") == "debug" else "libditer.so")

DI_OK, DI_EINVAL, DI_ENOMEM, DI_ECUDA, DI_ENOTCONVERGED, DI_ETIMEOUT, DI_EKERNEL = range(7)
DI_FP64, DI_FP32_MIXED = 0, 1
DI_SELECT_REF, DI_SELECT_OP, DI_SELECT_OP2 = 0, 1, 2
SELECT = {"ref": DI_SELECT_REF, "op": DI_SELECT_OP, "op2": DI_SELECT_OP2}
STATUS_NAMES = {0: "DI_OK", 1: "DI_EINVAL", 2: "DI_ENOMEM", 3: "DI_ECUDA", 4: "DI_ENOTCONVERGED", 5: "DI_ETIMEOUT",
                6: "DI_EKERNEL"}


class DiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class di_stats(ctypes.Structure):
    _fields_ = [("bound", ctypes.c_double), ("l1_F", ctypes.c_double), ("R", ctypes.c_double),
                ("edges_pushed", ctypes.c_int64), ("sources_pushed", ctypes.c_int64), ("sweeps", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class di_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("beta", ctypes.c_double), ("max_edge_pushes", ctypes.c_int64),
                ("max_sweeps", ctypes.c_int32), ("prec", ctypes.c_int32), ("normalize", ctypes.c_int32),
                ("trace", ctypes.c_int32), ("profile", ctypes.c_int32), ("select", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("scan_wait_polls", ctypes.c_int32)]


class di_sweep_record(ctypes.Structure):
    _fields_ = [("l1_F", ctypes.c_double), ("removed", ctypes.c_double), ("R", ctypes.c_double), ("T", ctypes.c_double),
                ("sources", ctypes.c_int64), ("edges", ctypes.c_int64), ("pushed", ctypes.c_int64),
                ("scan_ms", ctypes.c_double), ("push_ms", ctypes.c_double), ("pull", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class di_profile(ctypes.Structure):
    _fields_ = [("scan_ms", ctypes.c_double), ("push_ms", ctypes.c_double), ("finalize_ms", ctypes.c_double),
                ("sweeps", ctypes.c_int32), ("pull_sweeps", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class di_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("graph", ctypes.c_int32), ("status", ctypes.c_int32),
                ("bound", ctypes.c_double), ("sweeps", ctypes.c_int32), ("lane", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class di_tune_result(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("select", ctypes.c_int32), ("push_ctas_per_sm", ctypes.c_int32),
                ("ms", ctypes.c_double), ("edges_pushed", ctypes.c_int64), ("sweeps", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("cut1", ctypes.c_int32), ("cut2", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class di_batch_tune_result(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("ms", ctypes.c_double), ("max_bound", ctypes.c_double),
                ("edges_pushed", ctypes.c_int64), ("sweeps", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("pull_share", ctypes.c_int32), ("push_ctas_per_sm", ctypes.c_int32), ("cut1", ctypes.c_int32),
                ("cut2", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class di_server_graph_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("sweeps", ctypes.c_int64), ("edges_pushed", ctypes.c_int64),
                ("sources_pushed", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("width_sweeps", ctypes.c_int64), ("device_ms", ctypes.c_double), ("lanes", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("cancelled", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_lib = None


def load(path: str = LIB_PATH):
    """Load libditer.so and declare every entry point of include/diter.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "di_graph_create": ([i32, vp, vp, i64, f64, vp, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "di_free": ([vp], None),
        "di_graph_info": ([vp, vp, vp, vp], ctypes.c_int),
        "di_graph_export": ([vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "di_graph_hot_targets": ([vp, vp, ctypes.POINTER(i32)], ctypes.c_int),
        "di_solve": ([vp, f64, i64, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(di_stats)], ctypes.c_int),
        "di_solve_ex": ([vp, ctypes.POINTER(di_solve_opts), vp, ctypes.POINTER(di_stats)], ctypes.c_int),
        "di_autotune": ([vp, ctypes.POINTER(di_solve_opts), ctypes.POINTER(di_tune_result), vp, i32,
                         ctypes.POINTER(i32)], ctypes.c_int),
        "di_autotune_batch": ([vp, i32, vp, vp, vp, f64, ctypes.POINTER(di_batch_tune_result), vp, i32,
                               ctypes.POINTER(i32)], ctypes.c_int),
        "di_solve_update": ([vp, vp, ctypes.POINTER(di_solve_opts), vp, ctypes.POINTER(di_stats)], ctypes.c_int),
        "di_query": ([vp, vp, vp, i32, f64, ctypes.c_int, vp, ctypes.POINTER(di_stats)], ctypes.c_int),
        "di_power": ([vp, f64, i32, vp, ctypes.POINTER(di_stats)], ctypes.c_int),
        "di_query_batch": ([vp, i32, vp, vp, vp, f64, vp, vp, ctypes.POINTER(di_stats)], ctypes.c_int),
        "di_query_batch_ex": ([vp, i32, vp, vp, vp, f64, i32, vp, vp, ctypes.POINTER(di_stats),
                               ctypes.POINTER(di_profile)], ctypes.c_int),
        "di_power_ex": ([vp, f64, i32, i32, vp, ctypes.POINTER(di_stats), ctypes.POINTER(f64), ctypes.POINTER(f64)],
                        ctypes.c_int),
        "di_get_trace": ([vp, vp, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "di_get_state": ([vp, vp, vp], ctypes.c_int),
        "di_set_state": ([vp, vp, vp, f64, ctypes.POINTER(f64)], ctypes.c_int),
        "di_get_profile": ([vp, ctypes.POINTER(di_profile)], ctypes.c_int),
        "di_power_noalloc": ([i32, vp, vp, i64, vp, f64, f64, i32, vp, ctypes.POINTER(di_stats), vp], ctypes.c_int),
        "di_plan_lanes": ([vp, vp, i32, i64, vp], ctypes.c_int),
        "di_server_create": ([vp, i32, i64, i32, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "di_server_lanes": ([vp, vp], ctypes.c_int),
        "di_server_submit": ([vp, i32, vp, vp, i32, f64, vp, ctypes.POINTER(i64)], ctypes.c_int),
        "di_server_poll": ([vp, f64, vp, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "di_server_stats": ([vp, i32, ctypes.POINTER(di_server_graph_stats)], ctypes.c_int),
        "di_server_pending": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "di_server_cancel": ([vp, i64, ctypes.POINTER(i32)], ctypes.c_int),
        "di_server_free": ([vp], None),
        "di_clock": ([], f64),
        "di_last_error": ([], ctypes.c_char_p),
        "di_version": ([], ctypes.c_char_p),
        "di_selftest_wait": ([i32, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "di_debug_build": ([], i32),
        "di_debug_selftest": ([ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status: int, ok=(DI_OK,)) -> int:
    if status not in ok:
        raise DiError(status, load().di_last_error().decode())
    return status


def ptr(a) -> int | None:
    """Raw address of a numpy array or torch tensor (host or device); None for None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def current_stream() -> int | None:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None
