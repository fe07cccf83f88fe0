"""ctypes binding of the C ABI in include/msf.h (argument marshalling only).

Every function keeps the C name and signature; pointers are passed as
integers (``tensor.data_ptr()`` or ``ndarray.ctypes.data``) and streams as
``torch.cuda.Stream.cuda_stream`` handles.  The shared library is built
in-tree by ``build_lib.build()``; importing this module raises when it is
missing, so nothing can silently run elsewhere.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmsf.so")

MSF_F32, MSF_U32 = 0, 1
MSF_OK = 0
STATUS_NAMES = {
    0: "MSF_OK", 1: "MSF_ERR_INVALID_ARG", 2: "MSF_ERR_OOM", 3: "MSF_ERR_CUDA",
    4: "MSF_ERR_ROUND_LIMIT", 5: "MSF_ERR_SHORTCUT_LIMIT", 6: "MSF_ERR_TOO_LARGE", 7: "MSF_ERR_CHECK",
}
(OPT_COMPACT_TAU, OPT_ROUND_LIMIT, OPT_JUMP_LIMIT, OPT_SLOTS_PER_LANE, OPT_BLOCKS_PER_SM, OPT_PREFETCH,
 OPT_EXEC_MODE, OPT_SHORTCUT, OPT_OS_THRESHOLD, OPT_KERNEL, OPT_BUILD, OPT_EARLY_STOP, OPT_SWEEP,
 OPT_HOST_INPUT, OPT_RELABEL) = range(15)
SHORTCUT_CSP, SHORTCUT_ORIGINAL, SHORTCUT_FULL, SHORTCUT_OPTIMIZED = range(4)

# Every symbol include/msf.h declares.
EXPORTS = ["msf_build_csr", "msf_compute", "msf_compute_batched", "msf_free", "msf_last_error",
           "msf_min_edge", "msf_weight_backward", "msf_get_stats", "msf_set_option", "msf_get_option",
           "msf_forest_weight_noalloc", "msf_connected_components", "msf_min_edge_part", "msf_apply_round"]


class MsfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rows", ctypes.c_int64), ("rounds", ctypes.c_int32), ("compactions", ctypes.c_int32),
                ("forest_edges", ctypes.c_int64), ("jump_steps", ctypes.c_int32), ("min_edge_ms", ctypes.c_float),
                ("cc_rounds", ctypes.c_int32), ("kernels", ctypes.c_int32), ("builder", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libmsf.so; raises FileNotFoundError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run paper_2110_04865_gb300.build_lib.build()")
    lib = ctypes.CDLL(path)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.msf_build_csr.argtypes = [I64, I64, P, P, P, P, ctypes.c_int, ctypes.c_uint32, P, ctypes.POINTER(P)]
    lib.msf_build_csr.restype = ctypes.c_int
    lib.msf_compute.argtypes = [P, P, P, P, P]
    lib.msf_compute.restype = ctypes.c_int
    lib.msf_compute_batched.argtypes = [I32, P, P, P, P, P, ctypes.c_int, P, P, P, P]
    lib.msf_compute_batched.restype = ctypes.c_int
    lib.msf_free.argtypes = [P]
    lib.msf_free.restype = None
    lib.msf_last_error.argtypes = []
    lib.msf_last_error.restype = ctypes.c_char_p
    lib.msf_min_edge.argtypes = [P, P, P, P]
    lib.msf_min_edge.restype = ctypes.c_int
    lib.msf_weight_backward.argtypes = [I64, I32, P, P, P, P, P]
    lib.msf_weight_backward.restype = ctypes.c_int
    lib.msf_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.msf_get_stats.restype = ctypes.c_int
    lib.msf_set_option.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.msf_set_option.restype = ctypes.c_int
    lib.msf_get_option.argtypes = [ctypes.c_int]
    lib.msf_get_option.restype = ctypes.c_double
    lib.msf_connected_components.argtypes = [P, P, P]
    lib.msf_connected_components.restype = ctypes.c_int
    lib.msf_forest_weight_noalloc.argtypes = [I32, I64, P, P, P, ctypes.c_int, P, P]
    lib.msf_forest_weight_noalloc.restype = ctypes.c_int
    lib.msf_min_edge_part.argtypes = [P, P, I32, I32, P, P]
    lib.msf_min_edge_part.restype = ctypes.c_int
    lib.msf_apply_round.argtypes = [P, P, P, P, P, ctypes.POINTER(I64), P]
    lib.msf_apply_round.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != MSF_OK:
        raise MsfError(rc, (load().msf_last_error() or b"").decode())


def msf_build_csr(n, m, src, dst, row_ptr, w, wtype, flags=0, stream=0) -> int:
    out = ctypes.c_void_p()
    _check(load().msf_build_csr(n, m, src or None, dst or None, row_ptr or None, w or None, wtype, flags,
                                stream or None, ctypes.byref(out)))
    return out.value


def msf_compute(g, edge_mask, labels, total, stream=0):
    _check(load().msf_compute(g, edge_mask or None, labels or None, total or None, stream or None))


def msf_compute_batched(G, voff, eoff, src, dst, w, wtype, edge_mask, labels, totals, stream=0):
    _check(load().msf_compute_batched(G, voff, eoff, src or None, dst or None, w or None, wtype,
                                      edge_mask or None, labels or None, totals or None, stream or None))


def msf_free(g):
    if g:
        load().msf_free(g)


def msf_last_error() -> str:
    return (load().msf_last_error() or b"").decode()


def msf_min_edge(g, parent, r, stream=0):
    _check(load().msf_min_edge(g, parent, r, stream or None))


def msf_weight_backward(m, G, eoff, edge_mask, grad_total, grad_w, stream=0):
    _check(load().msf_weight_backward(m, G, eoff or None, edge_mask, grad_total, grad_w, stream or None))


def msf_get_stats(g) -> Stats:
    st = Stats()
    _check(load().msf_get_stats(g, ctypes.byref(st)))
    return st


def msf_set_option(option: int, value: float):
    _check(load().msf_set_option(option, float(value)))


def msf_get_option(option: int) -> float:
    return float(load().msf_get_option(option))


def msf_connected_components(g, labels, stream=0):
    _check(load().msf_connected_components(g, labels, stream or None))


def msf_forest_weight_noalloc(G, m, eoff, edge_mask, w, wtype, totals, stream=0):
    _check(load().msf_forest_weight_noalloc(G, m, eoff or None, edge_mask or None, w or None, wtype,
                                            totals or None, stream or None))


def msf_min_edge_part(g, parent, part, nparts, r, stream=0):
    _check(load().msf_min_edge_part(g, parent, part, nparts, r, stream or None))


def msf_apply_round(g, r, parent, edge_mask, labels, stream=0) -> int:
    """Returns the number of roots that hooked in the round."""
    hooks = ctypes.c_int64(0)
    _check(load().msf_apply_round(g, r, parent, edge_mask, labels or None, ctypes.byref(hooks), stream or None))
    return int(hooks.value)
