"""PyTorch-facing wrappers of the C ABI.

PyTorch supplies device memory and the current stream; every step of the
computation runs in the CUDA library (``_abi``).  Inputs may be CUDA tensors
(the usual case) or numpy arrays in host memory (the library stages them).

Weights: float32 tensors are MSF_F32; int32/uint32 tensors are read as
uint32 words (MSF_U32).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from ._abi import MSF_F32, MSF_U32


def _stream_handle(device) -> int:
    if device is None or (isinstance(device, torch.device) and device.type != "cuda"):
        return int(torch.cuda.current_stream().cuda_stream)
    return int(torch.cuda.current_stream(device).cuda_stream)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _wtype(w) -> int:
    dt = w.dtype
    if dt in (torch.float32, np.float32):
        return MSF_F32
    if dt in (torch.int32, np.int32, np.uint32) or str(dt) == "torch.uint32":
        return MSF_U32
    raise TypeError("weights must be float32 (MSF_F32) or 32-bit integers (MSF_U32)")


def _check_i32(x, name):
    if x.dtype not in (torch.int32, np.int32):
        raise TypeError(f"{name} must be int32")


def _out(like, shape, dtype_t, dtype_np):
    if isinstance(like, torch.Tensor):
        return torch.empty(shape, dtype=dtype_t, device=like.device)
    return np.empty(shape, dtype=dtype_np)


class Graph:
    """A graph stored on the device (msf_build_csr).  COO form by default;
    pass ``row_ptr`` for a symmetric CSR (``dst`` = columns, one weight per
    slot; the slots with row < column are the edges)."""

    def __init__(self, n: int, src, dst, w, row_ptr=None):
        _check_i32(dst, "dst")
        if row_ptr is None:
            _check_i32(src, "src")
        self.n = int(n)
        self.m = int(dst.shape[0])
        self.wtype = _wtype(w)
        self._like = dst
        self.device = dst.device if isinstance(dst, torch.Tensor) else None
        self.handle = _abi.msf_build_csr(self.n, self.m, _ptr(src) if row_ptr is None else 0, _ptr(dst),
                                         _ptr(row_ptr), _ptr(w), self.wtype, 0, _stream_handle(self.device))

    def compute(self, mask: bool = True, labels: bool = True, total: bool = True):
        """Returns (edge_mask uint8[m], labels int32[n], total float64[1])."""
        mk = _out(self._like, (self.m,), torch.uint8, np.uint8) if mask else None
        lb = _out(self._like, (self.n,), torch.int32, np.int32) if labels else None
        tt = _out(self._like, (1,), torch.float64, np.float64) if total else None
        _abi.msf_compute(self.handle, _ptr(mk), _ptr(lb), _ptr(tt), _stream_handle(self.device))
        return mk, lb, tt

    def min_edge(self, parent):
        """One multilinear min-edge application with projection (msf_min_edge)."""
        r = _out(parent, (self.n,), torch.int64, np.uint64)
        _abi.msf_min_edge(self.handle, _ptr(parent), _ptr(r), _stream_handle(self.device))
        return r

    def components(self):
        """Connected-component labels by the Awerbuch-Shiloach connectivity
        algorithm (msf_connected_components): int32[n]."""
        lb = _out(self._like, (self.n,), torch.int32, np.int32)
        _abi.msf_connected_components(self.handle, _ptr(lb), _stream_handle(self.device))
        return lb

    def stats(self) -> _abi.Stats:
        return _abi.msf_get_stats(self.handle)

    def free(self):
        if self.handle:
            _abi.msf_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def compute(n: int, src, dst, w):
    """Minimum spanning forest of one graph: (edge_mask, labels, total)."""
    g = Graph(n, src, dst, w)
    try:
        return g.compute()
    finally:
        g.free()


def compute_batched(voff, eoff, src, dst, w):
    """Forests of a batch of graphs (local vertex ids): (edge_mask, labels, totals).
    ``voff``/``eoff`` are host int64 arrays of length G+1."""
    voff = np.ascontiguousarray(np.asarray(voff, dtype=np.int64))
    eoff = np.ascontiguousarray(np.asarray(eoff, dtype=np.int64))
    G = len(voff) - 1
    mk = _out(dst, (int(eoff[-1]),), torch.uint8, np.uint8)
    lb = _out(dst, (int(voff[-1]),), torch.int32, np.int32)
    tt = _out(dst, (G,), torch.float64, np.float64)
    dev = dst.device if isinstance(dst, torch.Tensor) else None
    _abi.msf_compute_batched(G, voff.ctypes.data, eoff.ctypes.data, _ptr(src), _ptr(dst), _ptr(w), _wtype(w),
                             _ptr(mk), _ptr(lb), _ptr(tt), _stream_handle(dev))
    return mk, lb, tt


@dataclass
class Batch:
    """Structure of a batch of graphs for MSFWeight (weights excluded)."""
    voff: np.ndarray
    eoff: np.ndarray
    src: torch.Tensor
    dst: torch.Tensor

    @staticmethod
    def single(n: int, src, dst) -> "Batch":
        return Batch(np.array([0, n], np.int64), np.array([0, int(dst.shape[0])], np.int64), src, dst)


class MSFWeight(torch.autograd.Function):
    """Total forest weight per graph as a differentiable function of the
    float32 edge weights.  Backward: grad_w[e] = [e in forest] * grad_total[g(e)]
    (msf_weight_backward)."""

    @staticmethod
    def forward(ctx, w: torch.Tensor, batch: Batch):
        if w.dtype != torch.float32:
            raise TypeError("MSFWeight needs float32 weights")
        G = len(batch.voff) - 1
        if G == 1:
            g = Graph(int(batch.voff[-1]), batch.src, batch.dst, w)
            try:
                mask, _, totals = g.compute(labels=False)
            finally:
                g.free()
        else:
            mask, _, totals = compute_batched(batch.voff, batch.eoff, batch.src, batch.dst, w)
        ctx.save_for_backward(mask)
        ctx.eoff = batch.eoff
        ctx.m = int(w.shape[0])
        ctx.mark_non_differentiable(mask)
        return totals, mask

    @staticmethod
    def backward(ctx, grad_totals, grad_mask):
        (mask,) = ctx.saved_tensors
        G = len(ctx.eoff) - 1
        gt = grad_totals.contiguous().to(torch.float64)
        gw = torch.empty(ctx.m, dtype=torch.float32, device=mask.device)
        _abi.msf_weight_backward(ctx.m, G, ctx.eoff.ctypes.data if G > 1 else 0, _ptr(mask), _ptr(gt), _ptr(gw),
                                 _stream_handle(mask.device))
        return gw, None


def msf_weight(w: torch.Tensor, batch: Batch):
    """Differentiable forest weight(s): returns (totals float64[G], mask uint8[m])."""
    return MSFWeight.apply(w, batch)


def set_option(option: int, value: float):
    _abi.msf_set_option(option, value)


def get_option(option: int) -> float:
    return _abi.msf_get_option(option)
