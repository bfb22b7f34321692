"""torch.autograd.Function over rpp_barcodes_batched / rpp_barcodes_backward.

Forward computes the barcodes of a batch of clouds on the GPU; the interval
endpoints come back as CUDA tensors (gathered from every result at once and
copied to the device in one pinned transfer per dtype). Backward calls the library's backward
kernel, which sends each endpoint's gradient to the two points of the edge
that realises it (an endpoint is the length of that edge).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N
from .api import default_context, _take_result, _stats_dict


class _Handles:
    """Keeps the library's result handles alive until backward has run."""

    def __init__(self, handles):
        self.handles = handles

    def __del__(self):
        L = N.lib()
        for h in self.handles:
            if h:
                L.rpp_result_free(h)


def _forward_handles(points: torch.Tensor, max_dim: int, thresholds=None, context=None):
    B, n, d = points.shape
    ctx = context or default_context(points.device.index or 0)
    x = points.detach().contiguous()
    ptrs = (C.c_void_p * B)(*[x[i].data_ptr() for i in range(B)])
    ns = (C.c_int64 * B)(*([n] * B))
    dims = (C.c_int32 * B)(*([d] * B))
    th = (C.c_float * B)(*thresholds) if thresholds is not None else None
    outs = (C.c_void_p * B)()
    s = torch.cuda.current_stream(points.device).cuda_stream
    N.check(N.lib().rpp_barcodes_batched(ctx.handle, B, ptrs, ns, dims, max_dim, th, None, s,
                                         outs), "rpp_barcodes_batched")
    return ctx, [outs[i] for i in range(B)]


def _flatten(handles, max_dim: int):
    """births, deaths (float32 [2, m]) and cloud index, dimension (int64
    [2, m]) of every interval, in (cloud, dimension, interval) order, gathered
    from all results with one rpp_results_gather call per dimension."""
    L = N.lib()
    B = len(handles)
    arr = (C.c_void_p * B)(*handles)
    ivs, clouds, dims = [], [], []
    for q in range(max_dim + 1):
        offs = np.zeros(B + 1, np.int64)
        N.check(L.rpp_results_gather(arr, B, q, offs.ctypes.data, None, None),
                "rpp_results_gather")
        iv = np.empty((int(offs[-1]), 2), np.float32)
        if len(iv):
            N.check(L.rpp_results_gather(arr, B, q, offs.ctypes.data, iv.ctypes.data, None),
                    "rpp_results_gather")
        ivs.append(iv)
        clouds.append(np.repeat(np.arange(B, dtype=np.int64), np.diff(offs)))
        dims.append(np.full(len(iv), q, np.int64))
    iv = np.concatenate(ivs)
    cloud = np.concatenate(clouds)
    dim = np.concatenate(dims)
    order = np.argsort(cloud, kind="stable")  # dimension-major -> cloud-major
    return (np.ascontiguousarray(iv[order].T),
            np.ascontiguousarray(np.stack([cloud[order], dim[order]])))


class RipsPersistence(torch.autograd.Function):
    """points (B, n, d) CUDA float32 -> (births, deaths, cloud, dim) over every
    interval of every cloud; births and deaths are differentiable."""

    @staticmethod
    def forward(ctx, points, max_dim: int):
        # The intervals are formed on the host (the submatrix reduction runs
        # there), so they reach the device once: two pinned buffers, copied
        # without blocking on the points' stream.
        lctx, handles = _forward_handles(points, max_dim)
        keep = _Handles(handles)
        bd, cd = _flatten(handles, max_dim)
        dev = points.device
        ctx.keep = keep
        ctx.lctx = lctx
        ctx.save_for_backward(points)
        f = torch.from_numpy(bd).pin_memory().to(dev, non_blocking=True)
        i = torch.from_numpy(cd).pin_memory().to(dev, non_blocking=True)
        births, deaths = f[0], f[1]
        cloud, dims = i[0], i[1]
        ctx.mark_non_differentiable(cloud, dims)
        return births, deaths, cloud, dims

    @staticmethod
    def backward(ctx, g_birth, g_death, _g_cloud, _g_dim):
        (points,) = ctx.saved_tensors
        B, n, d = points.shape
        x = points.detach().contiguous()
        gb = (g_birth if g_birth is not None else torch.zeros(0, device=points.device)).contiguous().float()
        gd = (g_death if g_death is not None else torch.zeros(0, device=points.device)).contiguous().float()
        total = sum(N.lib().rpp_result_total(h) for h in ctx.keep.handles)
        if gb.numel() != total:
            gb = torch.zeros(total, device=points.device)
        if gd.numel() != total:
            gd = torch.zeros(total, device=points.device)
        grad = torch.empty_like(x)
        hs = (C.c_void_p * B)(*ctx.keep.handles)
        ns = (C.c_int64 * B)(*([n] * B))
        s = torch.cuda.current_stream(points.device).cuda_stream
        N.check(N.lib().rpp_barcodes_backward(ctx.lctx.handle, B, x.data_ptr(), ns, d, hs,
                                              gb.data_ptr(), gd.data_ptr(), grad.data_ptr(), s),
                "rpp_barcodes_backward")
        return grad, None


def rips_persistence(points: torch.Tensor, max_dim: int = 1):
    """(births, deaths, cloud, dim) of a batch of clouds, differentiable."""
    if points.dim() == 2:
        points = points.unsqueeze(0)
    return RipsPersistence.apply(points, max_dim)


def total_persistence(points: torch.Tensor, q: int = 1) -> torch.Tensor:
    """Sum over the finite intervals of dimension q of (death - birth), summed
    over the clouds of the batch."""
    births, deaths, _cloud, dims = rips_persistence(points, max_dim=q)
    mask = (dims == q) & torch.isfinite(deaths)
    return (deaths[mask] - births[mask]).sum()
