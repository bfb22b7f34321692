"""torch.autograd.Function over rpp_barcodes_batched / rpp_barcodes_backward.

Forward computes the barcodes of a batch of clouds on the GPU; the interval
endpoints come back as CUDA tensors. Backward calls the library's backward
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


def _flatten(handles):
    """births, deaths, cloud index, dimension of every interval, in
    (cloud, dimension, interval) order."""
    L = N.lib()
    births, deaths, cloud, dims = [], [], [], []
    for i, h in enumerate(handles):
        st = N.Stats()
        N.check(L.rpp_result_stats(h, C.byref(st)), "rpp_result_stats")
        for q in range(st.max_dim + 1):
            k = L.rpp_result_count(h, q)
            if k <= 0:
                continue
            iv = np.ctypeslib.as_array(C.cast(L.rpp_result_intervals(h, q), C.POINTER(C.c_float)),
                                       shape=(2 * k,)).reshape(k, 2)
            births.append(iv[:, 0].copy())
            deaths.append(iv[:, 1].copy())
            cloud.append(np.full(k, i, np.int64))
            dims.append(np.full(k, q, np.int64))
    if not births:
        z = np.zeros(0, np.float32)
        return z, z, np.zeros(0, np.int64), np.zeros(0, np.int64)
    return (np.concatenate(births), np.concatenate(deaths), np.concatenate(cloud),
            np.concatenate(dims))


class RipsPersistence(torch.autograd.Function):
    """points (B, n, d) CUDA float32 -> (births, deaths, cloud, dim) over every
    interval of every cloud; births and deaths are differentiable."""

    @staticmethod
    def forward(ctx, points, max_dim: int):
        lctx, handles = _forward_handles(points, max_dim)
        keep = _Handles(handles)
        b, d, cl, dm = _flatten(handles)
        dev = points.device
        ctx.keep = keep
        ctx.lctx = lctx
        ctx.save_for_backward(points)
        births = torch.from_numpy(b).to(dev)
        deaths = torch.from_numpy(d).to(dev)
        cloud = torch.from_numpy(cl).to(dev)
        dims = torch.from_numpy(dm).to(dev)
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
