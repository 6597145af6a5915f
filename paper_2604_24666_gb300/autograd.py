"""torch.autograd.Function over the library's encoding + MLP kernels.

`NIFSegments.apply(p0, p1, nif)` evaluates the network on linearized rest
segments (FP32 path): psi(p0) (+) psi(p1) -> MLP -> [n, 16]. Its backward runs
the library's MLP backward and encoding backward: the gradients of the
tables and weights are added into the handle's own gradient buffer (read with
`Nif.get_grads`, applied with `nif_adam_step`), and dL/dp0, dL/dp1 are
returned to autograd. Every step runs in libnif's kernels; torch only holds
the device buffers.
"""
from __future__ import annotations

import torch

from . import nif as N


class NIFSegments(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p0, p1, handle):
        net = handle.net
        n = p0.shape[0]
        lin = torch.zeros((n, 8), dtype=torch.float32, device=p0.device)
        lin[:, 0:3] = p0.detach()
        lin[:, 3:6] = p1.detach()
        feats = N.nif_encode_segments(handle.h, lin, net.in_dim)
        acts = torch.empty((net.mlp_depth, n, net.mlp_width), dtype=torch.float32, device=p0.device)
        out = N.nif_mlp_forward(handle.h, feats, acts=acts)
        ctx.save_for_backward(lin, feats, acts)
        ctx.handle = handle
        return out

    @staticmethod
    def backward(ctx, dout):
        lin, feats, acts = ctx.saved_tensors
        h = ctx.handle
        half = feats.shape[1] // 2
        dx = N.nif_mlp_backward(h.h, feats, acts, dout.contiguous())
        pts = torch.cat([lin[:, 0:3], lin[:, 3:6]], 0).contiguous()
        dfe = torch.cat([dx[:, :half], dx[:, half:]], 0).contiguous()
        dpts = N.nif_encode_points_backward(h.h, pts, dfe, None, want_dpts=True)
        n = lin.shape[0]
        return dpts[:n], dpts[n:], None


def nif_segments_forward(p0, p1, handle):
    """Differentiable network outputs [n, 16] of the segments (p0, p1)."""
    return NIFSegments.apply(p0, p1, handle)
