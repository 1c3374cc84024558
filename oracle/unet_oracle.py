"""FP64 CPU oracle of the learned preconditioner's U-Net (test infrastructure only).

Plain PyTorch CPU operations in float64.  The network is the one the CUDA
library trains: 14 3x3 convolutions (bias + ReLU) in four levels with 2x2
average pooling, nearest 2x upsampling and channel concatenation, and a final
1x1 convolution.  With `bf16=True` every tensor the GPU stores in BF16
(weights, activations, pre-activation gradients) is rounded to BF16 at the
same place, so the GPU and the oracle differ only by accumulation order.
Gradients come from torch.autograd on the float64 graph; the pre-activation
gradient rounding is inserted with a custom autograd function.

Parameter order (matches pic_unet_set_params): for each conv W[cout][9][cin]
(tap = 3*(dy+1) + (dx+1)) then bias[cout]; then the 1x1 weights [32] and bias.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CIN = [16, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32]
COUT = [32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32]


def param_count():
    return sum(9 * ci * co + co for ci, co in zip(CIN, COUT)) + 33


def _bf16(x):
    return x.to(torch.bfloat16).to(torch.float64)


class _RoundGrad(torch.autograd.Function):
    """Identity forward; rounds the incoming gradient to BF16 (the GPU's dPre)."""

    @staticmethod
    def forward(ctx, x):
        return x.view_as(x)

    @staticmethod
    def backward(ctx, g):
        return _bf16(g)


class _Conv32(torch.autograd.Function):
    """3x3 convolution whose sums (forward and both gradients) run in float32."""

    @staticmethod
    def forward(ctx, x, w):
        ctx.save_for_backward(x, w)
        return F.conv2d(x.float(), w.float(), padding=1).double()

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        gx = torch.nn.grad.conv2d_input(x.shape, w.float(), g.float(), padding=1).double()
        gw = torch.nn.grad.conv2d_weight(x.float(), w.shape, g.float(), padding=1).double()
        return gx, gw


def unpack(params):
    """Flat parameter vector -> list of (torch weight [co][ci][3][3], bias) and the 1x1."""
    p = torch.as_tensor(np.asarray(params, dtype=np.float64))
    out, o = [], 0
    for ci, co in zip(CIN, COUT):
        n = 9 * ci * co
        w = p[o:o + n].reshape(co, 3, 3, ci).permute(0, 3, 1, 2).contiguous()
        o += n
        b = p[o:o + co]
        o += co
        out.append((w, b))
    w1, b1 = p[o:o + 32], p[o + 32:o + 33]
    return out, (w1, b1)


def forward(params, inp, bf16=True, requires_grad=False):
    """inp: array [3, H, W] (rho~, chi, mask).  Returns (out [H, W] tensor, flat param tensor list)."""
    convs, (w1, b1) = unpack(params)
    leaves = []
    for w, b in convs:
        w.requires_grad_(requires_grad)
        b.requires_grad_(requires_grad)
        leaves += [w, b]
    w1.requires_grad_(requires_grad)
    b1.requires_grad_(requires_grad)
    rnd = _bf16 if bf16 else (lambda t: t)
    x = torch.zeros(1, 16, inp.shape[1], inp.shape[2], dtype=torch.float64)
    x[0, :3] = torch.as_tensor(np.asarray(inp, dtype=np.float64))
    x = rnd(x)

    def conv(t, l):
        w, b = convs[l]
        y = F.conv2d(t, rnd(w), b, padding=1)
        if bf16:
            y = _RoundGrad.apply(y)
        return rnd(F.relu(y))

    pool = lambda t: rnd(F.avg_pool2d(t, 2))
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    e0 = conv(conv(x, 0), 1)
    e1 = conv(conv(pool(e0), 2), 3)
    e2 = conv(conv(pool(e1), 4), 5)
    b = conv(conv(pool(e2), 6), 7)
    d2 = conv(conv(torch.cat([up(b), e2], 1), 8), 9)
    d1 = conv(conv(torch.cat([up(d2), e1], 1), 10), 11)
    d0 = conv(conv(torch.cat([up(d1), e0], 1), 12), 13)
    out = (d0[0] * w1[:, None, None]).sum(0) + b1[0]
    return out, leaves + [torch.cat([w1, b1])]


def flat_grads(leaves):
    """Gradients of the leaves in parameter order (conv W back to [co][9][ci])."""
    parts = []
    for k in range(len(CIN)):
        w, b = leaves[2 * k], leaves[2 * k + 1]
        parts.append(w.grad.permute(0, 2, 3, 1).reshape(-1))
        parts.append(b.grad)
    w1b1 = leaves[-1]
    return parts, w1b1


def forward_backward(params, inp, gout, bf16=True, acc32=False):
    """Output and the flat parameter gradient of sum(out * gout).

    acc32=True evaluates every convolution sum in float32 (inputs already rounded
    to BF16), the accumulation precision of the GPU's tensor cores; comparing it
    with the float64 sums measures how much accumulation-order effects are
    amplified by the BF16 rounding of activations."""
    convs, (w1, b1) = unpack(params)
    ws = []
    for w, b in convs:
        w.requires_grad_(True)
        b.requires_grad_(True)
        ws += [w, b]
    w1.requires_grad_(True)
    b1.requires_grad_(True)
    rnd = _bf16 if bf16 else (lambda t: t)
    x = torch.zeros(1, 16, inp.shape[1], inp.shape[2], dtype=torch.float64)
    x[0, :3] = torch.as_tensor(np.asarray(inp, dtype=np.float64))
    x = rnd(x)

    def conv(t, l):
        w, b = convs[l]
        if acc32:
            y = _Conv32.apply(t, rnd(w)) + b[None, :, None, None]
        else:
            y = F.conv2d(t, rnd(w), b, padding=1)
        if bf16:
            y = _RoundGrad.apply(y)
        return rnd(F.relu(y))

    pool = lambda t: rnd(F.avg_pool2d(t, 2))
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    e0 = conv(conv(x, 0), 1)
    e1 = conv(conv(pool(e0), 2), 3)
    e2 = conv(conv(pool(e1), 4), 5)
    bb = conv(conv(pool(e2), 6), 7)
    d2 = conv(conv(torch.cat([up(bb), e2], 1), 8), 9)
    d1 = conv(conv(torch.cat([up(d2), e1], 1), 10), 11)
    d0 = conv(conv(torch.cat([up(d1), e0], 1), 12), 13)
    out = (d0[0] * w1[:, None, None]).sum(0) + b1[0]
    (out * torch.as_tensor(np.asarray(gout, dtype=np.float64))).sum().backward()
    g = []
    for (w, b) in convs:
        g.append(w.grad.permute(0, 2, 3, 1).reshape(-1))
        g.append(b.grad)
    g.append(w1.grad)
    g.append(b1.grad)
    return out.detach().numpy(), torch.cat(g).numpy()


def init_params(seed):
    """He-initialised parameters (the input convolution sees 3 live channels)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(CIN, COUT):
        fan = 9 * (3 if ci == 16 else ci)
        parts.append(rng.normal(0, np.sqrt(2.0 / fan), 9 * ci * co))
        parts.append(np.zeros(co))
    parts.append(rng.normal(0, np.sqrt(1.0 / 32), 32))
    parts.append(np.zeros(1))
    return np.concatenate(parts)
