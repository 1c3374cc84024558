"""Pins of the U-Net oracle (CPU, float64): the convolution convention and the
parameter layout against a hand-written sum, and autograd gradients against
central finite differences of the same float64 function."""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U


def test_param_count():
    assert U.param_count() == 1950625  # sum over layers of 9*cin*cout + cout, plus 33


def test_first_conv_matches_direct_sum():
    """out[y][x] of the first conv = sum over taps (dy,dx) and input channels of
    W[co][3(dy+1)+(dx+1)][ci] in[ci][y+dy][x+dx] + b (zero padding), before ReLU."""
    rng = np.random.default_rng(0)
    p = U.init_params(1)
    convs, _ = U.unpack(p)
    w, b = convs[0]
    x = torch.zeros(1, 16, 8, 16, dtype=torch.float64)
    x[0, :3] = torch.as_tensor(rng.normal(size=(3, 8, 16)))
    y = torch.nn.functional.conv2d(x, w, b, padding=1)[0]
    Wf = p[:9 * 16 * 32].reshape(32, 9, 16)
    for co, yy, xx in ((0, 0, 0), (5, 3, 7), (31, 7, 15), (17, 4, 0)):
        s = 0.0
        for t in range(9):
            dy, dx = t // 3 - 1, t % 3 - 1
            if 0 <= yy + dy < 8 and 0 <= xx + dx < 16:
                s += float((Wf[co, t] * x[0, :, yy + dy, xx + dx].numpy()).sum())
        assert y[co, yy, xx].item() == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_gradients_match_finite_differences():
    """float64 network (no BF16 rounding): d/dtheta of sum(out * g) by autograd equals
    central differences for parameters sampled from every layer."""
    rng = np.random.default_rng(2)
    p = U.init_params(3)
    inp = rng.normal(size=(3, 16, 16))
    g = rng.normal(size=(16, 16))
    _, grad = U.forward_backward(p, inp, g, bf16=False)

    def f(q):
        out, _ = U.forward(q, inp, bf16=False)
        return float((out.detach().numpy() * g).sum())

    offs = np.cumsum([0] + [9 * ci * co + co for ci, co in zip(U.CIN, U.COUT)])
    idx = [int(offs[k] + rng.integers(0, 9 * U.CIN[k] * U.COUT[k])) for k in range(14)]
    idx += [int(offs[k] + 9 * U.CIN[k] * U.COUT[k]) for k in (0, 7, 13)] + [len(p) - 1, len(p) - 5]
    h = 1e-6
    for i in idx:
        q1, q2 = p.copy(), p.copy()
        q1[i] += h
        q2[i] -= h
        fd = (f(q1) - f(q2)) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=2e-5, abs=1e-8), i
