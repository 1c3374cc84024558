"""The U-Net's tensor-core forward and backward kernels against the FP64 CPU
oracle of the same network (BF16 rounding at the same places), through the C ABI."""
import numpy as np
import pytest

from gpu_common import pic
from oracle import unet_oracle as U
from util import rel_l2

pytestmark = pytest.mark.gpu


def _bf16_round(p):
    import torch

    return torch.as_tensor(p, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("Cin,Cout,H,W", [(16, 32, 40, 72), (96, 32, 16, 40), (384, 128, 8, 24), (256, 256, 12, 20),
                                          (64, 192, 24, 16)])
def test_conv_ops_match_float64(Cin, Cout, H, W):
    """Forward, input-gradient-style (flipped-weight forward) and weight-gradient
    convolutions of the tensor-core kernels against float64 sums of the same BF16
    operands: FP32 accumulation only (relative 1e-5), including ragged pixel tiles."""
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F

    P = pic()
    g = torch.Generator().manual_seed(Cin * 7 + Cout)
    x = torch.randn(H * W, Cin, generator=g).to(torch.bfloat16)
    w = (torch.randn(Cout, 9, Cin, generator=g) / (3 * Cin ** 0.5)).to(torch.bfloat16)
    dy = torch.randn(H * W, Cout, generator=g).to(torch.bfloat16)
    bias = torch.randn(Cout, generator=g).float()
    xd, wd, dyd, bd = x.cuda(), w.cuda(), dy.cuda(), bias.cuda()
    ref = F.conv2d(x.double().T.reshape(1, Cin, H, W), w.double().reshape(Cout, 3, 3, Cin).permute(0, 3, 1, 2),
                   padding=1)[0].reshape(Cout, -1).T
    out = torch.zeros(H * W, Cout, device="cuda")
    assert P.conv3x3_op(0, H, W, xd.data_ptr(), Cin, wd.data_ptr(), 0, out.data_ptr(), Cout) == 0
    assert rel_l2(out.cpu().double().numpy(), ref.numpy()) <= 1e-5
    outb = torch.zeros(H * W, Cout, dtype=torch.bfloat16, device="cuda")
    assert P.conv3x3_op(1, H, W, xd.data_ptr(), Cin, wd.data_ptr(), bd.data_ptr(), outb.data_ptr(), Cout) == 0
    refb = torch.relu(ref + bias.double()).to(torch.bfloat16).double()
    diff = (outb.cpu().double() - refb).abs()
    # at most one BF16 rounding step apart, or within the FP32 accumulation error near the ReLU kink
    pre = (ref + bias.double()).abs().max().item()
    assert (diff <= 2.0 ** -7 * refb.abs() + 1e-5 * pre).all()
    dw = torch.zeros(9 * Cin, Cout, device="cuda")
    assert P.conv3x3_op(2, H, W, xd.data_ptr(), Cin, dyd.data_ptr(), 0, dw.data_ptr(), Cout) == 0
    refw = torch.nn.grad.conv2d_weight(x.double().T.reshape(1, Cin, H, W), (Cout, Cin, 3, 3),
                                       dy.double().T.reshape(1, Cout, H, W), padding=1)
    refw = refw.permute(2, 3, 1, 0).reshape(9 * Cin, Cout)  # [(tap, cin)][cout]
    assert rel_l2(dw.cpu().double().numpy(), refw.numpy()) <= 1e-5


@pytest.mark.parametrize("H,W", [(64, 128), (32, 256)])
def test_unet_forward_and_gradients_match_oracle(H, W):
    torch = pytest.importorskip("torch")
    P = pic()
    rng = np.random.default_rng(H + W)
    params = U.init_params(7).astype(np.float32).astype(np.float64)
    # nonzero biases so every bias path is exercised
    offs = np.cumsum([0] + [9 * ci * co + co for ci, co in zip(U.CIN, U.COUT)])
    for k in range(14):
        params[offs[k] + 9 * U.CIN[k] * U.COUT[k]: offs[k + 1]] = rng.uniform(0.2, 0.6, U.COUT[k])
    params = params.astype(np.float32).astype(np.float64)
    inp = rng.normal(size=(3, H, W)).astype(np.float32).astype(np.float64)
    gout = rng.normal(size=(H, W)).astype(np.float32).astype(np.float64)
    net = P.UNet(H, W)
    net.set_params(params)
    d_in = torch.as_tensor(inp.reshape(3, -1), dtype=torch.float32, device="cuda").contiguous()
    d_out = torch.zeros(H * W, dtype=torch.float32, device="cuda")
    d_g = torch.as_tensor(gout.ravel(), dtype=torch.float32, device="cuda").contiguous()
    net.zero_grads()
    net.forward(d_in.data_ptr(), d_out.data_ptr())
    net.backward(d_g.data_ptr())
    assert net.status() == 0
    out_gpu = d_out.cpu().numpy().astype(np.float64).reshape(H, W)
    g_gpu = net.get_grads().astype(np.float64)
    # the master weights the GPU rounds to BF16 are the same float32 values
    out_ref, g_ref = U.forward_backward(params, inp, gout, bf16=True)
    # tolerance from the arithmetic: the same network with float32 sums (the tensor
    # cores' accumulation precision) against float64 sums; BF16 re-rounding of
    # activations amplifies the accumulation-order difference layer by layer
    out_32, g_32 = U.forward_backward(params, inp, gout, bf16=True, acc32=True)
    spread = rel_l2(out_32, out_ref)
    assert rel_l2(out_gpu, out_ref) <= max(3 * spread, 1e-3), (rel_l2(out_gpu, out_ref), spread)
    for k in range(14):
        for a, b, what in ((offs[k], offs[k] + 9 * U.CIN[k] * U.COUT[k], "W"),
                           (offs[k] + 9 * U.CIN[k] * U.COUT[k], offs[k + 1], "b")):
            sp = rel_l2(g_32[a:b], g_ref[a:b])
            err = rel_l2(g_gpu[a:b], g_ref[a:b])
            assert err <= max(3 * sp, 5e-3), (what, k, err, sp)
    sp = rel_l2(g_32[offs[14]:], g_ref[offs[14]:])
    assert rel_l2(g_gpu[offs[14]:], g_ref[offs[14]:]) <= max(3 * sp, 1e-3)
    # parameters round-trip
    np.testing.assert_array_equal(net.get_params(), params.astype(np.float32))


@pytest.mark.parametrize("Cin,Cout,H,W,tile_n,tile_mma", [
    (32, 64, 44, 256, 32, 8),    # one-row accumulators (128-pixel rows), ragged last row block
    (64, 64, 40, 128, 64, 4),
    (384, 128, 6, 128, 128, 2),  # 24 channel steps through a ring of fewer stages
    (256, 256, 30, 64, 256, 1),  # two image rows per accumulator
    (128, 256, 30, 64, 64, 2),   # four rows per CTA, ragged
    (64, 96, 20, 32, 32, 2),     # four rows per accumulator
    (16, 32, 40, 72, 32, 1),     # eight-pixel-wide strips
    (96, 32, 16, 40, -1, 0),     # the gather kernel
])
def test_conv_tilings_match_float64(Cin, Cout, H, W, tile_n, tile_mma):
    """Every tiling of the TMA-fed convolution (halo boxes for 128-pixel rows,
    shifted column copies for narrower strips, channel splits, several
    accumulators per CTA) gives the float64 sums of the same BF16 operands to
    FP32 accumulation accuracy."""
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F

    P = pic()
    g = torch.Generator().manual_seed(Cin * 13 + Cout + H)
    x = torch.randn(H * W, Cin, generator=g).to(torch.bfloat16)
    w = (torch.randn(Cout, 9, Cin, generator=g) / (3 * Cin ** 0.5)).to(torch.bfloat16)
    bias = torch.randn(Cout, generator=g).float()
    xd, wd, bd = x.cuda(), w.cuda(), bias.cuda()
    ref = F.conv2d(x.double().T.reshape(1, Cin, H, W), w.double().reshape(Cout, 3, 3, Cin).permute(0, 3, 1, 2),
                   padding=1)[0].reshape(Cout, -1).T
    out = torch.full((H * W, Cout), float("nan"), device="cuda")
    assert P.conv3x3_op(0, H, W, xd.data_ptr(), Cin, wd.data_ptr(), 0, out.data_ptr(), Cout,
                        tile_n=tile_n, tile_mma=tile_mma) == 0
    o = out.cpu().double().numpy()
    assert np.isfinite(o).all()
    assert rel_l2(o, ref.numpy()) <= 1e-5
    assert np.abs(o - ref.numpy()).max() <= 1e-5 * np.abs(ref.numpy()).max()
    outb = torch.zeros(H * W, Cout, dtype=torch.bfloat16, device="cuda")
    assert P.conv3x3_op(1, H, W, xd.data_ptr(), Cin, wd.data_ptr(), bd.data_ptr(), outb.data_ptr(), Cout,
                        tile_n=tile_n, tile_mma=tile_mma) == 0
    refb = torch.relu(ref + bias.double()).to(torch.bfloat16).double()
    pre = (ref + bias.double()).abs().max().item()
    assert ((outb.cpu().double() - refb).abs() <= 2.0 ** -7 * refb.abs() + 1e-5 * pre).all()


def test_conv_forced_tiling_that_does_not_fit_is_rejected():
    torch = pytest.importorskip("torch")
    P = pic()
    x = torch.zeros(16 * 20, 32, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(64, 9, 32, dtype=torch.bfloat16, device="cuda")
    out = torch.zeros(16 * 20, 64, device="cuda")
    # W = 20 has no 8-pixel strip; 48 output channels are not a multiple of 32
    assert P.conv3x3_op(0, 16, 20, x.data_ptr(), 32, w.data_ptr(), 0, out.data_ptr(), 64, tile_n=64) != 0
    assert P.conv3x3_op(0, 16, 24, x.data_ptr(), 32, w.data_ptr(), 0, out.data_ptr(), 48, tile_n=32) != 0
