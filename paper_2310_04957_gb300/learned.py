"""Training of the learned field-solve preconditioner on pairs the simulation
itself generates, and its use in the field solve (the U-Net of the library,
trained by the library's own forward/backward/Adam kernels).

Pairs (arXiv:2310.04957, Eq. 1 on the node grid): after a solve with warm
start phi_w and solution phi, r0 = b - A phi_w and delta = phi - phi_w =
A^-1 r0.  The network sees (D^-1 r0 / s, chi, Dirichlet mask) and is trained
to output delta / s (relative L2 loss over free nodes), s = rms of D^-1 r0.
Used as z = s U(D^-1 r / s, ...) it is both the learned initial-guess
correction (first application, on the warm start's residual) and the
preconditioner of the flexible CG (later applications, on its residuals);
pairs from those later residuals are added by keeping learned iterates
(pic_learned_snapshot) once a first network exists.

Device buffers here are torch tensors used as memory only; every arithmetic
step runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import pic


# Layer widths of the library's U-Net (the parameter layout of pic_unet_set_params).
CONV_IN = (16, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32)
CONV_OUT = (32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32)


def init_params(seed):
    """He-normal weights (fan-in 9 x live input channels; the first layer has 3
    live channels of 16), zero biases, 1x1 output weights N(0, 1/32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(CONV_IN, CONV_OUT):
        fan = 9 * (3 if ci == 16 else ci)
        parts.append(rng.normal(0.0, math.sqrt(2.0 / fan), 9 * ci * co))
        parts.append(np.zeros(co))
    parts.append(rng.normal(0.0, math.sqrt(1.0 / 32), 32))
    parts.append(np.zeros(1))
    return np.concatenate(parts).astype(np.float32)


class PairStore:
    """Device-resident training pairs: inputs [n][3][H*W] and targets [n][H*W] (FP32)."""

    def __init__(self, capacity, H, W, device="cuda"):
        import torch

        self.inp = torch.zeros(capacity, 3, H * W, dtype=torch.float32, device=device)
        self.tgt = torch.zeros(capacity, H * W, dtype=torch.float32, device=device)
        self.run = np.full(capacity, -1, np.int32)
        self.n = 0
        self.H, self.W = H, W

    def add_from(self, d, run_id, source=0):
        if self.n >= self.inp.shape[0]:
            return False
        k = self.n
        d.learned_pair(self.inp[k].data_ptr(), self.tgt[k].data_ptr(), source=source)
        self.run[k] = run_id
        self.n += 1
        return True


def collect_warm_pairs(d, store, steps, run_id):
    """Advance discharge d by `steps` steps, keeping the warm-start pair of each solve."""
    d.keep_warm(True)
    for _ in range(steps):
        d.step(1)
        if not store.add_from(d, run_id, source=0):
            break


def collect_iterate_pairs(d, store, steps, run_id, ks=(1, 2, 3), seed=0):
    """Advance d with the learned solver, keeping the pair of the iterate after k
    network applications (k drawn from ks each step) when the solve made k."""
    rng = np.random.default_rng(seed)
    for _ in range(steps):
        k = int(rng.choice(ks))
        d.learned_snapshot(k)
        d.step(1)
        if d.learned_stats()[0] >= k:
            if not store.add_from(d, run_id, source=1):
                break
    d.learned_snapshot(0)


def train(net, store, idx, steps, lr=1e-3, lr_end=1e-5, batch=4, seed=0, log_every=0):
    """Adam on the relative L2 loss over pairs idx; cosine learning-rate decay.
    Returns the mean training loss over each logging window."""
    import torch

    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=store.inp.device)
    hist = []
    window = 0
    for t in range(1, steps + 1):
        net.zero_grads()
        for i in rng.choice(idx, size=batch, replace=len(idx) < batch):
            net.forward(store.inp[i].data_ptr(), 0)
            net.loss_backward(store.inp[i].data_ptr(), store.tgt[i].data_ptr(), loss.data_ptr())
        a = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * (t - 1) / max(1, steps - 1)))
        net.adam(a / batch, t)
        window += 1
        if log_every and (t % log_every == 0 or t == steps):
            hist.append(float(loss.item()) / (window * batch))
            loss.zero_()
            window = 0
    return hist


def evaluate(net, store, idx):
    """Mean relative L2 error of the network on pairs idx."""
    import torch

    loss = torch.zeros(1, dtype=torch.float32, device=store.inp.device)
    for i in idx:
        net.forward(store.inp[i].data_ptr(), 0)
        net.zero_grads()
        net.loss_backward(store.inp[i].data_ptr(), store.tgt[i].data_ptr(), loss.data_ptr())
    net.zero_grads()
    return float(loss.item()) / max(1, len(idx))


def compare_solvers(d, modes=(pic.PIC_SOLVER_PLAIN, pic.PIC_SOLVER_MIXED, pic.PIC_SOLVER_MG, pic.PIC_SOLVER_LEARNED),
                    repeats=1):
    """Solve the last step's system again from its warm start (kept by
    pic_keep_warm or the learned solver) with each mode.  Returns {mode: (status,
    iterations, relative residual, ms, learned stats)}; the handle ends with the
    last mode's solution."""
    import torch

    phi0 = d.field("phi_warm").copy()
    out = {}
    for m in modes:
        best = None
        for _ in range(repeats):
            d.set_field("phi", phi0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            st, it, rr = d.field_solve(m)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ls = d.learned_stats() if m == pic.PIC_SOLVER_LEARNED else None
            if best is None or ms < best[3]:
                best = (st, it, rr, ms, ls)
        out[m] = best
    return out


def train_on_discharge(wl, warm_pairs=300, iterate_pairs=200, steps=1500, seed=0, settle=10, net=None):
    """Train a network for workload wl from scratch on pairs its own run
    generates: warm-start pairs from mixed-solver steps, a first training pass,
    then pairs from iterates of learned solves with that network, and a second
    pass on both.  Returns (net, discharge, info); the discharge has the network
    attached."""
    import time

    t0 = time.perf_counter()
    d = pic.Discharge(wl, solver=pic.PIC_SOLVER_MIXED)
    d.step(settle)
    store = PairStore(warm_pairs + iterate_pairs, wl.nz, wl.nr)
    collect_warm_pairs(d, store, warm_pairs, 0)
    if net is None:
        net = pic.UNet(wl.nz, wl.nr)
        net.set_params(init_params(seed))
    h1 = train(net, store, np.arange(store.n), steps, lr=1e-3, batch=4, seed=seed, log_every=steps)
    n0 = store.n
    d.set_solver(pic.PIC_SOLVER_LEARNED)
    d.attach_unet(net, maxit=60)
    collect_iterate_pairs(d, store, iterate_pairs, 1, seed=seed)
    h2 = train(net, store, np.arange(store.n), steps, lr=5e-4, batch=4, seed=seed + 1, log_every=steps)
    d.set_solver(pic.PIC_SOLVER_MIXED)
    info = {"warm_pairs": n0, "iterate_pairs": store.n - n0, "adam_steps": 2 * steps, "batch": 4,
            "loss_pass1": h1[-1], "loss_pass2": h2[-1], "seconds": time.perf_counter() - t0}
    del store
    return net, d, info
