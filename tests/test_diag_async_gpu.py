"""The enqueued scalar read (pic_diag_async) and device-buffer reads
(PIC_DIAG_DEVICE) against the synchronising host read (pic_diag), through the C ABI.

- At the same point of the stream both give the same PIC_NSCALARS doubles, bit
  for bit (one device-side assembly serves both).
- Reads enqueued after every step while the host keeps enqueuing the next steps
  each land in their own buffer, page-locked or pageable, and hold that step's
  values: the log of a pipelined run equals the synchronous reads of the same
  run stepped again from the same start (the step is deterministic).
- Another selector, a short or NULL buffer are rejected with PIC_EINVAL.
- Into CUDA tensors, every node array and the scalars equal the host read bit
  for bit; host-only selectors and short buffers are rejected.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import pic, small

pytestmark = pytest.mark.gpu

N_STEPS = 12


def sync_reads(P, wl, precision, solver, n):
    d = P.Discharge(wl, precision=precision, solver=solver)
    d.start()
    rows = []
    for _ in range(n):
        d.step(1)
        sc = d.scalars()
        rows.append([sc[k] for k in P.SCALARS])
    d.close()
    return np.array(rows)


@pytest.mark.parametrize("precision,solver", [(0, 3), (1, 0)])
def test_async_read_equals_sync_read_at_the_same_point(precision, solver):
    import torch

    P = pic()
    wl = small(20_000)
    d = P.Discharge(wl, precision=precision, solver=solver)
    d.start()
    buf = torch.empty(P.NSCALARS, dtype=torch.float64, pin_memory=True).numpy()
    for _ in range(4):
        d.step(1)
        d.scalars_async(buf)
        sc = d.scalars()  # synchronises: the enqueued copy has run
        np.testing.assert_array_equal(buf, np.array([sc[k] for k in P.SCALARS]))
    d.close()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("precision,solver", [(0, 3), (1, 0)])
def test_pipelined_log_holds_every_steps_scalars(precision, solver, pinned):
    import torch

    P = pic()
    wl = small(20_000)
    ref = sync_reads(P, wl, precision, solver, N_STEPS)
    d = P.Discharge(wl, precision=precision, solver=solver)
    d.start()
    if pinned:
        log = torch.empty((N_STEPS, P.NSCALARS), dtype=torch.float64, pin_memory=True).numpy()
    else:
        log = np.empty((N_STEPS, P.NSCALARS))
    log[:] = np.nan
    for k in range(N_STEPS):
        d.step(1)
        d.scalars_async(log[k])
    d.sync()
    np.testing.assert_array_equal(log[:, 0], np.arange(1, N_STEPS + 1))
    np.testing.assert_array_equal(log, ref)
    d.close()


def test_async_read_rejects_other_selectors_and_short_buffers():
    P = pic()
    d = P.Discharge(small(5_000))
    d.start()
    L = P.lib()
    buf = np.zeros(P.NSCALARS)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    assert L.pic_diag_async(d.h, P.DIAG_CIRCUIT, p, buf.nbytes) == P.PIC_EINVAL
    assert L.pic_diag_async(d.h, P.DIAG_SCALARS, p, buf.nbytes - 8) == P.PIC_EINVAL
    assert L.pic_diag_async(d.h, P.DIAG_SCALARS, None, buf.nbytes) == P.PIC_EINVAL
    with pytest.raises(ValueError):
        d.scalars_async(np.zeros(P.NSCALARS, np.float32))
    assert L.pic_diag_async(d.h, P.DIAG_SCALARS, p, buf.nbytes) == P.PIC_OK
    assert L.pic_sync(d.h) == P.PIC_OK
    assert buf[0] == 0.0  # step 0 after start
    d.close()


NODE_FIELDS = ("phi", "Er", "Ez", "chi", "dep_e", "dep_i", "sigma", "vnode", "rho", "ne_avg", "ni_avg",
               "phi_warm")


@pytest.mark.parametrize("precision,solver", [(0, 3), (1, 0)])
def test_device_buffers_receive_the_host_values(precision, solver):
    """pic_diag with PIC_DIAG_DEVICE into CUDA tensors: every node array and the
    scalars equal the host form bit for bit (one device-side conversion serves
    both), after steps that end an RF window (so the window averages are set)."""
    import dataclasses

    import torch

    P = pic()
    wl = dataclasses.replace(small(20_000), steps_per_rf=3)
    d = P.Discharge(wl, precision=precision, solver=solver)
    d.start()
    d.step(4)
    n = d.n_nodes
    for name in NODE_FIELDS:
        t = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        d.field_to(name, t)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), d.field(name).ravel(), err_msg=name)
    t = torch.full((P.NSCALARS,), float("nan"), dtype=torch.float64, device="cuda")
    d.scalars_to(t)
    torch.cuda.synchronize()
    sc = d.scalars()
    np.testing.assert_array_equal(t.cpu().numpy(), np.array([sc[k] for k in P.SCALARS]))
    d.close()


def test_device_buffers_reject_host_only_selectors_and_short_buffers():
    import torch

    P = pic()
    d = P.Discharge(small(5_000))
    d.start()
    L = P.lib()
    t = torch.zeros(d.n_nodes, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(t.data_ptr())
    for sel in (P.DIAG_CIRCUIT, P.DIAG_SOLVER, P.DIAG_STORE, P.DIAG["phiP"]):  # phiP: not a Vahedi handle
        assert L.pic_diag(d.h, sel | P.DIAG_DEVICE, ptr, t.numel() * 8) == P.PIC_EINVAL, sel
    assert L.pic_diag(d.h, P.DIAG["phi"] | P.DIAG_DEVICE, ptr, t.numel() * 8 - 8) == P.PIC_EINVAL
    with pytest.raises(ValueError):
        d.field_to("phi", torch.zeros(d.n_nodes, dtype=torch.float32, device="cuda"))
    d.close()
