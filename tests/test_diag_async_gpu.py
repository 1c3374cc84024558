"""The enqueued scalar read (pic_diag_async) against the synchronising one
(pic_diag), through the C ABI.

- At the same point of the stream both give the same PIC_NSCALARS doubles, bit
  for bit (one device-side assembly serves both).
- Reads enqueued after every step while the host keeps enqueuing the next steps
  each land in their own buffer, page-locked or pageable, and hold that step's
  values: the log of a pipelined run equals the synchronous reads of the same
  run stepped again from the same start (the step is deterministic).
- Another selector, a short or NULL buffer are rejected with PIC_EINVAL.
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
