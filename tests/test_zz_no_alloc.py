"""The allocation-free field solve, pic_pcg_solve_static.

Callers that cannot allocate GPU memory at solve time (a host application that
owns all device memory through its own pool, a real-time loop that must not
wait on the allocator) use this entry point on arrays they own.  This file
checks, through the C ABI, that it returns the same potential as the
handle-based pic_field_solve, within the tolerance the other field-solve tests
use, on two calls in a row (the second call runs on the work array the first
one left behind), and that a call that only enqueues the solve reports its
outcome through pic_pcg_static_result.  It sits last in the collection order
so that a failure here stops a -x run only after every other test has run.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import make_pair, pic, random_field, small
from util import rel_l2

pytestmark = pytest.mark.gpu


def _device(a, torch, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_static_solve_matches_field_solve_twice():
    torch = pytest.importorskip("torch")
    P = pic()
    wl = dataclasses.replace(small(20_000), phase_src=0.9)
    d, o = make_pair(wl, 0)
    o.init_fields()
    d.start()
    for call in range(2):
        # a different charge distribution for each call
        er, ez = random_field(wl, 31 + call, precision=0)
        d.set_field("Er", er)
        d.set_field("Ez", ez)
        d.set_step(call)
        d.particle_phase()
        phi0 = d.field("phi")  # warm start both solves from the same potential
        st, it_ref, rel_ref = d.field_solve(P.PIC_SOLVER_PLAIN)
        assert st == 0
        phi_ref = d.field("phi")
        # the same system on caller-owned device arrays: operator and charge of the
        # same deposits, built by the oracle (equal to the handle's to rounding)
        for name in ("dep_e", "dep_i"):
            o.set_field(name, d.field(name))
        o.set_field("phi", phi0)
        o.assemble()
        Gr, Gz = o.operator()
        kind = _device(wl.node_kind, torch, torch.int8)
        g_r = _device(Gr, torch, torch.float64)
        g_z = _device(Gz, torch, torch.float64)
        q = _device(o.field("rho"), torch, torch.float64)
        phi = _device(o.field("phi"), torch, torch.float64)
        torch.cuda.synchronize()
        st, it, rel = P.pcg_solve_static(wl.nr, wl.nz, kind.data_ptr(), g_r.data_ptr(), g_z.data_ptr(), q.data_ptr(),
                                         phi.data_ptr(), wl.pcg_tol, wl.pcg_maxit,
                                         stream=torch.cuda.current_stream().cuda_stream)
        assert st == 0, P.ERRORS.get(st, st)
        assert rel <= wl.pcg_tol
        assert abs(it - it_ref) <= max(3, 0.05 * it_ref)
        assert rel_l2(phi.cpu().numpy().reshape(phi_ref.shape), phi_ref) <= 1e-8
        # the same solve enqueued without waiting: the result slots report it
        phi2 = _device(o.field("phi"), torch, torch.float64)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream().cuda_stream
        st, _, _ = P.pcg_solve_static(wl.nr, wl.nz, kind.data_ptr(), g_r.data_ptr(), g_z.data_ptr(), q.data_ptr(),
                                      phi2.data_ptr(), wl.pcg_tol, wl.pcg_maxit, stream=stream, wait=False)
        assert st == 0
        st, it2, rel2 = P.pcg_static_result(stream=stream)
        assert st == 0 and it2 == it and rel2 == rel
        assert torch.equal(phi2, phi)


def test_static_solve_rejects_oversized_grids():
    pytest.importorskip("torch")
    P = pic()
    st, _, _ = P.pcg_solve_static(1024, 256, 1, 1, 1, 1, 1, 1e-10, 10)
    assert st == -1  # PIC_EINVAL: (1025 * 257) nodes exceed the fixed work area
