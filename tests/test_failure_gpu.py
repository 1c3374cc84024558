"""Failure detection through the C ABI, with no GPU fault: every failure is
provoked through the configuration or the host, ends in a status code, and the
handle stays usable (or is destroyed cleanly) afterwards.

- an iteration cap of 1 -> PIC_ENOCONV;
- a barrier spin limit of a few hundred clock cycles -> the bounded grid-barrier
  waits run out -> PIC_ETIMEOUT (nothing hangs: every wait is bounded and a
  block that gives up leaves the solve);
- a particle capacity below what one step needs -> particles dropped ->
  PIC_EOVERFLOW;
- a non-finite potential written through pic_set_field -> PIC_ENAN.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import pic, small
from paper_2310_04957_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SOLVERS = [0, 1, 3]  # plain FP64, mixed, multigrid-preconditioned


def started(wl, **kw):
    P = pic()
    d = P.Discharge(wl, **kw)
    d.start()
    return P, d


@pytest.mark.parametrize("solver", SOLVERS)
def test_iteration_cap_reports_noconv(solver):
    wl = dataclasses.replace(small(20_000), phase_src=1.0)
    P, capped = started(dataclasses.replace(wl, pcg_maxit=1), solver=solver)
    st, it, rel = capped.field_solve(solver)
    assert st == P.PIC_ENOCONV and it <= 2 and rel > wl.pcg_tol
    capped.step(1)
    assert capped.check() == P.PIC_ENOCONV
    assert capped.status() & P.PIC_FLAG_NOCONV
    assert capped.check() == 0  # pic_status cleared the bits
    capped.close()
    _, d = started(wl, solver=solver)  # the same discharge without the cap converges
    st, it, rel = d.field_solve(solver)
    assert st == 0 and rel <= wl.pcg_tol


@pytest.mark.parametrize("solver", SOLVERS)
def test_barrier_spin_limit_reports_timeout_and_recovers(solver):
    wl = dataclasses.replace(small(20_000), phase_src=1.0)
    P, d = started(wl, solver=solver)
    d.set_spin_limit(200)  # far below the time 150+ blocks take to meet at a barrier
    st, _, _ = d.field_solve(solver)
    assert st == P.PIC_ETIMEOUT
    assert d.check() == P.PIC_ETIMEOUT
    if solver == 3:  # a failed multigrid solve makes the next one rebuild its hierarchy
        assert d.solver_state()["mg_solves"] == 0
    d.step(1)  # the step graph is captured again with the short limit
    assert d.status() & P.PIC_FLAG_TIMEOUT
    d.set_spin_limit(0)  # back to the default: the handle solves again
    st, _, rel = d.field_solve(solver)
    assert st == 0 and rel <= wl.pcg_tol
    d.step(2)
    assert d.status() == 0


def test_capacity_below_one_step_reports_overflow():
    wl = small(20_000)
    P = pic()
    n = wl.particles[0].n
    # exactly the initial population: bins get no slack and the overflow region
    # has no room, so any particle that changes cell or is born is dropped
    d = P.Discharge(wl, capacity=(n, n))
    d.start()
    d.step(1)
    assert d.check() == P.PIC_EOVERFLOW
    assert d.status() & P.PIC_FLAG_OVERFLOW
    assert d.count(0) < n  # the dropped particles are gone, the rest is consistent
    d.close()


@pytest.mark.parametrize("solver", SOLVERS)
def test_nan_potential_reports_nan_and_recovers(solver):
    wl = dataclasses.replace(small(20_000), phase_src=1.0)
    P, d = started(wl, solver=solver)
    phi = d.field("phi")
    bad = phi.copy()
    free = np.argwhere(np.asarray(wl.node_kind).reshape(wl.nz + 1, wl.nr + 1) == W.NODE_FREE)
    j, i = free[len(free) // 2]
    bad[j, i] = np.nan
    d.set_field("phi", bad)
    st, _, _ = d.field_solve(solver)
    assert st == P.PIC_ENAN
    assert d.check() == P.PIC_ENAN
    assert d.status() & P.PIC_FLAG_NAN
    d.set_field("phi", phi)
    st, _, rel = d.field_solve(solver)
    assert st == 0 and rel <= wl.pcg_tol
