"""Circuit post-processing on the device (pic_diag PIC_DIAG_CIRCUIT, Sec. 3 Eqs. 11-14)
against the oracle's, through the C ABI.

The paper's vacuum case: circuit II with its matching network loaded by the vacuum
C_eq = 892.07 pF, 77 V source, started from the network's periodic steady state.  Both
sides step the same empty discharge; every window's Z_ccp, Z_load, Gamma, element
powers, forward and reflected power and U_E harmonic agree to 1e-9 (both integrate the
same linear ODE in FP64: a composed propagator on the device, substep eliminations in
the oracle).  With plasma the same quantities are compared window by window in the
GEC parity tests."""
import dataclasses

import numpy as np
import pytest

from gpu_common import pic
from oracle import orc
from paper_2310_04957_gb300 import workloads as W
from test_oracle_pins import _paper_vacuum_circuit, _phasor_circuit_ii
from util import with_particles

pytestmark = pytest.mark.gpu


def close(a, b, tol):
    """Each quantity within tol of its own size, or of the size of what it is a small part
    of: Gamma of 1, the reflected and plasma powers of the source power, the DC means of the
    fundamental's amplitude."""
    for k, v in b.items():
        scale = max(abs(v), 1e-30)
        if k in ("gamma", "gamma_abs"):
            scale = max(scale, 1.0)
        elif k in ("p_ref", "p_ccp"):
            scale = max(scale, abs(b["p_source"]))
        elif k == "u_dc":
            scale = max(scale, abs(b["u1"]))
        elif k == "i_dc":
            scale = max(scale, abs(b["u1"] / b["z_ccp"]))
        assert abs(a[k] - v) <= tol * scale, (k, a[k], v)


def test_vacuum_match_postprocessing_matches_oracle():
    g = _paper_vacuum_circuit()
    ref = _phasor_circuit_ii(g, g["C_eq"])
    base = W.small_cylinder(n_per_species=16)
    circ = (g["R_s"], g["C_m1"], g["L_m"], g["C_m2"], g["R_m"], g["C_stray"], g["R_stray"], g["L_stray"])
    wl = dataclasses.replace(with_particles(base), circuit=W.CIRCUIT_IMN, circ=circ, V_src=g["V_source"],
                             f_src=g["f"], phase_src=0.0, steps_per_rf=200, dt=1 / g["f"] / 200, ceq_refresh=0)
    P = pic()
    d = P.Discharge(wl, precision=P.PIC_FP64)
    o = orc.Oracle(wl)
    for x in (d, o):
        x.set_ceq(g["C_eq"])
        x.set_circuit_state(ref["y0"])
        x.set_step(0)
    d.start()
    o.init_fields()
    for x in (d, o):  # start from the steady state (the start-up may not touch the circuit)
        x.set_ceq(g["C_eq"])
        x.set_circuit_state(ref["y0"])
    for w in range(3):
        d.step(wl.steps_per_rf)
        o.step(wl.steps_per_rf)
        a, b = d.circuit_diag(), o.circuit_diag()
        close(a, b, 1e-9)
    assert abs(a["z_ccp"].imag + 13.157) < 1e-3
    assert a["gamma_abs"] < 1e-3
    assert abs(abs(a["u1"]) - 100.0) < 0.5
    assert d.status() == 0
