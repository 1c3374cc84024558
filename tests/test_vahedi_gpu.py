"""Multiple driven electrodes and Vahedi's decomposition of the potential
(Sec. 2, Eqs. 2-4) on the GPU, through the C ABI.

- A planar gap between the powered plate and a voltage-driven plate, in vacuum:
  the unit Laplace solutions are 1 - z/L and z/L and the potential at start is
  U_E (1 - z/L) + U_1 z/L, in both field modes, against the closed form.
- The GEC-like cell with its upper electrode voltage-driven (a second, 2 MHz
  source): full steps side by side with the FP64 oracle in the same mode, with
  every check of tests/test_gec_parity.py, across an RF-window end where the
  Laplace parts are re-solved with chi; the refreshed parts agree with the
  oracle's.
"""
import dataclasses
import math

import numpy as np
import pytest

from gpu_common import make_pair, pic
from parity_tools import StepParity, phi_err, rel_l2
from paper_2310_04957_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
MG, PLAIN = 3, 0
DRIVE = ((60.0, 2e6, 0.4),)


def planar(nr, nz, R, L, mode):
    node = np.zeros((nz + 1, nr + 1), np.int8)
    node[0, :] = W.NODE_POWERED
    node[nz, :] = W.NODE_DRIVEN
    cell = np.zeros((nz, nr), np.int8)
    eps = np.ones((nz, nr))
    wl = W.small_cylinder(n_per_species=16)
    empty = W.Particles(*(np.zeros(0) for _ in range(8)), np.zeros(0, np.uint64))
    return dataclasses.replace(wl, nr=nr, nz=nz, dr=R / nr, dz=L / nz, node_kind=node, cell_kind=cell, cell_eps=eps,
                               V_src=100.0, phase_src=1.1, particles=(empty, empty), capacity=(1024, 1024),
                               drive=((40.0, 2e6, 0.7),), field_mode=mode, ceq_refresh=0)


@pytest.mark.parametrize("mode", [W.FIELD_VAHEDI, W.FIELD_DIRECT], ids=["vahedi", "direct"])
@pytest.mark.parametrize("solver", [PLAIN, MG], ids=["plain", "mg"])
def test_planar_gap_with_a_driven_plate_is_the_closed_form(mode, solver):
    P = pic()
    nr, nz, L = 16, 40, 0.02
    wl = planar(nr, nz, 0.03, L, mode)
    d = P.Discharge(wl, precision=FP64, solver=solver)
    d.start()
    z = (np.arange(nz + 1) * L / nz)[:, None]
    UE, U1 = 100.0 * math.sin(1.1), 40.0 * math.sin(0.7)
    want = np.broadcast_to(UE * (1 - z / L) + U1 * z / L, (nz + 1, nr + 1))
    np.testing.assert_allclose(d.field("phi"), want, atol=1e-8 * 100.0)
    if mode == W.FIELD_VAHEDI:
        np.testing.assert_allclose(d.field("phiL0"), np.broadcast_to(1 - z / L, want.shape), atol=1e-10)
        np.testing.assert_allclose(d.field("phiL1"), np.broadcast_to(z / L, want.shape), atol=1e-10)
    else:
        with pytest.raises(P.PicError):
            d.field("phiP")
    assert d.status() == 0
    d.close()


def gec_driven_top(mode, n=200_000):
    """The parity cell (tests/test_gec_parity.py) with its upper electrode driven by a
    second source instead of grounded (a dual-frequency cell)."""
    wl = W.gec_case(128, 64, 30.0, 150.0, n_per_species=n, seed_index=21)
    wl = dataclasses.replace(wl, steps_per_rf=3, phase_src=0.9)
    node = wl.node_kind.copy()
    dr, dz = wl.dr, wl.dz
    ish, jt = int(round(0.055 / dr)), int(round(0.0404 / dz))
    block = node[jt:wl.nz, 0:ish + 1]
    node[jt:wl.nz, 0:ish + 1] = np.where(block == W.NODE_GROUNDED, W.NODE_DRIVEN, block)
    assert (node == W.NODE_DRIVEN).sum() > 100
    return dataclasses.replace(wl, node_kind=node, drive=DRIVE, field_mode=mode)


CASES = [
    pytest.param(FP32, MG, W.FIELD_VAHEDI, id="fp32-mg-vahedi"),
    pytest.param(FP64, MG, W.FIELD_VAHEDI, id="fp64-mg-vahedi"),
    pytest.param(FP32, MG, W.FIELD_DIRECT, id="fp32-mg-direct"),
]


@pytest.mark.parametrize("precision,solver,mode", CASES)
def test_gec_with_a_driven_upper_electrode_matches_oracle(precision, solver, mode):
    wl = gec_driven_top(mode)
    d, o = make_pair(wl, precision, solver=solver, tile=(4, 4))
    o.init_fields()
    d.start()
    assert phi_err(d.field("phi"), o.field("phi"), wl.V_src) <= 1e-8
    if mode == W.FIELD_VAHEDI:
        for k in (0, 1):
            assert rel_l2(d.field(f"phiL{k}"), o.field(f"phiL{k}")) <= 1e-9
    sp = StepParity(wl, d, o, precision == FP32)
    L1_start = d.field("phiL1") if mode == W.FIELD_VAHEDI else None
    for step in range(4):
        sp.step(lambda: d.step(1))
        if mode == W.FIELD_VAHEDI and step == 2:  # the window ended: parts re-solved with chi
            assert rel_l2(d.field("phiL1"), L1_start) > 1e-6
            for k in (0, 1):
                assert rel_l2(d.field(f"phiL{k}"), o.field(f"phiL{k}")) <= (1e-6 if precision == FP32 else 1e-9)
    assert d.status() == 0
    # the driven electrode takes particles: they count as grounded-type exits
    print(f"{mode=} {precision=} flips {sp.flips} of {sp.seen}, phi end to end {sp.phi_e2e}")


def test_vahedi_state_survives_save_and_load(tmp_path):
    """pic_save / pic_load carry phi_P and the Laplace parts: 5 steps + save + 5 steps equals
    load + 5 steps bit for bit across a window end (FP32, Vahedi composition)."""
    P = pic()
    wl = dataclasses.replace(gec_driven_top(W.FIELD_VAHEDI, n=50_000), steps_per_rf=4)
    d = P.Discharge(wl, precision=FP32, solver=MG)
    d.start()
    d.step(5)
    path = str(tmp_path / "v.picrst")
    d.save(path)
    d.step(5)
    a = {k: d.field(k) for k in ("phi", "phiP", "phiL0", "phiL1", "Ez")}
    d.close()
    e = P.Discharge.load(path, wl)
    e.step(5)
    for k, v in a.items():
        assert np.array_equal(v, e.field(k)), k
    assert e.status() == 0
    e.close()
