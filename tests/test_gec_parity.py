"""Full-step parity with the FP64 oracle on the configuration the benchmark runs:
the GEC-like cell (powered electrode, dielectric ring, grounded shield and
upper electrode), the L-type matching network of Eq. 10 (and circuit I's blocking
capacitor, Eq. 9) coupled through C_eq (Eqs. 5 and 8), the FP32 particle kernel with the tile shapes the tile
autotuner chooses from, and the multigrid-preconditioned solve.

Each step starts both sides from the same stored state (particles, surface
charge, circuit state and C_eq are carried over from the device after each
step) and compares, per step:
- every particle by id: position and velocity within 1e-5 relative (FP32) or
  1e-12 (FP64); every divergent particle must be a branch flip proven by the
  oracle's decision margins (tests/parity_tools.py), at most 1e-4 of the
  particles, and none in FP64 (both sides push in the device's pre-step field;
  the field solves are compared on their own);
- absorption counts per species and kind, collision and birth counts, within
  the flips;
- the surface charge on the dielectric node by node, in units of one
  macroparticle's charge, within the flips;
- electron and ion deposits and the node charge rho~ with the flipped
  particles' own deposits removed from both sides: 1e-6 relative L2 (FP32),
  1e-11 (FP64), unconditionally;
- the field solve on the device's own charge: phi within 1e-8 of the oracle's
  FP64 PCG on the same deposits;
- phi end to end (each side's own charge): 1e-8 in FP64, and in FP32 whenever no
  particle flipped in the step (measured 2e-9 to 4e-9; a flip moves one
  macroparticle's charge and is accounted for by the deposit check);
- U_E, Q_E and I_conv of the circuit (Eqs. 5, 8, 10), and after the RF window
  the chi-inclusive C_eq refresh (Eqs. 6-7) and the window averages;
- the window's circuit post-processing (Eqs. 11-14: impedances, powers, Gamma)
  to 1e-6 (FP32) or 1e-9 (FP64) while no particle has flipped: a flipped
  absorption at the powered electrode changes that step's I_conv by one
  macroparticle's charge over dt, which the per-step I_conv bound checks.
Whatever flipped, every step also compares phi with the oracle's solve of the
device's own charge (1e-8), so no FP32 step leaves phi unchecked.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import make_pair
from parity_tools import StepParity, phi_err
from paper_2310_04957_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
MG, PLAIN = 3, 0


# circuit I of Sec. 3 (Eq. 9): R_b = 0.5 ohm, L_b = 0.01 uH, blocking capacitor 5 nF
RLC = (0.5, 0.01e-6, 5e-9, 0.0, 0.0, 0.0, 0.0, 0.0)


def gec_small(n=200_000, circuit="imn", split_cells=0, nr=128, nz=64):
    # 128x64 is the coarsest grid on which the 1 mm dielectric ring survives
    # snapping (2 cells); a 3-step RF window makes the third step end a window
    wl = W.gec_case(nr, nz, 30.0, 150.0, n_per_species=n, seed_index=21, split_cells=split_cells)
    wl = dataclasses.replace(wl, steps_per_rf=3, phase_src=0.9)
    if circuit == "rlc":
        wl = dataclasses.replace(wl, circuit=W.CIRCUIT_RLC, circ=RLC)
    return wl


CASES = [
    pytest.param(FP32, MG, (2, 2), 0.0, "imn", id="fp32-mg-2x2"),
    pytest.param(FP32, MG, (4, 2), 0.0, "imn", id="fp32-mg-4x2"),
    pytest.param(FP32, MG, (4, 4), 0.0, "imn", id="fp32-mg-4x4"),
    pytest.param(FP32, MG, (8, 4), 0.0, "imn", id="fp32-mg-8x4"),
    pytest.param(FP32, MG, (4, 4), 1e-6, "imn", id="fp32-mg-4x4-overflow"),
    pytest.param(FP32, MG, (4, 4), 0.0, "rlc", id="fp32-mg-4x4-rlc"),
    pytest.param(FP64, MG, (4, 2), 0.0, "imn", id="fp64-mg-4x2"),
    pytest.param(FP64, PLAIN, (4, 4), 1e-6, "imn", id="fp64-plain-4x4-overflow"),
    pytest.param(FP64, MG, (4, 4), 0.0, "rlc", id="fp64-mg-4x4-rlc"),
    # unequal weights and splitting near the axis (Sec. 2): radially weighted
    # loading in the first 8 radial cells, split on entering a smaller cell
    pytest.param(FP32, MG, (4, 4), 0.0, "imn-split", id="fp32-mg-4x4-split"),
    pytest.param(FP32, MG, (4, 4), 1e-6, "imn-split", id="fp32-mg-4x4-split-overflow"),
    pytest.param(FP64, MG, (4, 2), 0.0, "imn-split", id="fp64-mg-4x2-split"),
    # a 130x66 grid: the last tile of every row and column is ragged (2 of 4 or
    # 8 cells), and the multigrid levels have odd node counts
    pytest.param(FP32, MG, (4, 4), 0.0, "imn-ragged", id="fp32-mg-4x4-ragged"),
    pytest.param(FP32, MG, (8, 4), 1e-6, "imn-ragged", id="fp32-mg-8x4-ragged-overflow"),
    pytest.param(FP64, MG, (4, 4), 0.0, "imn-ragged", id="fp64-mg-4x4-ragged"),
]


@pytest.mark.parametrize("precision,solver,tile,slack,circuit", CASES)
def test_gec_full_steps_match_oracle(precision, solver, tile, slack, circuit):
    split, ragged = circuit.endswith("-split"), circuit.endswith("-ragged")
    grid = dict(nr=130, nz=66) if ragged else {}
    wl = gec_small(circuit=circuit.split("-")[0], split_cells=8 if split else 0, **grid)
    if ragged:
        assert wl.nr % tile[0] and wl.nz % tile[1]
    d, o = make_pair(wl, precision, solver=solver, tile=tile, bin_slack=slack)
    o.init_fields()
    d.start()
    # the circuit starts at rest (U_E = 0) and each ion sits on its electron: phi ~ 0
    assert phi_err(d.field("phi"), o.field("phi"), wl.V_src) <= 1e-8
    assert d.scalars()["C_eq"] == pytest.approx(o.scalars()["C_eq"], rel=1e-9, abs=0)
    sp = StepParity(wl, d, o, precision == FP32)
    ceq_vac = d.scalars()["C_eq"]
    for step in range(4):
        sd = sp.step(lambda: d.step(1))
        if step == 2:
            assert sd["windows"] == 1
            assert sd["C_eq"] != pytest.approx(ceq_vac, rel=1e-6, abs=0)  # the window's refresh included chi
    assert d.status() == 0
    assert sp.surf_hits > 0, "no particle reached the dielectric surface: the surface-charge path went unchecked"
    if slack > 0:
        assert sp.overflow > 0, "the overflow region was never used"
    if split:
        assert sp.splits > 0, "no particle split: the splitting path went unchecked"
    print(f"{precision=} {tile=} flips {sp.flips} of {sp.seen} particle-steps, surface hits {sp.surf_hits}, "
          f"overflow-region particles {sp.overflow}, splits {sp.splits}, phi end to end (flips, rel L2) {sp.phi_e2e}")
