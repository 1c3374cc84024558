"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Every comparison starts both sides from the same state and the same seeded
inputs.  Tolerances: positions/velocities <= 1e-5 relative per
particle; rho~ <= 1e-6 relative L2; phi <= 1e-8 relative L2; collision-branch
divergences <= 1e-4 of particles per step; FP64 path: near machine precision.
"""
import dataclasses
import math

import numpy as np
import pytest

from gpu_common import by_id, make_pair, particles_from, pic, random_field, small
from oracle import orc
from parity_tools import COUNTERS, StepParity, classify, clean_deposits
from paper_2310_04957_gb300 import workloads as W
from util import beam, rel_l2, with_particles

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1


def test_philox_device_matches_oracle_bit_for_bit():
    P = pic()
    d = P.Discharge(small(64), precision=FP32)
    rng = np.random.default_rng(11)
    n = 20000
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    out = d.philox(ctr, key)
    assert list(out[0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    for k in range(0, n, 97):
        assert list(out[k]) == list(orc.philox(ctr[k], key[k]))


def _phase_parity(wl, precision, field_seed, steps=(3, 4)):
    """Particle phases from identical states in an identical seeded node field: every
    particle by id (1e-12 FP64, 1e-5 FP32), each divergence proven a branch flip by the
    oracle's decision margins (none allowed in FP64), the counters within the flips, and the
    deposits with the flipped particles' own removed from both sides, unconditionally."""
    d, o = make_pair(wl, precision)
    er, ez = random_field(wl, field_seed, precision=precision)
    for x in (d, o):
        x.set_field("Er", er)
        x.set_field("Ez", ez)
    tol = 1e-12 if precision == FP64 else 1e-5
    rtol_dep = 1e-11 if precision == FP64 else 1e-6
    flips = 0
    for step in steps:
        pre = [by_id(d.get_particles(s)) for s in (0, 1)]
        d.set_step(step)
        o.set_step(step)
        d.particle_phase()
        o.particle_phase()
        post_d = [d.get_particles(s) for s in (0, 1)]
        post_o = [o.get_particles(s) for s in (0, 1)]
        flipped, st = classify(wl, (er, ez), step, pre, post_d, post_o, tol)
        assert st["max_dpos"] <= tol and st["max_dvel"] <= tol, st
        n = sum(len(p["id"]) for p in pre)
        if precision == FP64:
            assert st["n"] == 0, st["margins"]
        assert st["n"] <= 1e-4 * n + 2, st
        flips += st["n"]
        sd, so = d.scalars(), o.scalars()
        for key in COUNTERS:
            assert abs(sd[key] - so[key]) <= st["n"], (key, sd[key], so[key])
        (de_d, di_d), (de_o, di_o) = clean_deposits(wl, d, o, post_d, post_o, flipped)
        assert rel_l2(de_d, de_o) <= rtol_dep
        assert rel_l2(di_d, di_o) <= rtol_dep
        rho_d = wl.q[0] * wl.w[0] * de_d + wl.q[1] * wl.w[1] * di_d
        rho_o = wl.q[0] * wl.w[0] * de_o + wl.q[1] * wl.w[1] * di_o
        assert rel_l2(rho_d, rho_o) <= rtol_dep
        assert d.field("dep_e").sum() == pytest.approx(d.count(0), rel=1e-12, abs=0)
        assert d.field("dep_i").sum() == pytest.approx(d.count(1), rel=1e-12, abs=0)
        # carry identical states into the next step
        for s in (0, 1):
            o.set_particles(s, particles_from(post_d[s]))
    return flips


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_particle_phase_parity(precision):
    """One particle phase (gather, correction, MCC, predictor, absorption, re-bin, deposit)
    from identical states with an identical random node field, twice."""
    _phase_parity(small(30_000), precision, 5)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_particles_on_faces_on_the_axis_and_at_the_outer_radius(precision):
    """Particles that start exactly on radial and axial cell faces, on the axis (r = 0) and
    just inside the outer wall (r = R(1 - 1e-12)), moving in every direction: the push, the
    axis reflection, the wall absorption and the re-bin agree with the oracle as above."""
    wl = small(16)
    rng = np.random.default_rng(17)
    nr, nz, dr, dz = wl.nr, wl.nz, wl.dr, wl.dz
    rs, zs = [], []
    for i in range(nr):  # radial faces (incl. the axis) at interior axial positions
        for z in rng.uniform(0.3, 0.7, 3) * nz * dz:
            rs.append(i * dr)
            zs.append(z)
    for j in range(1, nz):  # axial faces
        for r in rng.uniform(0.05, 0.95, 3) * nr * dr:
            rs.append(r)
            zs.append(j * dz)
    for z in rng.uniform(0.2, 0.8, 24) * nz * dz:  # at the outer radius
        rs.append(nr * dr * (1 - 1e-12))
        zs.append(z)
    n = len(rs)
    v = rng.normal(0, 3e5, (3, n))
    zeros = np.zeros(n)
    e = W.Particles(np.array(rs), np.array(zs), v[0], v[1], v[2], zeros, zeros.copy(), zeros.copy(),
                    np.arange(n, dtype=np.uint64))
    keep = np.array([wl.cell_kind[min(int(z / dz), nz - 1), min(int(r / dr), nr - 1)] == W.CELL_PLASMA
                     for r, z in zip(rs, zs)])
    e = e.take(np.nonzero(keep)[0])
    ions = dataclasses.replace(e, vr=e.vr * 1e-3, vt=e.vt * 1e-3, vz=e.vz * 1e-3,
                               id=np.arange(n, 2 * n, dtype=np.uint64)[keep])
    wl1 = with_particles(wl, electrons=e, ions=ions)
    assert e.n > 150
    _phase_parity(wl1, precision, 9, steps=(3, 4, 5))


def test_rebin_keeps_every_particle_in_its_cell():
    """After several steps every stored particle sits in the bin of its own cell, and the per-cell
    counts equal the oracle's on the same state (bit-exact integers, FP64 path)."""
    wl = small(20_000)
    d, o = make_pair(wl, FP64)
    er, ez = random_field(wl, 6, scale=5e3, precision=FP64)
    for x in (d, o):
        x.set_field("Er", er)
        x.set_field("Ez", ez)
    for step in range(3):
        d.set_step(step)
        o.set_step(step)
        d.particle_phase()
        o.particle_phase()
    for s in (0, 1):
        g = d.get_particles(s)
        i = np.floor(g["r"] / wl.dr).astype(int)
        j = np.floor(g["z"] / wl.dz).astype(int)
        assert np.array_equal(g["cell"], j * wl.nr + i)
        go = o.get_particles(s)
        cd = np.bincount(g["cell"], minlength=wl.nr * wl.nz)
        co = np.bincount(go["cell"], minlength=wl.nr * wl.nz)
        assert np.array_equal(cd, co)
        assert len(np.unique(g["id"])) == len(g["id"])


@pytest.mark.parametrize("nr,nz", [(96, 48), (128, 64), (256, 128), (64, 3)])
def test_multigrid_solve_parity_on_deeper_hierarchies(nr, nz):
    """The multigrid-preconditioned solve on grids whose coarse levels run in
    one block (in its shared memory) below one or two grid-wide levels, and on
    a 64x3 cylinder whose coarsening stops at 33x2 nodes (too many for the
    dense coarsest inverse: Jacobi sweeps there): phi and Ez within 1e-8
    relative L2 of the oracle's FP64 PCG solve of the same system."""
    if nz >= 8:
        wl = W.gec_case(nr, nz, 30.0, 150.0, n_per_species=20_000)
    else:
        wl = W._make(f"cylinder-{nr}x{nz}", nr, nz, 0.051, 0.0254, "cylinder", 100.0, 20_000, 400,
                     W.CIRCUIT_DIRECT, (), 100.0, 0)
    wl = dataclasses.replace(wl, phase_src=1.0)
    d, o = make_pair(wl, FP32)
    o.init_fields()
    d.start()
    er, ez = random_field(wl, 9, precision=FP32)
    for x in (d, o):
        x.set_field("Er", er)
        x.set_field("Ez", ez)
    d.particle_phase()
    # the deposits and the surface charge the particle phase left on the dielectric
    for name in ("dep_e", "dep_i", "sigma"):
        o.set_field(name, d.field(name))
    o.assemble()
    st_o, _, rel_o = o.field_solve()
    st_d, it_d, rel_d = d.field_solve(3)
    assert st_o == 0 and st_d == 0
    assert rel_d <= wl.pcg_tol and rel_o <= wl.pcg_tol
    assert rel_l2(d.field("rho"), o.field("rho")) <= 1e-13
    assert rel_l2(d.field("chi"), o.field("chi")) <= 1e-13
    assert it_d <= 100
    assert rel_l2(d.field("phi"), o.field("phi")) <= 1e-8
    assert rel_l2(d.field("Ez"), o.field("Ez")) <= 1e-8
    assert d.status() == 0


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_field_solve_parity(mode):
    """Assembly + field solve (0: plain FP64 PCG, 1: FP32 inner CG with FP64 refinement,
    3: FP32 inner CG preconditioned by a multigrid V-cycle, FP64 refinement) from
    identical deposits: phi within 1e-8 relative L2 of the oracle, rho~ and chi identical to
    rounding."""
    wl = small(30_000)
    wl = dataclasses.replace(wl, phase_src=1.0)
    d, o = make_pair(wl, FP32)
    o.init_fields()
    d.start()
    # move once to make a charge imbalance, then feed both the device's deposits
    er, ez = random_field(wl, 7, precision=FP32)
    for x in (d, o):
        x.set_field("Er", er)
        x.set_field("Ez", ez)
    d.particle_phase()
    for name in ("dep_e", "dep_i"):
        o.set_field(name, d.field(name))
    o.assemble()
    st_o, it_o, rel_o = o.field_solve()
    st_d, it_d, rel_d = d.field_solve(mode)
    assert st_o == 0 and st_d == 0
    assert rel_d <= wl.pcg_tol and rel_o <= wl.pcg_tol
    assert rel_l2(d.field("rho"), o.field("rho")) <= 1e-13
    assert rel_l2(d.field("chi"), o.field("chi")) <= 1e-13
    assert rel_l2(d.field("phi"), o.field("phi")) <= 1e-8
    assert rel_l2(d.field("Ez"), o.field("Ez")) <= 1e-8
    if mode == 0:
        assert abs(it_d - it_o) <= max(3, 0.05 * it_o)


@pytest.mark.parametrize("preset", ["c1", "c2"])
def test_ceq_parity(preset):
    """Vacuum C_eq (Eqs. 6-7) by the energy and the Gauss route on the GPU equals the oracle's."""
    wl = W.PRESETS[preset](n_per_species=64)
    P = pic()
    d = P.Discharge(wl, precision=FP32)
    o = orc.Oracle(wl)
    cd, gd = d.ceq(False)
    co, go = o.ceq(False)
    assert cd == pytest.approx(co, rel=1e-9, abs=0)
    assert gd == pytest.approx(go, rel=1e-7, abs=0)
    assert cd == pytest.approx(gd, rel=1e-7, abs=0)


def test_circuit_parity_imn():
    """Circuit II on the device follows the oracle's trapezoidal integration step by step."""
    wl = with_particles(W.gec_256(n_per_species=64))
    circ = (50.0, 2335.51e-12, 0.85e-6, 215.62e-12, 0.5, 10e-12, 0.5, 10e-9)
    wl = dataclasses.replace(wl, circ=circ, V_src=77.0)
    P = pic()
    d = P.Discharge(wl, precision=FP32)
    o = orc.Oracle(wl)
    for x in (d, o):
        x.set_ceq(892.07e-12)
        x.set_circuit_state(np.zeros(6))
        x.set_conv_current(0.0)
        x.set_step(0)
    Ud = d.circuit_run(4000)
    Uo = o.circuit_run(4000)
    assert np.max(np.abs(Ud - Uo)) <= 1e-9 * np.max(np.abs(Uo))


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_full_step_parity(precision):
    """Start-up and full steps (particles, circuit, assembly, PCG, E, diagnostics) from the
    same state on the direct-drive cylinder, with every per-step check of the GEC parity
    tests (tests/parity_tools.py: particles by id with proven flips, counters, deposits and
    rho~ unconditionally, U_E, C_eq, phi end to end and on the device's own charge)."""
    wl = dataclasses.replace(small(20_000), phase_src=0.7)
    d, o = make_pair(wl, precision)
    o.init_fields()
    d.start()
    assert rel_l2(d.field("phi"), o.field("phi")) <= 1e-8
    sp = StepParity(wl, d, o, precision == FP32)
    for _ in range(2):
        sd = sp.step(lambda: d.step(1))
        assert sd["U_E"] == pytest.approx(o.scalars()["U_E"], rel=1e-12, abs=0)
    assert d.status() == 0


def test_edge_cases():
    """Empty species, a single particle, invalid inputs and capacity overflow."""
    P = pic()
    wl = small(16)
    # empty
    d = P.Discharge(with_particles(wl), precision=FP32)
    d.start()
    d.step(2)
    assert d.count(0) == 0 and d.count(1) == 0
    assert d.status() == 0
    # single electron, no gas: moves ballistically
    one = beam(1, 0.02, 0.012, (1e5, 2e4, -3e4))
    wl1 = dataclasses.replace(with_particles(wl, electrons=one), n_gas=0.0, V_src=0.0)
    d = P.Discharge(wl1, precision=FP64)
    o = orc.Oracle(wl1, set_particles=False)
    o.set_particles(0, particles_from(d.get_particles(0)))
    o.set_particles(1, W.Particles(*(np.zeros(0) for _ in range(8)), np.zeros(0, np.uint64)))
    o.init_fields()
    d.start()
    o.step(3)
    d.step(3)
    gd, go = d.get_particles(0), o.get_particles(0)
    assert gd["r"][0] == pytest.approx(go["r"][0], rel=1e-12, abs=0)
    assert gd["z"][0] == pytest.approx(go["z"][0], rel=1e-12, abs=0)
    # invalid: particle inside metal
    bad = beam(1, 0.02, 0.0, (0, 0, 0))
    with pytest.raises(P.PicError):
        P.Discharge(with_particles(wl, electrons=dataclasses.replace(bad, z=np.array([-1e-3]))), precision=FP32)
    # invalid config
    with pytest.raises(P.PicError):
        P.Discharge(dataclasses.replace(wl, steps_per_rf=0), precision=FP32)
    # capacity overflow at upload
    with pytest.raises(P.PicError):
        P.Discharge(wl, precision=FP32, capacity=(8, 8))


@pytest.mark.slow
def test_rf_period_statistics_match_oracle():
    """One RF period (400 steps) of the small cylinder from the same start: RF-averaged n_e, n_i,
    ion current to the powered electrode and |I_1| within 2 % of the oracle's (FP32 path)."""
    wl = W.small_cylinder()
    d, o = make_pair(wl, FP32)
    o.init_fields()
    d.start()
    o.step(wl.steps_per_rf)
    d.step(wl.steps_per_rf)
    sd, so = d.scalars(), o.scalars()
    assert sd["windows"] == 1 and so["windows"] == 1
    for name in ("ne_avg", "ni_avg"):
        a, b = d.field(name), o.field(name)
        assert rel_l2(a, b) <= 0.02, name
    assert abs(sd["ioncur_pow"] - so["ioncur_pow"]) <= 0.02 * abs(so["ioncur_pow"]) + 1e-9
    i1d, i1o = math.hypot(sd["i1_re"], sd["i1_im"]), math.hypot(so["i1_re"], so["i1_im"])
    assert i1d == pytest.approx(i1o, rel=0.02, abs=0)
    assert d.status() == 0


def test_upload_round_trip_and_rejection():
    """The device-side upload bins every particle: downloaded by id, each keeps
    its velocity (FP32-rounded), its position within the FP32 cell offset's
    rounding and its cell; every id comes back once, and the store's per-cell
    counts match the cells of the input.  A particle in a metal cell (the
    powered electrode of the GEC-like cell) makes the upload fail."""
    wl = W.gec_case(96, 48, 30.0, 150.0, n_per_species=50_000)
    P = pic()
    d = P.Discharge(wl, precision=FP32)
    for s in (0, 1):
        src = wl.particles[s]
        g = by_id(d.get_particles(s))
        order = np.argsort(src.id, kind="stable")
        assert np.array_equal(g["id"], src.id[order])
        for k in ("vr", "vt", "vz", "ar", "at", "az"):
            np.testing.assert_array_equal(g[k], getattr(src, k)[order].astype(np.float32).astype(np.float64))
        # position: cell-relative FP32 offsets, so within ~1e-7 of a cell
        np.testing.assert_allclose(g["r"], src.r[order], rtol=0, atol=2e-7 * wl.dr)
        np.testing.assert_allclose(g["z"], src.z[order], rtol=0, atol=2e-7 * wl.dz)
        ci = np.floor(src.r[order] / wl.dr).astype(int)
        cj = np.floor(src.z[order] / wl.dz).astype(int)
        assert np.array_equal(g["cell"], cj * wl.nr + ci)
    assert d.status() == 0
    d.close()
    # a particle inside the powered electrode (r = 1 cm, z = 0.5 cm: metal)
    cell = np.asarray(wl.cell_kind).reshape(wl.nz, wl.nr)
    i, j = int(0.01 / wl.dr), int(0.005 / wl.dz)
    assert cell[j, i] != 0
    with pytest.raises(P.PicError):
        P.Discharge(with_particles(wl, electrons=beam(3, 0.01, 0.005, (0.0, 0.0, 0.0))), precision=FP32)


def test_multigrid_solve_with_reused_hierarchy_matches_oracle():
    """The multigrid solve rebuilds its coarse hierarchy every 8th solve and
    reuses it in between.  Eleven rounds of particle phase + solve while the
    deposits (and so chi and the operator) change: by the solve counter the
    kernel branches on, both the rebuild and the reuse branch run.  Each solve
    meets the tolerance, and phi and Ez stay within 1e-8 relative L2 of the
    oracle's FP64 PCG solve of the same system."""
    wl = W.gec_case(128, 64, 30.0, 150.0, n_per_species=50_000)
    wl = dataclasses.replace(wl, phase_src=1.0)
    d, o = make_pair(wl, FP32)
    o.init_fields()
    d.start()
    er, ez = random_field(wl, 13, precision=FP32)
    for x in (d, o):
        x.set_field("Er", er)
        x.set_field("Ez", ez)
    branches = set()
    for k in range(11):
        d.particle_phase()
        for name in ("dep_e", "dep_i", "sigma"):
            o.set_field(name, d.field(name))
        o.assemble()
        st_o, _, rel_o = o.field_solve()
        before = d.solver_state()
        branches.add("rebuild" if before["mg_solves"] % before["rebuild_every"] == 0 else "reuse")
        st_d, it_d, rel_d = d.field_solve(3)
        assert d.solver_state()["mg_solves"] == before["mg_solves"] + 1
        assert st_o == 0 and st_d == 0, k
        assert rel_d <= wl.pcg_tol and rel_o <= wl.pcg_tol, k
        assert rel_l2(d.field("phi"), o.field("phi")) <= 1e-8, k
        assert rel_l2(d.field("Ez"), o.field("Ez")) <= 1e-8, k
    assert branches == {"rebuild", "reuse"}, branches
    assert d.status() == 0
