"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks one part of the oracle against a closed form, a value the
paper prints, a published known answer, a library routine, or brute force;
chosen so that a dropped term, a wrong sign or index, or a transposed operand
in that part fails here.  No GPU is needed.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from oracle import orc
from paper_2310_04957_gb300 import workloads as W
from util import beam, field_only, grounded_box, rel_l2, with_particles

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS0 = 8.8541878128e-12


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors (Salmon et al. SC'11)."""
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for row in rows:
        ctr, key, want = row[:4], row[4:6], row[6:]
        assert list(orc.philox(ctr, key)) == want


def test_philox_uniformity():
    """Uniforms from consecutive counters pass a chi-square test of equidistribution."""
    u = []
    for c in range(4000):
        x = orc.philox([c, 7, 1, 0x5EED], [12345, 0])
        u.extend((int(v) >> 8) / 2**24 for v in x)
    h, _ = np.histogram(u, bins=20, range=(0, 1))
    exp = len(u) / 20
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < 45.0  # 19 dof, p ~ 1e-3


# ---------------------------------------------------------------- cross sections
def test_xs_lookup_matches_linear_interpolation():
    """Between table nodes the lookup is linear interpolation (numpy.interp); clamped outside;
    inelastic processes vanish below threshold."""
    wl = W.small_cylinder(n_per_species=16)
    o = orc.Oracle(with_particles(wl))
    E_tab, S = wl.xs_energy, wl.xs_sigma
    rng = np.random.default_rng(1)
    Es = np.concatenate([10 ** rng.uniform(-3.5, 3.5, 400), E_tab[::97]])
    for proc in range(5):
        want = np.interp(Es, E_tab, S[proc])
        if proc == 1:
            want = np.where(Es < W.THR_EXC, 0.0, want)
        if proc == 2:
            want = np.where(Es < W.THR_ION, 0.0, want)
        got = np.array([o.xs(proc, e) for e in Es])
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def test_numax_bounds_every_energy():
    """nu_max is an upper bound of n_g sigma_T(E) v(E) over the table range, and is attained
    within the interpolation slack (at most the largest neighbouring-node ratio)."""
    wl = W.small_cylinder(n_per_species=16)
    o = orc.Oracle(with_particles(wl))
    s = o.scalars()
    E = np.logspace(-3, 3, 20001)
    sig_e = sum(np.interp(E, wl.xs_energy, wl.xs_sigma[p]) * (E >= thr) for p, thr in ((0, 0), (1, W.THR_EXC), (2, W.THR_ION)))
    nu_e = wl.n_gas * sig_e * np.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ELECTRON_MASS)
    sig_i = np.interp(E, wl.xs_energy, wl.xs_sigma[3]) + np.interp(E, wl.xs_energy, wl.xs_sigma[4])
    nu_i = wl.n_gas * sig_i * np.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ARGON_MASS)
    assert nu_e.max() <= s["numax_e"] * (1 + 1e-12)
    assert nu_i.max() <= s["numax_i"] * (1 + 1e-12)
    assert nu_e.max() > 0.98 * s["numax_e"]
    assert nu_i.max() > 0.98 * s["numax_i"]
    assert s["pcoll_e"] == pytest.approx(1 - math.exp(-s["numax_e"] * wl.dt), rel=1e-14, abs=0)


# ---------------------------------------------------------------- kinematics primitives
def test_scatter_cos_is_inverse_cdf():
    """cos chi = (2 + E - 2(1+E)^R)/E is the inverse of R = ln(1 + E sin^2(chi/2)) / ln(1 + E)
    (Vahedi & Surendra's screened angular distribution), with the limits R=0 -> forward,
    R=1 -> backward, E->0 -> isotropic."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        E = 10 ** rng.uniform(-3, 3)
        R = rng.uniform()
        c = orc.scatter_cos(E, R)
        s2 = (1 - c) / 2
        assert math.log1p(E * s2) / math.log1p(E) == pytest.approx(R, abs=1e-9)
    assert orc.scatter_cos(50.0, 0.0) == pytest.approx(1.0, abs=1e-15)
    assert orc.scatter_cos(50.0, 1.0) == pytest.approx(-1.0, abs=1e-15)
    assert orc.scatter_cos(1e-14, 0.25) == pytest.approx(0.5, abs=1e-15)


def test_turn_rotates_by_the_given_angles():
    """The turned vector is a unit vector at polar angle chi from the original; over uniform
    azimuths it averages to cos(chi) times the original (no preferred side)."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        c = rng.normal(size=3)
        c /= np.linalg.norm(c)
        cc = rng.uniform(-1, 1)
        phis = np.linspace(0, 2 * math.pi, 64, endpoint=False)
        outs = np.array([orc.turn(c, cc, ph) for ph in phis])
        np.testing.assert_allclose(np.linalg.norm(outs, axis=1), 1.0, atol=1e-13)
        np.testing.assert_allclose(outs @ c, cc, atol=1e-13)
        np.testing.assert_allclose(outs.mean(axis=0), cc * c, atol=1e-12)
    # degenerate direction along z
    for sgn in (1.0, -1.0):
        out = orc.turn(np.array([0.0, 0.0, sgn]), 0.3, 1.1)
        assert np.linalg.norm(out) == pytest.approx(1.0)
        assert out[2] * sgn == pytest.approx(0.3)


# ---------------------------------------------------------------- mover
def _collisionless(wl):
    return dataclasses.replace(wl, n_gas=0.0)


def test_free_flight_is_a_straight_line():
    """E = 0, no collisions: the r-z mover with cylindrical rotation reproduces straight-line
    Cartesian motion r(t) = |(r0 + vr t, vt t)|, z = z0 + vz t, with r v_theta conserved,
    including particles that pass through the axis."""
    base = _collisionless(W.small_cylinder(n_per_species=16))
    rng = np.random.default_rng(4)
    n = 400
    r0 = rng.uniform(0.005, 0.03, n)
    z0 = rng.uniform(0.008, 0.017, n)
    v = rng.normal(0, 2e4, (3, n))
    v[0, :50] = -np.abs(v[0, :50]) * 5  # head for the axis
    v[1, :50] *= 0.01
    zeros = np.zeros(n)
    P = W.Particles(r0, z0, v[0], v[1], v[2], zeros, zeros.copy(), zeros.copy(), np.arange(n, dtype=np.uint64))
    wl = with_particles(base, electrons=P)
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    nsteps = 12
    for k in range(nsteps):
        o.set_step(k)
        o.particle_phase()
    g = o.get_particles(0)
    assert len(g["id"]) == n  # nothing reached a wall
    idx = g["id"].astype(np.int64)
    t = nsteps * wl.dt
    X = r0[idx] + v[0, idx] * t
    Y = v[1, idx] * t
    np.testing.assert_allclose(g["r"], np.hypot(X, Y), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(g["z"], z0[idx] + v[2, idx] * t, rtol=1e-12)
    np.testing.assert_allclose(g["r"] * g["vt"], r0[idx] * v[1, idx], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(g["vr"] ** 2 + g["vt"] ** 2, v[0, idx] ** 2 + v[1, idx] ** 2, rtol=1e-12)


def test_uniform_field_d1_push_is_exact_parabola():
    """Constant E_z, start-up state x~_0 = z0 - dt^2 a/2, v = v0 - 3/2 dt a, a-bar = a:
    the D1 push gives z_n = z0 + v0 t + a t^2 / 2 exactly, so x~_{n+1} = z_{n+1} - dt^2 a/2."""
    base = _collisionless(W.small_cylinder(n_per_species=16))
    Ez = -2000.0
    qm = base.q[0] / base.m[0]
    a = qm * Ez
    dt = base.dt
    n = 50
    rng = np.random.default_rng(5)
    z0 = rng.uniform(0.004, 0.006, n)
    v0 = rng.uniform(-1e5, 1e5, n)
    r0 = rng.uniform(0.01, 0.02, n)
    zeros = np.zeros(n)
    P = W.Particles(r0, z0 - 0.5 * dt * dt * a, zeros.copy(), zeros.copy(), v0 - 1.5 * dt * a, zeros.copy(),
                    zeros.copy(), a * np.ones(n), np.arange(n, dtype=np.uint64))
    o = orc.Oracle(with_particles(base, electrons=P))
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", Ez * np.ones(o.n_nodes))
    nsteps = 8
    for k in range(nsteps):
        o.set_step(k)
        o.particle_phase()
    g = o.get_particles(0)
    idx = g["id"].astype(np.int64)
    t1 = nsteps * dt  # x~ after nsteps phases predicts z at t_nsteps
    want = z0[idx] + v0[idx] * t1 + 0.5 * a * t1 * t1 - 0.5 * dt * dt * a
    np.testing.assert_allclose(g["z"], want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["r"], r0[idx], rtol=1e-14)
    # stored velocity after the last phase is v_{n-1/2} with n = nsteps - 1: v0 + a (n - 1/2) dt
    np.testing.assert_allclose(g["vz"], v0[idx] + a * ((nsteps - 1.5) * dt), rtol=1e-10)


# ---------------------------------------------------------------- weighting
def test_area_weighting_moments():
    """Deposited weights sum to one and reproduce r^2 and z linearly (the volume weighting's
    defining moments); a uniform density is recovered exactly by the node volumes."""
    base = W.small_cylinder(n_per_species=16)
    rng = np.random.default_rng(6)
    R, Z = base.nr * base.dr, base.nz * base.dz
    for _ in range(20):
        r, z = rng.uniform(0, R * 0.999), rng.uniform(0, Z * 0.999)
        P = beam(1, r, z, (0, 0, 0))
        o = orc.Oracle(with_particles(base, electrons=P))
        o.deposit_only()
        d = o.field("dep_e")
        rr = (np.arange(base.nr + 1) * base.dr)[None, :]
        zz = (np.arange(base.nz + 1) * base.dz)[:, None]
        assert d.sum() == pytest.approx(1.0, abs=1e-14)
        assert (d * rr**2).sum() == pytest.approx(r * r, rel=1e-12, abs=0)
        assert (d * zz).sum() == pytest.approx(z, rel=1e-12, abs=0)
        assert (d >= -1e-15).all()
    # node volumes: sum equals the plasma volume; interior node volume 2 pi r dr dz
    o = orc.Oracle(with_particles(base))
    V = o.field("vnode")
    assert V.sum() == pytest.approx(math.pi * R * R * Z, rel=1e-13, abs=0)
    i, j = 7, 5
    assert V[j, i] == pytest.approx(2 * math.pi * i * base.dr * base.dr * base.dz, rel=1e-13, abs=0)
    assert V[j, 0] == pytest.approx(0.5 * math.pi * base.dr**2 * base.dz, rel=1e-13, abs=0)


# ---------------------------------------------------------------- field solve
def test_manufactured_quadratic_is_exact():
    """phi = (R^2 - r^2) z (L - z) solves the 5-point axisymmetric finite-volume form of Eq. 1
    (eps uniform, chi = 0) exactly when the node charge is the source f = eps0 [4 z(L-z) +
    2 (R^2 - r^2)] times the node's axial face area times dz; PCG reaches it to 1e-10."""
    nr, nz, R, L = 24, 20, 0.05, 0.03
    node, cell, eps = grounded_box(nr, nz, R, L)
    wl = field_only(nr, nz, R, L, node, cell, eps)
    o = orc.Oracle(wl)
    o.assemble()
    dr, dz = R / nr, L / nz
    r = np.arange(nr + 1) * dr
    z = np.arange(nz + 1) * dz
    rh = np.minimum((np.arange(nr + 1) + 0.5) * dr, R)
    rl = np.maximum((np.arange(nr + 1) - 0.5) * dr, 0)
    area = math.pi * (rh**2 - rl**2)
    f = EPS0 * (4 * (z * (L - z))[:, None] + 2 * (R * R - r * r)[None, :])
    q = f * area[None, :] * dz
    o.set_field("rho", q)
    st, it, rel = o.solve_tol(1e-13)
    assert st == 0
    exact = (R * R - r * r)[None, :] * (z * (L - z))[:, None]
    phi = o.field("phi")
    assert rel_l2(phi, exact) < 1e-10
    # E at interior nodes: central difference of a quadratic is exact for E_z
    Ez = o.field("Ez")
    assert np.abs(Ez[1:-1, 1:-1] - (-(R * R - r * r)[None, 1:-1] * (L - 2 * z)[1:-1, None])).max() < 1e-8 * np.abs(Ez).max()


def test_layered_dielectric_capacitor():
    """Plates at z = 0 (1 V) and z = L (0 V), Neumann outer wall, dielectric layer eps_r = 4
    below row k: phi is piecewise linear with continuous D, and C_eq from the field energy
    (Eqs. 6-7) equals eps0 pi R^2 / (d1/eps_r + d2) exactly; the Gauss-law charge agrees."""
    nr, nz, R, L = 16, 24, 0.04, 0.024
    k, er = 9, 4.0
    node, cell, eps = grounded_box(nr, nz, R, L, neumann_wall=True, powered_bottom=True)
    eps[:k, :] = er
    cell[:k, :] = W.CELL_DIELECTRIC
    wl = field_only(nr, nz, R, L, node, cell, eps, V=1.0, phase=math.pi / 2)
    o = orc.Oracle(wl)
    ceq, gauss = o.ceq()
    d1, d2 = k * L / nz, (nz - k) * L / nz
    want = EPS0 * math.pi * R * R / (d1 / er + d2)
    assert ceq == pytest.approx(want, rel=1e-11, abs=0)
    assert gauss == pytest.approx(want, rel=1e-9, abs=0)
    o.init_fields()
    phi = o.field("phi")
    z = np.arange(nz + 1) * L / nz
    Dn = 1.0 / (d1 / er + d2)  # D / eps0
    exact = np.where(z <= d1, 1.0 - Dn * z / er, 1.0 - Dn * d1 / er - Dn * (z - d1))
    np.testing.assert_allclose(phi, np.broadcast_to(exact[:, None], phi.shape), atol=1e-10)


def test_parallel_plate_ceq_vacuum():
    """Vacuum parallel plates with a Neumann outer wall: C_eq = eps0 pi R^2 / d on any grid."""
    for nr, nz in ((8, 5), (20, 33)):
        R, d = 0.051, 0.0254
        node, cell, eps = grounded_box(nr, nz, R, d, neumann_wall=True, powered_bottom=True)
        o = orc.Oracle(field_only(nr, nz, R, d, node, cell, eps))
        c, g = o.ceq()
        assert c == pytest.approx(EPS0 * math.pi * R * R / d, rel=1e-11, abs=0)
        assert g == pytest.approx(c, rel=1e-9, abs=0)


def test_pcg_matches_dense_solve():
    """On small grids with dielectric, metal inserts and random charge, the PCG solution equals
    a dense direct solve (numpy.linalg.solve) of the same conductance network."""
    rng = np.random.default_rng(7)
    for trial in range(3):
        nr, nz = 9 + trial, 7 + 2 * trial
        R, Z = 0.02, 0.015
        node, cell, eps = grounded_box(nr, nz, R, Z, neumann_wall=(trial == 1), powered_bottom=True)
        eps[: 2, 3:6] = 3.0
        cell[: 2, 3:6] = W.CELL_DIELECTRIC
        node[3:5, 6:8] = W.NODE_GROUNDED
        cell[3:4, 6:7] = W.CELL_GROUNDED
        wl = field_only(nr, nz, R, Z, node, cell, eps, V=37.0, phase=0.4)
        o = orc.Oracle(wl)
        o.init_fields()
        q = rng.normal(0, 1e-12, (nz + 1, nr + 1)) * (node == W.NODE_FREE)
        o.set_field("rho", q)
        st, it, rel = o.solve_tol(1e-13)
        assert st == 0
        Gr, Gz = o.operator()
        n = (nr + 1) * (nz + 1)
        A = np.zeros((n, n))
        idx = lambda i, j: j * (nr + 1) + i
        for j in range(nz + 1):
            for i in range(nr):
                a, b, g = idx(i, j), idx(i + 1, j), Gr[j, i]
                A[a, a] += g; A[b, b] += g; A[a, b] -= g; A[b, a] -= g
        for j in range(nz):
            for i in range(nr + 1):
                a, b, g = idx(i, j), idx(i, j + 1), Gz[j, i]
                A[a, a] += g; A[b, b] += g; A[a, b] -= g; A[b, a] -= g
        U = 37.0 * math.sin(0.4)
        fixed = node.ravel() != W.NODE_FREE
        phid = np.where(node.ravel() == W.NODE_POWERED, U, 0.0)
        free = ~fixed
        rhs = q.ravel()[free] - A[np.ix_(free, fixed)] @ phid[fixed]
        sol = np.linalg.solve(A[np.ix_(free, free)], rhs)
        phi = o.field("phi").ravel()
        assert rel_l2(phi[free], sol) < 1e-10
        assert np.all(phi[fixed] == phid[fixed])


# ---------------------------------------------------------------- circuit
def _phasor_rlc(V, f, Rb, Lb, Cb, Ceq):
    w = 2 * math.pi * f
    Zb = Rb + 1j * w * Lb + 1 / (1j * w * Cb)
    Zc = 1 / (1j * w * Ceq)
    return V * Zc / (Zc + Zb)


def _phasor_imn(V, f, Rs, Cm1, Lm, Cm2, Rm, Cst, Rst, Lst, Ceq):
    w = 2 * math.pi * f
    Zc = 1 / (1j * w * Ceq)
    Zst = Rst + 1j * w * Lst + 1 / (1j * w * Cst)
    Zload = Zc * Zst / (Zc + Zst)
    Z2 = Rm + 1j * w * Lm + 1 / (1j * w * Cm2) + Zload
    Z1 = 1 / (1j * w * Cm1)
    Zin = Z1 * Z2 / (Z1 + Z2)
    Uin = V * Zin / (Rs + Zin)
    return Uin * Zload / Z2


def _run_circuit(wl, ceq, periods):
    o = orc.Oracle(wl)
    o.set_ceq(ceq)
    o.set_circuit_state(np.zeros(6))
    o.set_conv_current(0.0)
    o.set_step(0)
    N = wl.steps_per_rf
    U = o.circuit_run(periods * N)[-N:]
    t = (np.arange((periods - 1) * N, periods * N) + 1) * wl.dt
    c = 2 / N * np.sum(U * np.exp(-1j * 2 * math.pi * wl.f_src * t))
    return c, U


def test_circuit_rlc_matches_phasor():
    """Circuit I (Eq. 9) with the electrode as C_eq (Eqs. 5, 8): periodic steady state of the
    trapezoidal integrator equals the phasor solution of the series R-L-C_b-C_eq loop."""
    wl = with_particles(W.small_cylinder(n_per_species=16))
    wl = dataclasses.replace(wl, circuit=W.CIRCUIT_RLC, circ=(0.5, 0.01e-6, 5e-9) + (0.0,) * 5, steps_per_rf=200,
                             dt=1 / W.F_RF / 200, V_src=100.0)
    ceq = 7.35e-12
    c, U = _run_circuit(wl, ceq, 40)
    want = _phasor_rlc(100.0, W.F_RF, 0.5, 0.01e-6, 5e-9, ceq)
    # phasor of sin(wt) is -j * amplitude in the e^{-j w t} DFT convention
    assert abs(c) == pytest.approx(abs(want), rel=2e-5, abs=0)
    assert np.angle(c / (-1j * want)) == pytest.approx(0.0, abs=2e-4)


def test_circuit_imn_reproduces_paper_vacuum_match():
    """Circuit II (Eq. 10) with the paper's vacuum numbers (C_eq = 892.07 pF, matched C_m1, C_m2,
    77 V source): the integrator's steady state equals the phasor solution, and the electrode
    amplitude is the paper's ~100 V (Sec. 3)."""
    g = {}
    for line in open(os.path.join(GOLDEN, "paper_circuit2_vacuum.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        g[k] = float(v)
    circ = (g["R_s"], g["C_m1"], g["L_m"], g["C_m2"], g["R_m"], g["C_stray"], g["R_stray"], g["L_stray"])
    wl = with_particles(W.small_cylinder(n_per_species=16))
    wl = dataclasses.replace(wl, circuit=W.CIRCUIT_IMN, circ=circ, steps_per_rf=200, dt=1 / g["f"] / 200,
                             V_src=g["V_source"], f_src=g["f"])
    c, U = _run_circuit(wl, g["C_eq"], 500)  # the matched network settles in ~400 periods
    want = _phasor_imn(g["V_source"], g["f"], *circ, g["C_eq"])
    assert abs(c) == pytest.approx(abs(want), rel=2e-6, abs=0)
    assert abs(want) == pytest.approx(g["U_electrode_amplitude"], rel=5e-3, abs=0)
    assert np.abs(U).max() == pytest.approx(g["U_electrode_amplitude"], rel=5e-3, abs=0)


# ---------------------------------------------------------------- MCC
def _mcc_workload(n_gas, T_gas=300.0, zero_rows=()):
    wl = W.small_cylinder(n_per_species=16)
    sig = wl.xs_sigma.copy()
    for r in zero_rows:
        sig[r] = 0.0
    return dataclasses.replace(wl, n_gas=n_gas, T_gas=T_gas, xs_sigma=sig)


def _energy_eV(g, mass):
    return 0.5 * mass * (g["vr"] ** 2 + g["vt"] ** 2 + g["vz"] ** 2) / W.ELEMENTARY_CHARGE


def test_electron_collision_counts_match_rates():
    """Monoenergetic electrons, no field: per process, the number of collisions in one step is
    N P nu_k(E)/nu_max within 5 binomial standard deviations (null-collision method, Sec. 2)."""
    for E in (5.0, 30.0, 120.0):
        base = _mcc_workload(3.2e21)
        speed = math.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ELECTRON_MASS)
        n = 200_000
        wl = with_particles(base, electrons=beam(n, 0.02, 0.0127, (0.0, 0.0, speed)))
        o = orc.Oracle(wl)
        o.set_field("Er", np.zeros(o.n_nodes))
        o.set_field("Ez", np.zeros(o.n_nodes))
        o.set_step(3)
        o.particle_phase()
        s = o.scalars()
        P = s["pcoll_e"]
        nus = [base.n_gas * np.interp(E, base.xs_energy, base.xs_sigma[p]) * speed * (E >= thr)
               for p, thr in ((0, 0), (1, W.THR_EXC), (2, W.THR_ION))]
        for nu, key in zip(nus, ("coll_e_el", "coll_e_ex", "coll_e_iz")):
            p = P * nu / s["numax_e"]
            mean, sd = n * p, math.sqrt(n * p * (1 - p))
            assert abs(s[key] - mean) <= 5 * sd + 1, (E, key, s[key], mean)
        assert s["born_e"] == s["coll_e_iz"] and s["born_i"] == s["coll_e_iz"]


def test_ion_collision_counts_cold_gas():
    """Ions in a (nearly) cold gas: relative speed = ion speed, so counts follow nu_k/nu_max."""
    E = 8.0
    base = _mcc_workload(3.2e21, T_gas=1e-9)
    speed = math.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ARGON_MASS)
    n = 200_000
    wl = with_particles(base, ions=beam(n, 0.02, 0.0127, (speed, 0.0, 0.0)))
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    o.set_step(9)
    o.particle_phase()
    s = o.scalars()
    for proc, key in ((3, "coll_i_iso"), (4, "coll_i_cx")):
        nu = base.n_gas * np.interp(E, base.xs_energy, base.xs_sigma[proc]) * speed
        p = s["pcoll_i"] * nu / s["numax_i"]
        mean, sd = n * p, math.sqrt(n * p * (1 - p))
        assert abs(s[key] - mean) <= 5 * sd + 1, (key, s[key], mean)


def test_ionization_and_excitation_energy_balance():
    """With only ionization (or only excitation) enabled, the electrons' total kinetic energy
    drops by exactly 15.76 eV (11.5 eV) per collision: E_in - 15.76 = E_scattered + E_ejected.
    New Ar+ are Maxwellian at the gas temperature."""
    E = 100.0
    speed = math.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ELECTRON_MASS)
    n = 100_000
    for zero_rows, thr, key in (((0, 1), W.THR_ION, "coll_e_iz"), ((0, 2), W.THR_EXC, "coll_e_ex")):
        base = _mcc_workload(3.0e22, zero_rows=zero_rows)
        wl = with_particles(base, electrons=beam(n, 0.025, 0.0127, (0.3 * speed, 0.0, 0.9539392014169456 * speed)))
        o = orc.Oracle(wl)
        o.set_field("Er", np.zeros(o.n_nodes))
        o.set_field("Ez", np.zeros(o.n_nodes))
        o.set_step(1)
        o.particle_phase()
        s = o.scalars()
        g = o.get_particles(0)
        assert s[key] > 1000
        total_in = n * 0.5 * W.ELECTRON_MASS * speed**2 / W.ELEMENTARY_CHARGE
        total_out = _energy_eV(g, W.ELECTRON_MASS).sum()
        assert total_out == pytest.approx(total_in - s[key] * thr, rel=1e-11, abs=0)
        if key == "coll_e_iz":
            ions = o.get_particles(1)
            assert len(ions["id"]) == s["coll_e_iz"]
            sig2 = W.BOLTZMANN * base.T_gas / W.ARGON_MASS
            for comp in ("vr", "vt", "vz"):
                v = ions[comp]
                m = len(v)
                assert abs(v.mean()) < 5 * math.sqrt(sig2 / m)
                assert v.var() == pytest.approx(sig2, rel=5 * math.sqrt(2 / m), abs=0)
            assert np.all(ions["id"] >= np.uint64(1 << 63))
            assert len(np.unique(ions["id"])) == len(ions["id"])


def test_ion_isotropic_and_charge_exchange_cold_gas():
    """Cold gas (neutral at rest): charge exchange leaves the ion at rest; isotropic scattering in
    the centre-of-mass frame of equal masses gives |v'|^2/|v|^2 = (1 + cos theta)/2, uniform on
    [0, 1] (energy conservation in the CM frame)."""
    E = 30.0
    speed = math.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ARGON_MASS)
    n = 100_000
    for zero_row, key in ((4, "coll_i_iso"), (3, "coll_i_cx")):
        base = _mcc_workload(3.0e23, T_gas=1e-12, zero_rows=(zero_row,))
        wl = with_particles(base, ions=beam(n, 0.025, 0.0127, (0.0, 0.0, speed)))
        o = orc.Oracle(wl)
        o.set_field("Er", np.zeros(o.n_nodes))
        o.set_field("Ez", np.zeros(o.n_nodes))
        o.set_step(2)
        o.particle_phase()
        s = o.scalars()
        g = o.get_particles(1)
        ratio = (g["vr"] ** 2 + g["vt"] ** 2 + g["vz"] ** 2) / speed**2
        moved = ratio < 1 - 1e-9
        assert moved.sum() == pytest.approx(s[key], abs=2)
        if key == "coll_i_cx":
            assert np.all(ratio[moved] < 1e-15)  # neutral speed at 1e-12 K is ~1e-5 m/s
        else:
            x = np.sort(ratio[moved])
            ks = np.abs(x - np.arange(1, len(x) + 1) / len(x)).max()
            assert ks < 1.95 / math.sqrt(len(x))  # KS test vs uniform, p ~ 1e-3


def test_elastic_energy_loss_bounds():
    """Electron elastic scattering loses a fraction 2 m/M (1 - cos chi) in [0, 4 m/M] of E."""
    E = 40.0
    speed = math.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ELECTRON_MASS)
    n = 50_000
    base = _mcc_workload(3.0e22, zero_rows=(1, 2))
    wl = with_particles(base, electrons=beam(n, 0.025, 0.0127, (0.0, 0.0, speed)))
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    o.particle_phase()
    g = o.get_particles(0)
    frac = 1 - _energy_eV(g, W.ELECTRON_MASS) / E
    assert (frac > -1e-12).all()
    assert (frac < 4 * W.ELECTRON_MASS / W.ARGON_MASS + 1e-12).all()
    assert (frac > 1e-9).sum() == pytest.approx(o.scalars()["coll_e_el"], abs=5)


# ---------------------------------------------------------------- whole step
def test_step_conserves_particles_and_charge():
    """One full step of the small cylinder: deposited counts sum to the particle numbers, the
    number balance old + born - absorbed = new holds, and the field residual meets 1e-10."""
    wl = W.small_cylinder(n_per_species=20_000)
    o = orc.Oracle(wl)
    o.init_fields()
    n0 = [o.count(0), o.count(1)]
    o.step(1)
    s = o.scalars()
    for spc, tag in ((0, "e"), (1, "i")):
        absn = sum(s[f"absn_{tag}_{k}"] for k in ("pow", "gnd", "surf"))
        assert o.count(spc) == n0[spc] + s[f"born_{tag}"] - absn
        assert o.field("dep_e" if spc == 0 else "dep_i").sum() == pytest.approx(o.count(spc), rel=1e-12, abs=0)
    assert s["pcg_relres"] <= 1e-10
    g = o.get_particles(0)
    assert np.all(np.diff(g["cell"]) >= 0)  # re-binned by cell


def test_efield_rules_on_a_linear_potential():
    """Between plates with a Neumann wall phi is linear in z (slope -D/eps in each layer): the
    node field is exact with central differences inside each layer, one-sided at the plates,
    and E_r = 0 everywhere (axis rule and no radial variation)."""
    nr, nz, R, L = 10, 12, 0.03, 0.024
    node, cell, eps = grounded_box(nr, nz, R, L, neumann_wall=True, powered_bottom=True)
    o = orc.Oracle(field_only(nr, nz, R, L, node, cell, eps, V=3.0, phase=math.pi / 2))
    o.init_fields()
    Ez, Er = o.field("Ez"), o.field("Er")
    np.testing.assert_allclose(Ez, 3.0 / L, rtol=1e-8)  # PCG tolerance; a wrong one-sided rule is off by 2x
    assert np.abs(Er).max() < 1e-9 * 3.0 / L


def test_first_harmonic_of_direct_drive_current():
    """Direct drive, no particles: I_ccp(t_{n+1}) = C_eq (U(t_{n+1}) - U(t_n)) / dt, whose
    first Fourier coefficient over one RF period is C_eq V (2 sin(w dt/2)/dt) exp(-i w dt/2)
    (the diagnostic's DFT, Eq. 11's fundamental)."""
    base = W.small_cylinder(n_per_species=16)
    wl = dataclasses.replace(with_particles(base), V_src=80.0, phase_src=0.3, ceq_refresh=0)
    o = orc.Oracle(wl)
    o.init_fields()
    o.step(wl.steps_per_rf)
    s = o.scalars()
    assert s["windows"] == 1
    w, dt = 2 * math.pi * wl.f_src, wl.dt
    amp = s["C_eq"] * 80.0 * 2 * math.sin(w * dt / 2) / dt
    # I_ccp(t_{n+1}) = C V (sin(w t_{n+1}+ph) - sin(w t_n+ph))/dt = amp cos(w t_{n+1} + ph - w dt/2)
    # -> coefficient of exp(i w t): amp/2 exp(i(ph - w dt/2)); the DFT returns 2 x conj-coefficient
    want = amp * complex(math.cos(0.3 - w * dt / 2), math.sin(0.3 - w * dt / 2))
    got = complex(s["i1_re"], s["i1_im"])
    assert abs(got - want) <= 1e-9 * abs(want)
    assert np.abs(o.field("ne_avg")).max() == 0.0


# ---------------------------------------------------------------- implicit susceptibility chi
def _exact_uniform_deposit(o, wl, n, species=(0, 1)):
    """Node counts of a uniform density n: w dep / V_node = n exactly."""
    v = o.field("vnode")
    for s in (0, 1):
        o.set_field("dep_e" if s == 0 else "dep_i", n * v / wl.w[s] if s in species else 0 * v)
    return v


def _omega_p2(n, mass):
    """Plasma frequency squared n e^2 / (eps0 m) (textbook form)."""
    return n * W.ELEMENTARY_CHARGE**2 / (EPS0 * mass)


def test_chi_of_a_uniform_density_is_half_omega_p_dt_squared():
    """For a uniform density n of both species, chi = (dt^2 / 2) (w_pe^2 + w_pi^2) at every node
    that touches plasma (the D1 susceptibility, Eq. 1 and its implicit coefficient), and 0 at
    nodes inside the metal and dielectric of the GEC-like cell."""
    wl = W.gec_case(64, 32, 30.0, 150.0, n_per_species=1000)
    o = orc.Oracle(wl)
    n = 3.7e15
    v = _exact_uniform_deposit(o, wl, n)
    o.assemble()
    chi = o.field("chi")
    want = 0.5 * wl.dt**2 * (_omega_p2(n, W.ELECTRON_MASS) + _omega_p2(n, W.ARGON_MASS))
    assert 0.05 < want < 5  # a regime where a factor 2 is visible
    touched = v > 0
    assert touched.sum() > 100 and (~touched).sum() > 100
    np.testing.assert_allclose(chi[touched], want, rtol=1e-12)
    assert np.all(chi[~touched] == 0.0)
    # the statistical version: a seeded uniform population of density n0 deposited by the
    # oracle's own weighting gives the same chi on average over the interior nodes
    wl2 = W.small_cylinder(n_per_species=200_000)
    o2 = orc.Oracle(wl2)
    o2.deposit_only()
    o2.assemble()
    n0 = 1e15
    want2 = 0.5 * wl2.dt**2 * (_omega_p2(n0, W.ELECTRON_MASS) + _omega_p2(n0, W.ARGON_MASS))
    inner = o2.field("chi")[1:-1, 1:-1]
    assert inner.mean() == pytest.approx(want2, rel=0.02, abs=0)


def test_chi_filled_layered_capacitor():
    """Plates at z = 0 (1 V) and z = L, Neumann outer wall, a dielectric layer (eps_r = 4, no
    chi: particles never enter it) below row k and plasma of uniform chi above: the chi-inclusive
    C_eq (Eqs. 6-7 with the implicit coefficient of Eq. 1) is
    eps0 pi R^2 / (d1/eps_r + d2/(1 + chi)) exactly, and the vacuum one has chi -> 0."""
    nr, nz, R, L = 16, 24, 0.04, 0.024
    k, er = 9, 4.0
    node, cell, eps = grounded_box(nr, nz, R, L, neumann_wall=True, powered_bottom=True)
    eps[:k, :] = er
    cell[:k, :] = W.CELL_DIELECTRIC
    wl = field_only(nr, nz, R, L, node, cell, eps, V=1.0, phase=math.pi / 2)
    o = orc.Oracle(wl)
    chi0 = 0.7
    n = chi0 / (0.5 * wl.dt**2 * _omega_p2(1.0, W.ELECTRON_MASS))  # electrons only
    _exact_uniform_deposit(o, wl, n, species=(0,))
    o.assemble()
    d1, d2 = k * L / nz, (nz - k) * L / nz
    c_chi, g_chi = o.ceq(with_chi=True)
    assert c_chi == pytest.approx(EPS0 * math.pi * R * R / (d1 / er + d2 / (1 + chi0)), rel=1e-10, abs=0)
    assert g_chi == pytest.approx(c_chi, rel=1e-8, abs=0)
    c_vac, _ = o.ceq(with_chi=False)
    assert c_vac == pytest.approx(EPS0 * math.pi * R * R / (d1 / er + d2), rel=1e-10, abs=0)


# ---------------------------------------------------------------- absorption credit
def _gec_ballistic(particles_e, particles_i, **kw):
    """The 128x64 GEC-like cell with no gas and no source: particles fly straight."""
    base = W.gec_case(128, 64, 30.0, 150.0, n_per_species=16)
    wl = with_particles(dataclasses.replace(base, n_gas=0.0, V_src=0.0, **kw), electrons=particles_e,
                        ions=particles_i)
    return wl


def test_credit_routes_each_exit_to_its_node():
    """A particle that leaves the plasma gives its charge to the node nearest its exit point
    (Sec. 2's boundary treatment, Eq. 8): into the powered electrode's top face -> that
    electrode's convective charge; into the grounded upper electrode -> grounded tally only;
    into the dielectric ring, nearest a free ring node -> surface charge on that node.  The
    ring case exits at 0.7 of a cell past a powered node, so truncating instead of rounding
    sends it to the electrode."""
    base = W.gec_case(128, 64, 30.0, 150.0, n_per_species=16)
    dr, dz, dt = base.dr, base.dz, base.dt
    node = np.asarray(base.node_kind).reshape(base.nz + 1, base.nr + 1)
    assert node[16, 65] == W.NODE_POWERED and node[16, 66] == W.NODE_FREE and node[16, 67] == W.NODE_GROUNDED
    assert node[43, 11] == W.NODE_GROUNDED
    v = 0.5 * dz / dt
    e = W.Particles(np.array([30.3 * dr, 10.6 * dr, 65.7 * dr]), np.array([16.2 * dz, 42.8 * dz, 16.3 * dz]),
                    np.zeros(3), np.zeros(3), np.array([-v, v, -v]), np.zeros(3), np.zeros(3), np.zeros(3),
                    np.arange(3, dtype=np.uint64))
    i = beam(1, 20.4 * dr, 16.3 * dz, (0.0, 0.0, -v), start_id=10)
    wl = _gec_ballistic(e, i)
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    o.particle_phase()
    s = o.scalars()
    qe, qi = wl.q[0] * wl.w[0], wl.q[1] * wl.w[1]
    assert (s["absn_e_pow"], s["absn_e_gnd"], s["absn_e_surf"]) == (1, 1, 1)
    assert (s["absn_i_pow"], s["absn_i_gnd"], s["absn_i_surf"]) == (1, 0, 0)
    assert s["absq_e_pow"] == qe and s["absq_e_gnd"] == qe and s["absq_e_surf"] == qe
    assert s["absq_i_pow"] == qi
    sig = o.field("sigma")
    assert sig[16, 66] == qe
    assert np.count_nonzero(sig) == 1
    assert o.count(0) == 0 and o.count(1) == 0
    # the convective current of Eq. 8 is the powered electrode's absorbed charge per dt
    wl1 = _gec_ballistic(e.take([0]), i.take([]) if hasattr(i, "take") else None)
    o1 = orc.Oracle(wl1)
    o1.init_fields()
    o1.step(1)
    assert o1.scalars()["I_conv"] == pytest.approx(qe / dt, rel=1e-14, abs=0)


# ---------------------------------------------------------------- window averages
def test_window_average_of_a_frozen_uniform_population_is_n0():
    """Particles at rest on a lattice that samples a uniform density n0 exactly (per cell, r^2
    and z at the midpoints of equal subdivisions, counts proportional to the cell volume), ions on
    their electrons, no gas, no source: nothing moves, and the RF-window averages of n_e and n_i
    equal n0 at every node that touches plasma (Sec. 3's averaged densities)."""
    base = W.small_cylinder(n_per_species=16)
    nr, nz, dr, dz = base.nr, base.nz, base.dr, base.dz
    K0, M = 1, 2
    rs, zs = [], []
    for j in range(nz):
        for i in range(nr):
            K = K0 * (2 * i + 1)
            for k in range(K):
                for m in range(M):
                    rs.append(math.sqrt((i * dr) ** 2 + (k + 0.5) / K * (((i + 1) * dr) ** 2 - (i * dr) ** 2)))
                    zs.append((j + (m + 0.5) / M) * dz)
    n = len(rs)
    n0 = 2.5e15
    w = n0 * math.pi * dr * dr * dz / (K0 * M)  # N_cell / V_cell = K0 M / (pi dr^2 dz)
    z0 = np.zeros(n)
    e = W.Particles(np.array(rs), np.array(zs), z0, z0, z0, z0, z0, z0, np.arange(n, dtype=np.uint64))
    ions = W.Particles(np.array(rs), np.array(zs), z0, z0, z0, z0, z0, z0, np.arange(n, 2 * n, dtype=np.uint64))
    wl = with_particles(dataclasses.replace(base, n_gas=0.0, V_src=0.0, steps_per_rf=4, w=(w, w), ceq_refresh=0),
                        electrons=e, ions=ions)
    o = orc.Oracle(wl)
    o.init_fields()
    o.step(4)
    s = o.scalars()
    assert s["windows"] == 1
    v = o.field("vnode")
    for name in ("ne_avg", "ni_avg"):
        a = o.field(name)
        np.testing.assert_allclose(a[v > 0], n0, rtol=1e-12)
        assert np.all(a[v == 0] == 0.0)
    assert o.count(0) == n and o.count(1) == n


def test_window_ion_current_of_a_steady_beam():
    """Ions of negligible weight in layers half a flight apart above the powered plate, moving
    down at 0.3 cells per step: exactly one layer of K ions reaches the plate each step, so the
    window's ion current to the powered electrode is K q w / dt and nothing reaches ground."""
    base = W.small_cylinder(n_per_species=16)
    dt, dz, dr = base.dt, base.dz, base.dr
    v = 0.3 * dz / dt
    K, L, N = 7, 6, 5
    rs = np.repeat((12.0 + np.linspace(0.2, 0.8, K)) * dr, L)
    zs = np.tile((np.arange(L) + 0.5) * v * dt, K)
    nI = K * L
    z0 = np.zeros(nI)
    ions = W.Particles(rs, zs, z0, z0, np.full(nI, -v), z0, z0, z0, np.arange(nI, dtype=np.uint64))
    wl = with_particles(dataclasses.replace(base, n_gas=0.0, V_src=0.0, steps_per_rf=N, w=(base.w[0], 1e-3),
                                            ceq_refresh=0), ions=ions)
    o = orc.Oracle(wl)
    o.init_fields()
    o.step(N)
    s = o.scalars()
    assert s["windows"] == 1
    assert s["ioncur_pow"] == pytest.approx(K * W.ELEMENTARY_CHARGE * 1e-3 / dt, rel=1e-12, abs=0)
    assert s["ioncur_gnd"] == 0.0 and s["ioncur_surf"] == 0.0
    assert o.count(1) == nI - N * K


# ---------------------------------------------------------------- elastic energy loss
def test_elastic_energy_loss_mean_matches_the_screened_closed_form():
    """Averaged over the scattering-angle law cos chi = (2 + E - 2 (1+E)^R)/E (R uniform), the
    fractional energy loss 2 (m/M)(1 - cos chi) of an elastic collision has the closed form
    2 (m/M) (2/ln(1+E) - 2/E) (using E[(1+E)^R] = E / ln(1+E)); the mean over the collided
    electrons of one step matches it within 5 standard errors."""
    E = 40.0
    speed = math.sqrt(2 * E * W.ELEMENTARY_CHARGE / W.ELECTRON_MASS)
    n = 200_000
    base = _mcc_workload(1.0e22, zero_rows=(1, 2))
    wl = with_particles(base, electrons=beam(n, 0.025, 0.0127, (0.0, 0.0, speed)))
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    o.particle_phase()
    g = o.get_particles(0)
    frac = 1 - _energy_eV(g, W.ELECTRON_MASS) / E
    hit = frac > 1e-12
    assert hit.sum() > 20_000
    mM = W.ELECTRON_MASS / W.ARGON_MASS
    want = 2 * mM * (2 / math.log(1 + E) - 2 / E)
    got, se = frac[hit].mean(), frac[hit].std() / math.sqrt(hit.sum())
    assert abs(got - want) <= 5 * se, (got, want, se)


def test_chi_filled_coaxial_capacitor():
    """A powered rod (r <= r_a), a dielectric shell (eps_r = 3, no chi) to r_b, plasma of
    uniform chi out to the grounded wall at R, free (Neumann) end faces: phi depends on r
    only, every column of radial edges is one series chain, and the chi-inclusive C_eq is
    1 / sum_i dr / (eps0 kappa_i 2 pi r_{i+1/2} Z) exactly (the radial face area of the
    finite-volume grid, kappa = eps_r in the shell and 1 + chi in the plasma)."""
    nr, nz, R, Z = 20, 6, 0.02, 0.006
    ia, ib, er = 4, 9, 3.0
    dr = R / nr
    node = np.zeros((nz + 1, nr + 1), np.int8)
    node[:, : ia + 1] = W.NODE_POWERED
    node[:, nr] = W.NODE_GROUNDED
    cell = np.zeros((nz, nr), np.int8)
    eps = np.ones((nz, nr))
    cell[:, :ia] = W.CELL_POWERED
    cell[:, ia:ib] = W.CELL_DIELECTRIC
    eps[:, ia:ib] = er
    wl = field_only(nr, nz, R, Z, node, cell, eps, V=1.0, phase=math.pi / 2)
    o = orc.Oracle(wl)
    chi0 = 0.9
    n = chi0 / (0.5 * wl.dt**2 * _omega_p2(1.0, W.ELECTRON_MASS))
    _exact_uniform_deposit(o, wl, n, species=(0,))
    o.assemble()
    kappa = np.where(np.arange(nr) < ib, er, 1 + chi0)[ia:]
    rh = (np.arange(ia, nr) + 0.5) * dr
    want = 1.0 / np.sum(dr / (EPS0 * kappa * 2 * math.pi * rh * Z))
    c_chi, g_chi = o.ceq(with_chi=True)
    assert c_chi == pytest.approx(want, rel=1e-10, abs=0)
    assert g_chi == pytest.approx(c_chi, rel=1e-8, abs=0)


# ---------------------------------------------------------------- circuit post-processing
def _paper_vacuum_circuit():
    g = {}
    for line in open(os.path.join(GOLDEN, "paper_circuit2_vacuum.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = float(v)
    return g


def _phasor_circuit_ii(g, C_load):
    """Steady state of circuit II (Eq. 10's network) with a capacitive load C_load by complex
    impedances: source V (amplitude) and R_s, shunt C_m1, series R_m + L_m + C_m2, then the
    stray branch (R, L, C) in parallel with the load.  Returns the currents, voltages, the
    impedances Z_ccp and Z_load, Gamma and the period-averaged powers 1/2 Re(U I*)."""
    w = 2 * math.pi * g["f"]
    zc = lambda C: 1 / (1j * w * C)
    z_ccp = zc(C_load)
    z_st = g["R_stray"] + 1j * w * g["L_stray"] + zc(g["C_stray"])
    z_b = 1 / (1 / z_ccp + 1 / z_st)
    z_a = g["R_m"] + 1j * w * g["L_m"] + zc(g["C_m2"]) + z_b
    z_load = 1 / (1 / zc(g["C_m1"]) + 1 / z_a)
    V = g["V_source"]
    I1 = V / (g["R_s"] + z_load)
    Uin = I1 * z_load
    I2 = Uin / z_a
    Ub = I2 * z_b
    Iccp, Ist = Ub / z_ccp, Ub / z_st
    gamma = (z_load - g["R_s"]) / (z_load + g["R_s"])
    P = lambda U, I: 0.5 * (U * I.conjugate()).real
    pf = P(Uin, I1)
    # the time-domain state at t = 0 of Eq. 10 (Q_1, Q_2, I_2, Q_ccp, I_stray, Q_E) for a
    # source V sin(w t) = Re(-j V e^{jwt}): x(0) = Re(X) with X the phasor, charge = current / (j w)
    s = -1j  # phasors above are for a source V e^{jwt}; a sine source multiplies them by -j
    q = lambda I: (s * I / (1j * w)).real
    y0 = np.array([q(I1), q(I2), (s * I2).real, q(Iccp), (s * Ist).real, q(Iccp)])
    return dict(z_ccp=z_ccp, z_load=z_load, gamma=gamma, Ub=Ub, p_source=P(V, I1), p_rs=0.5 * g["R_s"] * abs(I1) ** 2,
                p_series=0.5 * g["R_m"] * abs(I2) ** 2, p_stray=0.5 * g["R_stray"] * abs(Ist) ** 2, p_ccp=P(Ub, Iccp),
                p_forward=pf, p_ref=pf * abs(gamma) ** 2, y0=y0)


def _vacuum_match_run(g, ref, n_sub, periods=5):
    base = W.small_cylinder(n_per_species=16)
    circ = (g["R_s"], g["C_m1"], g["L_m"], g["C_m2"], g["R_m"], g["C_stray"], g["R_stray"], g["L_stray"])
    wl = dataclasses.replace(with_particles(base), circuit=W.CIRCUIT_IMN, circ=circ, V_src=g["V_source"],
                             f_src=g["f"], phase_src=0.0, steps_per_rf=200, dt=1 / g["f"] / 200, ceq_refresh=0,
                             n_sub=n_sub)
    o = orc.Oracle(wl)
    o.set_ceq(g["C_eq"])
    o.set_circuit_state(ref["y0"])
    o.set_conv_current(0.0)
    o.set_step(0)
    out = []
    for _ in range(periods):
        o.circuit_run(wl.steps_per_rf)
        out.append(o.circuit_diag())
    return out


def test_circuit_postprocessing_matches_phasor_solution_of_the_vacuum_match():
    """Circuit II loaded by the paper's vacuum C_eq = 892.07 pF with its matching network
    (golden fixture, Sec. 3), driven at 77 V from its periodic steady state: the window's
    post-processing -- Z = U_1/I_1 of the fundamental (Eq. 11), Gamma (Eq. 12), the
    period-averaged element powers (Eq. 13) and P_ref = P_forward |Gamma|^2 (Eq. 14) -- equals
    the complex-impedance solution of the same network up to the trapezoidal rule's O(h^2)
    error, which falls 16x when the substeps go from 16 to 64.  Z_ccp = -j / (w C_eq) =
    -j 13.157 ohm (Table 1's reactance) and the electrode amplitude is ~100 V as the paper
    states.  Had the circuit equations or the post-processing a wrong term, the run would
    neither stay periodic nor converge to the network solution."""
    g = _paper_vacuum_circuit()
    ref = _phasor_circuit_ii(g, g["C_eq"])
    coarse, fine = _vacuum_match_run(g, ref, 16), _vacuum_match_run(g, ref, 64)
    b = fine[-1]
    assert abs(b["z_ccp"] - fine[-2]["z_ccp"]) <= 1e-7 * abs(b["z_ccp"])  # periodic
    e16, e64 = abs(coarse[-1]["z_load"] - ref["z_load"]), abs(b["z_load"] - ref["z_load"])
    assert 12 < e16 / e64 < 20, (e16, e64)  # second order in the substep
    assert abs(b["z_ccp"] - ref["z_ccp"]) <= 1e-7 * abs(ref["z_ccp"])
    assert abs(b["z_ccp"].imag + 13.157) < 5e-4 and abs(b["z_ccp"].real) < 1e-5
    assert e64 <= 1e-4
    assert abs(b["gamma"] - ref["gamma"]) <= 1e-6
    assert abs(ref["gamma"]) < 1e-3  # the paper's matching is nearly perfect in vacuum
    for k in ("p_source", "p_rs", "p_series", "p_stray", "p_forward"):
        assert b[k] == pytest.approx(ref[k], rel=1e-6, abs=0), k
    assert abs(b["p_ccp"]) <= 1e-6 * b["p_source"]  # a capacitor takes no active power
    assert b["p_ref"] == pytest.approx(b["p_forward"] * b["gamma_abs"] ** 2, rel=1e-12, abs=0)
    # energy balance over a period: what the source delivers is dissipated in the elements
    assert b["p_source"] == pytest.approx(b["p_rs"] + b["p_series"] + b["p_stray"] + b["p_ccp"], rel=1e-6, abs=0)
    assert abs(b["u1"]) == pytest.approx(abs(ref["Ub"]), rel=1e-6, abs=0)
    assert abs(b["u1"]) == pytest.approx(g["U_electrode_amplitude"], rel=5e-3, abs=0)


def test_blocking_capacitor_charges_at_the_closed_form_rate():
    """Circuit I (Eq. 9: source, R_b, L_b and the blocking capacitor C_b in series with the
    electrode's C_eq, Sec. 3's values) with a constant net convective current I0 into the
    electrode (Eq. 8): at DC the inductor and resistor drop nothing, so the blocking capacitor
    and the electrode charge together (Q_b = -C_b U_E): the electrode's window-mean potential --
    the DC self-bias -- rises by I0 T / (C_eq + C_b) per RF period T, the loop carries the mean
    current -I0 C_b / (C_eq + C_b), and the fundamental stays periodic.  The trapezoidal rule is
    exact on this linear drift."""
    base = W.small_cylinder(n_per_species=16)
    Rb, Lb, Cb, Ceq, I0 = 0.5, 0.01e-6, 5e-9, 892.07e-12, 0.37
    wl = dataclasses.replace(with_particles(base), circuit=W.CIRCUIT_RLC, circ=(Rb, Lb, Cb, 0.0, 0.0, 0.0, 0.0, 0.0), V_src=150.0,
                             phase_src=0.0, ceq_refresh=0)
    o = orc.Oracle(wl)
    o.set_ceq(Ceq)
    o.set_circuit_state(np.zeros(6))
    o.set_conv_current(I0)
    o.set_step(0)
    o.circuit_run(wl.steps_per_rf * 12)
    a = o.circuit_diag()
    o.circuit_run(wl.steps_per_rf)
    b = o.circuit_diag()
    T = wl.steps_per_rf * wl.dt
    assert b["u_dc"] - a["u_dc"] == pytest.approx(I0 * T / (Ceq + Cb), rel=1e-9, abs=0)
    assert b["i_dc"] == pytest.approx(-I0 * Cb / (Ceq + Cb), rel=1e-9, abs=0)
    assert abs(b["u1"] - a["u1"]) <= 1e-9 * abs(b["u1"])


# ---------------------------------------------------------------- unequal weights and splitting
def test_weight_ratio_scales_deposit_and_credit_linearly():
    """A macroparticle of weight ratio w deposits w times the node weights of one of ratio 1 at
    the same place (the deposit is linear in the weight), and an absorbed one credits q w_s w."""
    base = W.small_cylinder(n_per_species=16)
    n = 2000
    rng = np.random.default_rng(3)
    r = np.sqrt(rng.uniform(0.01**2, 0.04**2, n))
    z = rng.uniform(0.003, 0.02, n)
    z0 = np.zeros(n)
    mk = lambda w: W.Particles(r, z, z0, z0, z0, z0, z0, z0, np.arange(n, dtype=np.uint64), w)
    deps = []
    for w in (None, np.full(n, 0.25)):
        o = orc.Oracle(with_particles(base, electrons=mk(w)))
        o.deposit_only()
        deps.append(o.field("dep_e"))
    np.testing.assert_allclose(deps[1], 0.25 * deps[0], rtol=1e-15, atol=0)
    assert deps[1].sum() == pytest.approx(0.25 * n, rel=1e-13, abs=0)
    # an electron of ratio 0.375 flying into the powered plate at z = 0
    e = beam(1, 0.02, 0.3 * base.dz, (0.0, 0.0, -0.5 * base.dz / base.dt))
    e.w = np.array([0.375])
    wl = dataclasses.replace(with_particles(base, electrons=e), n_gas=0.0, V_src=0.0)
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    o.particle_phase()
    s = o.scalars()
    assert s["absn_e_pow"] == 1 and s["absq_e_pow"] == pytest.approx(0.375 * wl.q[0] * wl.w[0], rel=1e-15, abs=0)


def test_splitting_halves_heavy_particles_entering_small_axial_cells():
    """The splitting rule (Sec. 2's noise fix for unequal weights): radial cell i < i_s has the
    target ratio (2i+1)/(2 i_s + 1); an electron of ratio 1 moving inward from cell 3 to cell 2
    (i_s = 8: target 5/17, twice that 10/17 < 1) becomes two halves of ratio 1/2 with identical
    state, the second with the split id; one cell further in (target 3/17, 6/17 < 1/2) each half
    splits again; at cell 0 (2/17 < 1/4) again.  Weight and deposited count are conserved at
    every step, and a particle moving outward never splits."""
    base = W.small_cylinder(n_per_species=16)
    dr, dt = base.dr, base.dt
    e = W.Particles(np.array([3.5 * dr, 5.5 * dr]), np.array([0.0127, 0.0127]), np.array([-dr / dt, dr / dt]),
                    np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2), np.array([7, 8], np.uint64),
                    np.ones(2))
    wl = dataclasses.replace(with_particles(base, electrons=e), n_gas=0.0, V_src=0.0, split_cells=8)
    o = orc.Oracle(wl)
    o.set_field("Er", np.zeros(o.n_nodes))
    o.set_field("Ez", np.zeros(o.n_nodes))
    counts, splits = [], []
    for step in range(3):
        o.set_step(step)
        o.particle_phase()
        g = o.get_particles(0)
        counts.append(len(g["id"]))
        splits.append(o.scalars()["splits_e"])
        assert g["w"].sum() == pytest.approx(2.0, rel=1e-15, abs=0)
        assert o.field("dep_e").sum() == pytest.approx(2.0, rel=1e-13, abs=0)
        inward = g["vr"] < 0
        assert np.all(g["w"][~inward] == 1.0)  # the outward electron keeps its ratio
        np.testing.assert_allclose(g["w"][inward], 0.5 ** (step + 1), rtol=0, atol=0)
        assert np.ptp(g["r"][inward]) == 0.0 and np.ptp(g["vr"][inward]) == 0.0  # halves are copies
    assert counts == [3, 5, 9] and splits == [1, 2, 4]
    # the second halves carry the split ids of their parents in the step they split
    g = o.get_particles(0)
    first = orc.split_ids(0, wl.seed, [7])[0]
    assert first in set(g["id"].tolist())


def test_radially_weighted_loading_samples_the_uniform_density():
    """Radially weighted loading (ratio (2i+1)/(2 i_s + 1) near the axis, uniform counts there)
    still samples the uniform density n0: the deposited density averaged over the inner nodes
    is n0 within a few per cent, near the axis as far out."""
    wl = W.gec_case(64, 32, 30.0, 150.0, n_per_species=400_000, split_cells=16)
    o = orc.Oracle(wl)
    o.deposit_only()
    dens = wl.w[0] * o.field("dep_e") / np.where(o.field("vnode") > 0, o.field("vnode"), np.inf)
    cell = np.asarray(wl.cell_kind).reshape(wl.nz, wl.nr)
    rows = slice(10, 20)  # the gap between the electrodes
    assert (cell[10:20, :50] == 0).all()
    near, far = dens[rows, 1:8].mean(), dens[rows, 30:50].mean()
    assert near == pytest.approx(1e15, rel=0.03, abs=0)
    assert far == pytest.approx(1e15, rel=0.03, abs=0)
    e = wl.particles[0]
    i = np.floor(e.r / wl.dr).astype(int)
    np.testing.assert_array_equal(e.w, W.radial_weight(i, 16).astype(np.float32).astype(np.float64))


# ---------------------------------------------------------------- Vahedi decomposition (Eqs. 2-4)
def _planar_two_electrodes(nr=8, nz=20, R=0.03, L=0.02, mode=W.FIELD_VAHEDI, drive=((40.0, 2e6, 0.7),)):
    """Powered plate at z = 0 (direct drive, 100 V at phase 1.1), a voltage-driven plate at
    z = L (node kind 3), free outer wall and axis, vacuum, no particles."""
    node, cell, eps = grounded_box(nr, nz, R, L, neumann_wall=True, powered_bottom=True)
    node[nz, :] = W.NODE_DRIVEN
    wl = field_only(nr, nz, R, L, node, cell, eps, V=100.0, phase=1.1)
    return dataclasses.replace(wl, drive=drive, field_mode=mode, ceq_refresh=0)


def test_vahedi_decomposition_of_a_planar_gap_is_the_closed_form():
    """Two plates, a uniform volume charge rho0 between them (node charges rho0 A_a dz, A_a the
    node's axial face area, so the discrete problem is r-independent), no chi: the unit Laplace solutions are phi_L0 = 1 - z/L (powered plate) and
    phi_L1 = z/L (driven plate), the zero-boundary Poisson solution is
    phi_P = rho0 z (L - z) / (2 eps0), and phi = phi_P + U_E phi_L0 + U_1 phi_L1 (Eq. 2) with
    U_E = 100 sin(1.1) V and U_1 = 40 sin(0.7) V; the direct solve gives the same phi."""
    nr, nz, L = 8, 20, 0.02
    rho0 = 3e-6  # C / m^3
    z = (np.arange(nz + 1) * L / nz)[:, None]
    UE, U1 = 100.0 * math.sin(1.1), 40.0 * math.sin(0.7)
    want_P = rho0 * z * (L - z) / (2 * EPS0)
    want = want_P + UE * (1 - z / L) + U1 * z / L
    phis = {}
    for mode in (W.FIELD_VAHEDI, W.FIELD_DIRECT):
        wl = _planar_two_electrodes(nr, nz, L=L, mode=mode)
        o = orc.Oracle(wl, set_particles=False)
        o.assemble()
        _, Gz = o.operator()
        dz = L / nz
        o.set_field("sigma", np.broadcast_to(rho0 * Gz[0] * dz * dz / EPS0, (nz + 1, nr + 1)))
        o.init_fields()
        phi = o.field("phi")
        np.testing.assert_allclose(phi, np.broadcast_to(want, phi.shape), rtol=0, atol=1e-9 * np.abs(want).max())
        phis[mode] = phi
        if mode == W.FIELD_VAHEDI:
            np.testing.assert_allclose(o.field("phiL0"), np.broadcast_to(1 - z / L, phi.shape), atol=1e-11)
            np.testing.assert_allclose(o.field("phiL1"), np.broadcast_to(z / L, phi.shape), atol=1e-11)
            np.testing.assert_allclose(o.field("phiP"), np.broadcast_to(want_P, phi.shape), rtol=0,
                                       atol=1e-9 * want_P.max())
    # both solves stop at the workload's relative residual (1e-10), the closed form above holds to 1e-9
    assert rel_l2(phis[W.FIELD_VAHEDI], phis[W.FIELD_DIRECT]) <= 1e-9


def test_vahedi_laplace_solutions_see_a_dielectric_layer():
    """A dielectric layer eps_r = 4 over the powered plate (rows below k): phi_L1 of the driven
    plate is the series-capacitor profile, linear in each layer with continuous D; and with two
    driven electrodes side by side (inner and outer halves of the top plate) the unit solutions
    of the three electrodes sum to 1 everywhere (superposition of the all-ones boundary)."""
    nr, nz, R, L, k, er = 12, 24, 0.03, 0.024, 9, 4.0
    wl = _planar_two_electrodes(nr, nz, R, L)
    cell = wl.cell_kind.copy()
    eps = wl.cell_eps.copy()
    cell[:k, :] = W.CELL_DIELECTRIC
    eps[:k, :] = er
    wl = dataclasses.replace(wl, cell_kind=cell, cell_eps=eps)
    o = orc.Oracle(wl, set_particles=False)
    o.init_fields()
    z = (np.arange(nz + 1) * L / nz)[:, None]
    d1, d2 = k * L / nz, (nz - k) * L / nz
    Dn = 1.0 / (d1 / er + d2)
    want = np.where(z <= d1, Dn * z / er, Dn * d1 / er + Dn * (z - d1))
    np.testing.assert_allclose(o.field("phiL1"), np.broadcast_to(want, (nz + 1, nr + 1)), atol=1e-11)
    # split the top plate into two driven electrodes
    node = wl.node_kind.copy()
    node[nz, nr // 2:] = W.NODE_DRIVEN + 1
    wl2 = dataclasses.replace(wl, node_kind=node, drive=((40.0, 2e6, 0.7), (-15.0, 1e6, 0.2)))
    o2 = orc.Oracle(wl2, set_particles=False)
    o2.init_fields()
    total = o2.field("phiL0") + o2.field("phiL1") + o2.field("phiL2")
    np.testing.assert_allclose(total, 1.0, atol=1e-10)
    assert o2.field("phiL2")[nz, nr] == 1.0 and o2.field("phiL2")[nz, 0] == 0.0


def _eq1_residual(o, phi):
    """Relative residual of Eq. 1's finite-volume form at the free nodes:
    ||sum_b G_ab (phi_a - phi_b) - Q_a|| / ||(Q + Dirichlet lift)_free||."""
    Gr, Gz = o.operator()
    q = o.field("rho")
    kind = o.kind
    Ap = np.zeros_like(phi)
    lift = np.zeros_like(phi)
    d = phi[:, :-1] - phi[:, 1:]
    Ap[:, :-1] += Gr * d
    Ap[:, 1:] -= Gr * d
    d = phi[:-1, :] - phi[1:, :]
    Ap[:-1, :] += Gz * d
    Ap[1:, :] -= Gz * d
    metal = kind != W.NODE_FREE
    pm = np.where(metal, phi, 0.0)
    lift[:, :-1] += Gr * pm[:, 1:]
    lift[:, 1:] += Gr * pm[:, :-1]
    lift[:-1, :] += Gz * pm[1:, :]
    lift[1:, :] += Gz * pm[:-1, :]
    free = ~metal
    return float(np.linalg.norm((Ap - q)[free]) / np.linalg.norm((q + lift)[free]))


def test_vahedi_laplace_parts_refresh_with_chi_once_per_window():
    """With particles (chi > 0) the Laplace parts stay the vacuum ones until the first RF window
    ends, then are re-solved with that step's chi.  phi = phi_P + sum U phi_L solves Eq. 1 only
    when the parts carry the solve's chi: the window's last step (formed with the vacuum parts)
    leaves a residual, the same step re-solved after the refresh does not."""
    wl = W.small_cylinder(n_per_species=4000)
    node = wl.node_kind.copy()
    top = node.shape[0] - 1
    node[top, :] = np.where(node[top, :] == W.NODE_GROUNDED, W.NODE_DRIVEN, node[top, :])
    wl = dataclasses.replace(wl, node_kind=node, drive=((30.0, 4e6, 0.3),), field_mode=W.FIELD_VAHEDI,
                             steps_per_rf=3, ceq_refresh=1)
    o = orc.Oracle(wl)
    o.kind = node
    o.init_fields()
    L1_vac = o.field("phiL1")
    o.step(2)
    np.testing.assert_array_equal(o.field("phiL1"), L1_vac)  # no window has ended
    o.step(1)  # the third step ends the window
    assert rel_l2(o.field("phiL1"), L1_vac) > 1e-6
    o.assemble()  # the same step's charge and chi again
    before = _eq1_residual(o, o.field("phi"))
    st, _, _ = o.field_solve()
    assert st == 0
    after = _eq1_residual(o, o.field("phi"))
    assert after <= 1e-9 < before, (after, before)
