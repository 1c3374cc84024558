"""The seeded input generator (paper_2310_04957_gb300/workloads.py) against the
recipe it states for the initial population: positions uniform in volume over
the plasma cells, kept a margin from the cell faces and exact in FP32;
Maxwellian velocities at the stated temperatures; zero initial accelerations;
ions placed on their electrons (zero initial charge); the macro weight
n0 V_plasma / N; unique ids; the same arrays for the same preset and seed."""
import math

import numpy as np

from paper_2310_04957_gb300 import workloads as W

N = 200_000


def _cells(wl, P):
    i = np.floor(P.r / wl.dr).astype(np.int64)
    j = np.floor(P.z / wl.dz).astype(np.int64)
    return i, j


def test_positions_fill_plasma_cells_uniformly_in_volume():
    wl = W.small_cylinder(N)
    el = wl.particles[0]
    i, j = _cells(wl, el)
    assert (wl.cell_kind[j, i] == W.CELL_PLASMA).all()
    # FP32-exact positions, a relative margin of 1e-3 from the faces (up to that rounding)
    assert np.array_equal(el.r, el.r.astype(np.float32).astype(np.float64))
    assert np.array_equal(el.z, el.z.astype(np.float32).astype(np.float64))
    fr = (el.r**2 - (i * wl.dr) ** 2) / (((i + 1) * wl.dr) ** 2 - (i * wl.dr) ** 2)  # r^2 fraction in the annulus
    fz = el.z / wl.dz - j
    assert fr.min() > 0.9e-3 and fr.max() < 1 - 0.9e-3
    assert fz.min() > 0.9e-3 and fz.max() < 1 - 0.9e-3
    # uniform in r^2 and z inside the cell: means 1/2 within 6 standard errors
    se = math.sqrt(1.0 / 12.0 / N)
    assert abs(fr.mean() - 0.5) < 6 * se and abs(fz.mean() - 0.5) < 6 * se
    # counts per cell proportional to the cell's volume, pi dr^2 dz (2i + 1): chi-square
    nz, nr = wl.cell_kind.shape
    vol = ((wl.cell_kind == W.CELL_PLASMA) * (2.0 * np.arange(nr) + 1.0)[None, :]).ravel()
    expect = N * vol / vol.sum()
    got = np.bincount(j * nr + i, minlength=nr * nz).astype(np.float64)
    m = expect > 0
    chi2 = float((((got - expect) ** 2)[m] / expect[m]).sum())
    dof = int(m.sum()) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)
    assert got[~m].sum() == 0


def test_velocities_are_maxwellian_at_the_stated_temperatures():
    wl = W.small_cylinder(N)
    for P, T_eV, mass in ((wl.particles[0], 2.0, W.ELECTRON_MASS), (wl.particles[1], 0.026, W.ARGON_MASS)):
        v = np.stack([P.vr, P.vt, P.vz])
        sig = math.sqrt(T_eV * W.ELEMENTARY_CHARGE / mass)
        # per-component mean zero and variance sig^2; temperature from <v^2> within 1 %
        assert np.abs(v.mean(axis=1)).max() < 6 * sig / math.sqrt(N)
        assert np.allclose(v.var(axis=1), sig**2, rtol=0.02)
        T = mass * (v**2).sum(axis=0).mean() / (3 * W.ELEMENTARY_CHARGE)
        assert abs(T / T_eV - 1) < 0.01
        assert not P.ar.any() and not P.at.any() and not P.az.any()


def test_ions_sit_on_their_electrons_and_the_weight_is_n0_v_over_n():
    wl = W.small_cylinder(N)
    el, io = wl.particles
    assert np.array_equal(io.r, el.r) and np.array_equal(io.z, el.z)
    for P in (el, io):
        assert np.array_equal(P.id, np.arange(N, dtype=np.uint64))
        assert P.w is None
    vp = W.plasma_volume(wl.cell_kind, wl.dr, wl.dz)
    assert wl.w[0] == wl.w[1] == 1e15 * vp / N
    assert wl.q == (-W.ELEMENTARY_CHARGE, W.ELEMENTARY_CHARGE)


def test_same_preset_same_arrays_other_seed_other_arrays():
    a, b = W.small_cylinder(5_000), W.small_cylinder(5_000)
    for Pa, Pb in zip(a.particles, b.particles):
        for k in ("r", "z", "vr", "vt", "vz", "id"):
            assert np.array_equal(getattr(Pa, k), getattr(Pb, k))
    c = W.gec_case(64, 32, 30.0, 150.0, n_per_species=5_000, seed_index=40)
    d = W.gec_case(64, 32, 30.0, 150.0, n_per_species=5_000, seed_index=41)
    assert c.seed != d.seed and not np.array_equal(c.particles[0].r, d.particles[0].r)
