"""Seeded synthetic workloads for the r-z PIC/MCC discharge.

This module builds the *inputs* of a run and nothing else: the reactor
geometry rasterised onto the grid, the gas and species parameters, the
external-circuit parameters, tabulated synthetic cross sections, and the
initial particle population.  It holds none of the method's arithmetic (no
push, collision, deposit, field or circuit step); both the CUDA library and
the CPU oracle receive exactly these arrays.

The geometries stand in for the GEC reference cell of arXiv:2310.04957
(Sec. 2, Fig. 1: powered electrode, grounded shield and wall, dielectric
insulator, 2.54 cm gap).  The paper's exact drawing and its argon cross
sections are not available, so the shapes below are GEC-like rectangles and
the cross sections are analytic forms with argon's thresholds (11.5 eV
excitation, 15.76 eV ionization); see the design notes for the recipe.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Physical constants used to *define inputs* (masses, gas density, thermal speeds).
ELEMENTARY_CHARGE = 1.602176634e-19
ELECTRON_MASS = 9.1093837015e-31
ATOMIC_MASS_UNIT = 1.66053906660e-27
ARGON_MASS = 39.948 * ATOMIC_MASS_UNIT
BOLTZMANN = 1.380649e-23
MILLITORR = 0.13332236842105263  # Pa

NODE_FREE, NODE_POWERED, NODE_GROUNDED = 0, 1, 2
NODE_DRIVEN = 3  # first voltage-driven electrode (3, 4, 5)
FIELD_DIRECT, FIELD_VAHEDI = 0, 1
CELL_PLASMA, CELL_POWERED, CELL_GROUNDED, CELL_DIELECTRIC = 0, 1, 2, 3
CIRCUIT_DIRECT, CIRCUIT_RLC, CIRCUIT_IMN = 0, 1, 2
SEED_BASE = 0x5EED0000

N_XS = 1000
XS_EMIN, XS_EMAX = 1e-3, 1e3
THR_EXC, THR_ION = 11.5, 15.76
B_EJECT = 10.0


@dataclasses.dataclass
class Particles:
    """Structure of arrays of one species (FP64 copies of the initial state)."""

    r: np.ndarray
    z: np.ndarray
    vr: np.ndarray
    vt: np.ndarray
    vz: np.ndarray
    ar: np.ndarray
    at: np.ndarray
    az: np.ndarray
    id: np.ndarray
    w: np.ndarray = None  # weight ratios in (0, 1] (macro weight w * Workload.w); None: all 1

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    def take(self, idx) -> "Particles":
        return Particles(*(None if getattr(self, f.name) is None else getattr(self, f.name)[idx]
                           for f in dataclasses.fields(self)))


@dataclasses.dataclass
class Workload:
    name: str
    nr: int
    nz: int
    dr: float
    dz: float
    node_kind: np.ndarray  # int8 [(nz+1), (nr+1)]
    cell_kind: np.ndarray  # int8 [nz, nr]
    cell_eps: np.ndarray  # float64 [nz, nr]
    dt: float
    n_gas: float
    T_gas: float
    m_gas: float
    q: tuple
    m: tuple
    w: tuple
    xs_energy: np.ndarray  # float64 [N_XS]
    xs_sigma: np.ndarray  # float64 [5, N_XS]
    thr_ex: float
    thr_iz: float
    B_ej: float
    circuit: int
    circ: tuple  # 8 values
    V_src: float
    f_src: float
    phase_src: float
    n_sub: int
    steps_per_rf: int
    pcg_tol: float
    pcg_maxit: int
    ceq_refresh: int
    seed: int
    particles: tuple  # (electrons, ions)
    capacity: tuple
    split_cells: int = 0  # particle splitting in the first split_cells radial cells (0: off)
    drive: tuple = ()  # voltage-driven electrodes (node kinds 3, 4, 5): (V, f, phase) each, V sin(2 pi f t + phase)
    field_mode: int = 0  # FIELD_DIRECT or FIELD_VAHEDI

    @property
    def n_nodes(self) -> int:
        return (self.nr + 1) * (self.nz + 1)

    @property
    def weighted(self) -> bool:
        """Particles carry weight ratios: splitting is on or a species has ratios."""
        return self.split_cells > 0 or any(p.w is not None for p in self.particles)


# --------------------------------------------------------------------------
# Cross sections (synthetic, analytic; m^2 vs eV).  Argon's real data are not
# in this environment; these forms keep the thresholds and rough magnitudes.
# --------------------------------------------------------------------------
def xs_table(n: int = N_XS):
    """Log-spaced energy grid and the five synthetic cross sections.

    Rows: e-Ar elastic, e-Ar excitation (11.5 eV), e-Ar ionization (15.76 eV),
    Ar+-Ar isotropic elastic, Ar+-Ar charge exchange.
    """
    k = np.arange(n, dtype=np.float64)
    E = 10.0 ** (-3.0 + 6.0 * k / (n - 1))
    x = E / 10.0
    el = 1e-20 * (1.0 + 15.0 * x / (1.0 + x)) / (1.0 + E / 200.0)
    ex = np.where(E > THR_EXC, 1.5e-20 * math.e * np.log(np.maximum(E / THR_EXC, 1.0)) / (E / THR_EXC), 0.0)
    iz = np.where(E > THR_ION, 3.0e-20 * math.e * np.log(np.maximum(E / THR_ION, 1.0)) / (E / THR_ION), 0.0)
    iso = 2e-19 / np.sqrt(E + 0.01)
    cx = 4e-19 * (1.0 - 0.07 * np.log(E))
    return E, np.stack([el, ex, iz, iso, cx]).astype(np.float64)


# --------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------
def _paint_nodes(kind, i0, i1, j0, j1, value):
    kind[j0 : j1 + 1, i0 : i1 + 1] = value


def _paint_cells(kind, i0, i1, j0, j1, value):
    """Cells whose four corners lie in node rectangle [i0,i1] x [j0,j1]."""
    if i1 > i0 and j1 > j0:
        kind[j0:j1, i0:i1] = value


def cylinder_geometry(nr, nz, R, Z):
    """Planar powered electrode at z = 0, grounded plate at z = Z and wall at r = R."""
    node = np.zeros((nz + 1, nr + 1), np.int8)
    node[0, :nr] = NODE_POWERED
    node[0, nr] = NODE_GROUNDED  # the corner shared with the wall is grounded
    node[nz, :] = NODE_GROUNDED
    node[:, nr] = NODE_GROUNDED
    cell = np.zeros((nz, nr), np.int8)
    eps = np.ones((nz, nr), np.float64)
    return node, cell, eps


def gec_geometry(nr, nz, R=0.10, Z=0.06, eps_r=4.0):
    """GEC-cell-like chamber snapped to nodes.

    Powered electrode r <= 5.1 cm, 0 <= z <= 1.5 cm (its z = 0 face is the
    domain boundary); dielectric ring 5.1-5.2 cm (eps_r = 4); grounded shield
    5.2-5.5 cm; grounded upper electrode r <= 5.5 cm, 4.04 <= z <= 6 cm
    (2.54 cm gap); grounded chamber bottom for r >= 5.2 cm, top and outer
    wall.  The domain's z = 0 face under the dielectric ring is a free
    (symmetry) boundary.  Rectangles do not overlap, so no node is both
    powered and grounded.
    """
    dr, dz = R / nr, Z / nz
    ip = int(round(0.051 / dr))
    idl = int(round(0.052 / dr))
    ish = int(round(0.055 / dr))
    je = int(round(0.015 / dz))
    jt = int(round(0.0404 / dz))
    node = np.zeros((nz + 1, nr + 1), np.int8)
    cell = np.zeros((nz, nr), np.int8)
    eps = np.ones((nz, nr), np.float64)
    # powered electrode
    _paint_nodes(node, 0, ip, 0, je, NODE_POWERED)
    _paint_cells(cell, 0, ip, 0, je, CELL_POWERED)
    # dielectric ring
    cell[0:je, ip:idl] = CELL_DIELECTRIC
    eps[0:je, ip:idl] = eps_r
    # grounded shield, upper electrode, chamber bottom, top, outer wall
    _paint_nodes(node, idl, ish, 0, je, NODE_GROUNDED)
    _paint_cells(cell, idl, ish, 0, je, CELL_GROUNDED)
    _paint_nodes(node, 0, ish, jt, nz, NODE_GROUNDED)
    _paint_cells(cell, 0, ish, jt, nz, CELL_GROUNDED)
    node[0, idl:] = NODE_GROUNDED
    node[nz, :] = NODE_GROUNDED
    node[:, nr] = NODE_GROUNDED
    return node, cell, eps


def plasma_volume(cell_kind, dr, dz):
    nz, nr = cell_kind.shape
    i = np.arange(nr)
    vol_row = math.pi * ((i + 1) ** 2 - i**2) * dr * dr * dz
    return float(((cell_kind == CELL_PLASMA) * vol_row[None, :]).sum())


# --------------------------------------------------------------------------
# Particle loading: uniform in volume over plasma cells, Maxwellian velocities
# --------------------------------------------------------------------------
def radial_weight(i, split_cells):
    """Weight ratio of a particle loaded in radial cell i: (2i+1)/(2 i_s + 1), the
    cell's volume relative to that of cell i_s, within the first i_s = split_cells
    cells, and 1 beyond (the target the splitting rule keeps particles near)."""
    i = np.asarray(i)
    return np.where(i < split_cells, (2.0 * i + 1.0) / (2.0 * split_cells + 1.0), 1.0)


def load_particles(cell_kind, dr, dz, n, T_eV, mass, rng, co_located=None, edge_margin=1e-3, split_cells=0):
    """n particles over the plasma cells, uniform in volume (in density).

    A cell is picked with probability proportional to its volume divided by its
    weight ratio (radial_weight; 1 everywhere when split_cells is 0), so each
    cell's total weight is proportional to its volume; inside it r^2 is uniform
    in [r_i^2, r_{i+1}^2] and z uniform, kept a relative `edge_margin` away from
    the cell faces so that FP32 and FP64 agree on the containing cell.  If
    `co_located` is given the positions and ratios are copied from it (ions
    placed on their electrons, so the initial charge density is zero).
    """
    nz, nr = cell_kind.shape
    w = None
    if co_located is not None:
        r, z = co_located.r.copy(), co_located.z.copy()
        w = None if co_located.w is None else co_located.w.copy()
    else:
        i = np.arange(nr)
        vol = ((cell_kind == CELL_PLASMA) * ((((i + 1) ** 2 - i**2).astype(np.float64)) /
                                               radial_weight(i, split_cells))[None, :]).ravel()
        p = vol / vol.sum()
        cells = rng.choice(nr * nz, size=n, p=p)
        ci, cj = cells % nr, cells // nr
        u1 = edge_margin + (1 - 2 * edge_margin) * rng.random(n)
        u2 = edge_margin + (1 - 2 * edge_margin) * rng.random(n)
        r = np.sqrt((ci * dr) ** 2 + u1 * (((ci + 1) * dr) ** 2 - (ci * dr) ** 2))
        z = (cj + u2) * dz
        r = r.astype(np.float32).astype(np.float64)
        z = z.astype(np.float32).astype(np.float64)
        if split_cells > 0:
            w = radial_weight(ci, split_cells).astype(np.float32).astype(np.float64)
    sig = math.sqrt(T_eV * ELEMENTARY_CHARGE / mass)
    v = (sig * rng.standard_normal((3, n))).astype(np.float32).astype(np.float64)
    zeros = np.zeros(n)
    return Particles(r, z, v[0], v[1], v[2], zeros.copy(), zeros.copy(), zeros.copy(), np.arange(n, dtype=np.uint64),
                     w)


# --------------------------------------------------------------------------
# Presets
# --------------------------------------------------------------------------
F_RF = 13.56e6


def _make(name, nr, nz, R, Z, geometry, pressure_mtorr, n_per_species, steps_per_rf, circuit, circ, V_src,
          seed_index, n0=1e15, Te=2.0, Ti=0.026, T_gas=300.0, capacity_factor=1.5, n_particles_override=None,
          split_cells=0):
    dr, dz = R / nr, Z / nz
    if geometry == "cylinder":
        node, cell, eps = cylinder_geometry(nr, nz, R, Z)
    else:
        node, cell, eps = gec_geometry(nr, nz, R, Z)
    n = n_per_species if n_particles_override is None else n_particles_override
    seed = SEED_BASE + seed_index
    rng = np.random.default_rng(seed)
    vp = plasma_volume(cell, dr, dz)
    el = load_particles(cell, dr, dz, n, Te, ELECTRON_MASS, rng, split_cells=split_cells)
    io = load_particles(cell, dr, dz, n, Ti, ARGON_MASS, rng, co_located=el)
    w = n0 * vp / (n if el.w is None else float(el.w.sum()))  # macro weight of ratio 1
    E, sig = xs_table()
    cap = int(capacity_factor * n) + 4096
    return Workload(
        name=name, nr=nr, nz=nz, dr=dr, dz=dz, node_kind=node, cell_kind=cell, cell_eps=eps,
        dt=1.0 / F_RF / steps_per_rf, n_gas=pressure_mtorr * MILLITORR / (BOLTZMANN * T_gas), T_gas=T_gas,
        m_gas=ARGON_MASS, q=(-ELEMENTARY_CHARGE, ELEMENTARY_CHARGE), m=(ELECTRON_MASS, ARGON_MASS), w=(w, w),
        xs_energy=E, xs_sigma=sig, thr_ex=THR_EXC, thr_iz=THR_ION, B_ej=B_EJECT, circuit=circuit,
        circ=tuple(circ) + (0.0,) * (8 - len(circ)), V_src=V_src, f_src=F_RF, phase_src=0.0, n_sub=16,
        steps_per_rf=steps_per_rf, pcg_tol=1e-10, pcg_maxit=20000, ceq_refresh=1, seed=seed & 0xFFFFFFFF,
        particles=(el, io), capacity=(cap, cap), split_cells=split_cells)


# L-network of the 150 V GEC-like case: Rs, Cm1 (shunt), Lm, Cm2 (series), Rm, Cstray, Rstray, Lstray.
IMN_GEC = (50.0, 500e-12, 1e-6, 200e-12, 0.5, 10e-12, 0.5, 10e-9)


def small_cylinder(n_per_species=50_000, **kw):
    """32x32 cylinder, 100 V direct drive at 13.56 MHz, 100 mTorr, dt = T_RF/400."""
    return _make("cylinder-32x32-100k", 32, 32, 0.051, 0.0254, "cylinder", 100.0, 50_000, 400,
                 CIRCUIT_DIRECT, (), 100.0, 0, n_particles_override=n_per_species, **kw)


def gec_256(n_per_species=4_000_000, **kw):
    """256x128 GEC-like cell, 10 mTorr, 150 V through the L-network, dt = T_RF/200."""
    return _make("gec-256x128-8M", 256, 128, 0.10, 0.06, "gec", 10.0, 4_000_000, 200,
                 CIRCUIT_IMN, IMN_GEC, 150.0, 1, n_particles_override=n_per_species, **kw)


def gec_512(n_per_species=32_000_000, **kw):
    """512x256 GEC-like cell, 30 mTorr, 150 V through the L-network, dt = T_RF/200."""
    return _make("gec-512x256-64M", 512, 256, 0.10, 0.06, "gec", 30.0, 32_000_000, 200,
                 CIRCUIT_IMN, IMN_GEC, 150.0, 2, n_particles_override=n_per_species, **kw)


def gec_case(nr, nz, pressure_mtorr, V_src, cm2=200e-12, n_per_species=1_000_000, seed_index=16, name=None,
             split_cells=0):
    """GEC-like cell on an nr x nz grid at a given pressure, source amplitude and
    series matching capacitor (the L-network of IMN_GEC otherwise); split_cells
    > 0 loads radially weighted particles and enables splitting."""
    circ = list(IMN_GEC)
    circ[3] = cm2
    nm = name or f"gec-{nr}x{nz}-{pressure_mtorr:g}mT-{V_src:g}V"
    return _make(nm, nr, nz, 0.10, 0.06, "gec", pressure_mtorr, n_per_species, 200, CIRCUIT_IMN, tuple(circ), V_src,
                 seed_index, n_particles_override=n_per_species, split_cells=split_cells)


PRESETS = {"c1": small_cylinder, "c2": gec_256, "c3": gec_512}
