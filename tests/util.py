"""Small workload builders and comparison helpers shared by the tests."""
import dataclasses

import numpy as np

from paper_2310_04957_gb300 import workloads as W


def with_particles(wl, electrons=None, ions=None):
    e = electrons if electrons is not None else W.Particles(*(np.zeros(0) for _ in range(8)), np.zeros(0, np.uint64))
    i = ions if ions is not None else W.Particles(*(np.zeros(0) for _ in range(8)), np.zeros(0, np.uint64))
    cap = (2 * (e.n + i.n) + 1024,) * 2  # room for births
    return dataclasses.replace(wl, particles=(e, i), capacity=cap)


def beam(n, r, z, v, start_id=0):
    """n particles at (r,z) with velocity v = (vr, vt, vz)."""
    o = np.ones(n)
    zeros = np.zeros(n)
    return W.Particles(r * o, z * o, v[0] * o, v[1] * o, v[2] * o, zeros.copy(), zeros.copy(), zeros.copy(),
                       np.arange(start_id, start_id + n, dtype=np.uint64))


def grounded_box(nr, nz, R, Z, neumann_wall=False, powered_bottom=False):
    """All outer faces grounded (or the r = R wall free), axis free."""
    node = np.zeros((nz + 1, nr + 1), np.int8)
    node[0, :] = W.NODE_POWERED if powered_bottom else W.NODE_GROUNDED
    node[nz, :] = W.NODE_GROUNDED
    if not neumann_wall:
        node[:, nr] = W.NODE_GROUNDED
        if powered_bottom:
            node[0, nr] = W.NODE_GROUNDED
    cell = np.zeros((nz, nr), np.int8)
    eps = np.ones((nz, nr))
    return node, cell, eps


def field_only(nr, nz, R, Z, node, cell, eps, V=0.0, phase=0.0):
    wl = W.small_cylinder(n_per_species=16)
    wl = dataclasses.replace(wl, nr=nr, nz=nz, dr=R / nr, dz=Z / nz, node_kind=node, cell_kind=cell, cell_eps=eps,
                             V_src=V, phase_src=phase)
    return with_particles(wl)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
