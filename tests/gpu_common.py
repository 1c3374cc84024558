"""Helpers for the GPU parity tests: identical start states for the CUDA path and
the oracle, and per-particle comparison by id."""
import dataclasses

import numpy as np

from oracle import orc
from paper_2310_04957_gb300 import workloads as W


def pic():
    from paper_2310_04957_gb300 import build, pic as P

    build.build()
    return P


def particles_from(g):
    return W.Particles(g["r"], g["z"], g["vr"], g["vt"], g["vz"], g["ar"], g["at"], g["az"], g["id"], g.get("w"))


def make_pair(wl, precision, **kw):
    """CUDA discharge + oracle starting from the same state: the oracle takes the
    device's stored representation (cell-relative FP32/FP64 position read back as
    FP64), so both start from identical numbers."""
    P = pic()
    d = P.Discharge(wl, precision=precision, **kw)
    o = orc.Oracle(wl, set_particles=False)
    for s in (0, 1):
        o.set_particles(s, particles_from(d.get_particles(s)))
    return d, o


def random_field(wl, seed, scale=2e4, precision=0):
    """Seeded node E field (V/m), rounded to FP32 for the FP32 path."""
    rng = np.random.default_rng(seed)
    n = (wl.nr + 1) * (wl.nz + 1)
    er = rng.normal(0, scale, n)
    ez = rng.normal(0, scale, n) + scale
    er.reshape(wl.nz + 1, wl.nr + 1)[:, 0] = 0.0
    if precision == 0:
        er = er.astype(np.float32).astype(np.float64)
        ez = ez.astype(np.float32).astype(np.float64)
    return er, ez


def by_id(g):
    order = np.argsort(g["id"], kind="stable")
    return {k: v[order] for k, v in g.items()}


def compare_particles(gd, go, rtol):
    """Match particles by id; return (n_common, n_only_device, n_only_oracle, n_bad, detail)
    where bad = position or velocity differing by more than rtol (relative to the particle's
    radius-scale / speed)."""
    a, b = by_id(gd), by_id(go)
    common, ia, ib = np.intersect1d(a["id"], b["id"], assume_unique=True, return_indices=True)
    pos_scale = np.maximum(np.hypot(b["r"][ib], b["z"][ib]), 1e-3)
    dpos = np.hypot(a["r"][ia] - b["r"][ib], a["z"][ia] - b["z"][ib]) / pos_scale
    va = np.stack([a["vr"][ia], a["vt"][ia], a["vz"][ia]])
    vb = np.stack([b["vr"][ib], b["vt"][ib], b["vz"][ib]])
    dvel = np.linalg.norm(va - vb, axis=0) / np.maximum(np.linalg.norm(vb, axis=0), 1.0)
    bad = (dpos > rtol) | (dvel > rtol)
    return dict(common=len(common), only_dev=len(a["id"]) - len(common), only_orc=len(b["id"]) - len(common),
                bad=int(bad.sum()), dpos_max=float(dpos[~bad].max(initial=0)), dvel_max=float(dvel[~bad].max(initial=0)),
                ids_bad=common[bad])


def small(n=20_000, **kw):
    wl = W.small_cylinder(n_per_species=n)
    return dataclasses.replace(wl, **kw) if kw else wl
