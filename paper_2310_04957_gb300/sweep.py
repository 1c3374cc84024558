"""Parameter sweep of independent discharges and the particle-tile autotuner.

The sweep stands in for a matching-network / operating-point study of the
paper's GEC-like cell (arXiv:2310.04957, Sec. 2 and the matching study of its
Sec. 3): source amplitude, gas pressure and series matching capacitor are
drawn on a seeded Latin hypercube, with grids and particle counts that differ
from discharge to discharge.  Everything here is host logic (the design, the
workload list, the tile choice); the stepping runs in the library, either one
discharge at a time (pic_step) or all together (pic_batch_step).
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

# ranges of the sweep
V_RANGE = (50.0, 300.0)          # source amplitude, V
P_RANGE = (5.0, 100.0)           # pressure, mTorr
CM2_RANGE = (100e-12, 400e-12)   # series matching capacitor, F
GRID_STEPS = (64, 96, 128, 160, 192, 224, 256)  # nr; nz = nr / 2
N_RANGE = (200_000, 4_000_000)   # macroparticles per species

# particle tiles the autotuner tries (cells per CTA tile: tile_r x tile_z)
TILE_CANDIDATES = ((2, 2), (4, 2), (4, 4), (8, 4), (8, 8))


def latin_hypercube(n, dims, seed):
    """n points in [0, 1)^dims: in every dimension each of the n strata
    [k/n, (k+1)/n) holds exactly one point (random permutation + jitter)."""
    rng = np.random.default_rng(seed)
    u = np.empty((n, dims))
    for d in range(dims):
        u[:, d] = (rng.permutation(n) + rng.random(n)) / n
    return u


def design(n=64, seed=4):
    """The sweep's operating points: list of dicts (V, p_mtorr, cm2, nr, nz, n_per_species)."""
    u = latin_hypercube(n, 5, seed)
    out = []
    for k in range(n):
        nr = GRID_STEPS[min(len(GRID_STEPS) - 1, int(u[k, 3] * len(GRID_STEPS)))]
        npart = int(round((N_RANGE[0] + (N_RANGE[1] - N_RANGE[0]) * u[k, 4]) / 1000.0)) * 1000
        out.append(dict(V=V_RANGE[0] + (V_RANGE[1] - V_RANGE[0]) * u[k, 0],
                        p_mtorr=P_RANGE[0] + (P_RANGE[1] - P_RANGE[0]) * u[k, 1],
                        cm2=CM2_RANGE[0] + (CM2_RANGE[1] - CM2_RANGE[0]) * u[k, 2],
                        nr=nr, nz=nr // 2, n_per_species=npart))
    return out


def workloads(points, scale=1.0, seed_base=100):
    """Workloads of the design points (particle counts times `scale`)."""
    return [W.gec_case(p["nr"], p["nz"], p["p_mtorr"], p["V"], cm2=p["cm2"],
                       n_per_species=max(1000, int(p["n_per_species"] * scale)), seed_index=seed_base + k)
            for k, p in enumerate(points)]


def shard(weights, rank, world):
    """Indices of the items rank `rank` of `world` takes: items dealt largest
    first, each to the rank with the least weight so far (ties to the lowest
    rank).  The shares are disjoint, cover every item and are balanced."""
    order = sorted(range(len(weights)), key=lambda k: (-weights[k], k))
    load = [0] * world
    mine = []
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += weights[k]
        if r == rank:
            mine.append(k)
    return sorted(mine)


def tile_class(wl):
    """Discharges of one grid size share a tile choice."""
    return (wl.nr, wl.nz)


def autotune_tiles(wls, candidates=TILE_CANDIDATES, reps=3, precision=0):
    """For each grid class, time the particle phase of one representative
    discharge (the one with the median particle count) with every candidate
    tile and keep the fastest.  Returns ({class: tile}, {class: {tile: ms}})."""
    import torch

    from . import pic

    by_class = {}
    for wl in wls:
        by_class.setdefault(tile_class(wl), []).append(wl)
    choice, timings = {}, {}
    for cls, members in sorted(by_class.items()):
        members = sorted(members, key=lambda w: w.particles[0].n)
        wl = members[len(members) // 2]
        t_ms = {}
        for tile in candidates:
            d = pic.Discharge(wl, precision=precision, tile=tile)
            d.start()
            d.particle_phase()  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                d.particle_phase()
            e1.record()
            torch.cuda.synchronize()
            t_ms[tile] = e0.elapsed_time(e1) / reps
            d.close()
        choice[cls] = min(t_ms, key=t_ms.get)
        timings[cls] = t_ms
    return choice, timings
