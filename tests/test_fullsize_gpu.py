"""Parity at full size: the 512x256 GEC-like cell with 61 M particles, stepped by
the path the benchmark times (FP32 particles, multigrid-preconditioned mixed
solve, 4x4 tiles, one captured step graph).

The oracle cannot step 61 M particles in a test's time, so the comparison takes
what it can compute one by one, and properties that hold at any size:

- sampled particles: 20 000 electrons and 20 000 ions, drawn at random from the
  stored state, are pushed by the oracle alone in the node field the device's
  step started from; the device's results for the same ids (and the children
  of sampled electrons that ionize) agree within 1e-5, and every divergence is
  a branch flip proven by the oracle's decision margins;
- every stored particle (all 61 M) lies in the cell of its bin, ids are
  unique, and each species' count after the step is the count before, less
  the absorbed, plus the born;
- each species' deposit sums to its particle count (integer fixed point);
- the field solve of the step, repeated by the oracle in FP64 on the device's
  own deposits, surface charge and circuit state: phi and E_z within 1e-8.
"""
import numpy as np
import pytest

from gpu_common import pic
from oracle import orc
from paper_2310_04957_gb300 import workloads as W
from parity_tools import _particles, by_id, classify, phi_err, rel_l2

pytestmark = pytest.mark.gpu

N_SAMPLE = 20_000
FP32, MG = 0, 3
TILE = (4, 4)  # the tile the benchmark's autotuner picks for this cell


def subset(g, ids):
    m = np.isin(g["id"], ids)
    return {k: (v[m] if v is not None else None) for k, v in g.items()}


@pytest.fixture(scope="module")
def fullsize():
    P = pic()
    wl = W.PRESETS["c3"]()
    d = P.Discharge(wl, precision=FP32, solver=MG, tile=TILE)
    d.start()
    d.step(3)
    return P, wl, d


def test_full_size_step_against_the_oracle(fullsize):
    P, wl, d = fullsize
    rng = np.random.default_rng(2310)
    sc0 = d.scalars()
    k_step, ceq_solve = int(sc0["step"]), sc0["C_eq"]
    assert k_step % wl.steps_per_rf != 0 and (k_step + 1) % wl.steps_per_rf != 0  # no window end in this step
    E_pre = (d.field("Er"), d.field("Ez"))
    n_pre = [d.count(s) for s in (0, 1)]
    pre = []
    for s in (0, 1):
        g = d.get_particles(s)
        pick = np.sort(rng.choice(len(g["id"]), N_SAMPLE, replace=False))
        pre.append(by_id({k: (v[pick] if v is not None else None) for k, v in g.items()}))
        del g
    # the benchmark's step: one graph launch
    d.step(1)
    sd = d.scalars()
    assert sd["step"] == k_step + 1 and sd["pcg_status"] == 0 and d.status() == 0
    kids = orc.child_ids(k_step, wl.seed, pre[0]["id"])  # children of the sampled electrons
    keep = [np.concatenate([pre[0]["id"], kids[:, 0]]), np.concatenate([pre[1]["id"], kids[:, 1]])]
    post_d, n_post = [], []
    for s in (0, 1):
        g = d.get_particles(s)
        n_post.append(len(g["id"]))
        # properties of the whole store: each particle lies in its stored cell.  The
        # position read back is (i + f) dr with the FP32 offset f in [0, 1 - 2^-24];
        # f = 0 exactly (a particle on the cell's lower face) can read back an ulp
        # below i, so the lower bound allows 1e-9 of a cell
        i, j = g["cell"] % wl.nr, g["cell"] // wl.nr
        x, y = g["r"] / wl.dr - i, g["z"] / wl.dz - j
        assert x.min() >= -1e-9 and x.max() < 1.0, (x.min(), x.max())
        assert y.min() >= -1e-9 and y.max() < 1.0, (y.min(), y.max())
        assert len(np.unique(g["id"])) == len(g["id"])
        post_d.append(subset(g, keep[s]))
        del g
    for s, sp in enumerate(("e", "i")):
        absorbed = sum(sd[f"absn_{sp}_{k}"] for k in ("pow", "gnd", "surf"))
        assert n_post[s] == n_pre[s] - absorbed + sd[f"born_{sp}"], (s, n_pre[s], n_post[s])
    assert d.field("dep_e").sum() == pytest.approx(n_post[0], rel=1e-12, abs=0)
    assert d.field("dep_i").sum() == pytest.approx(n_post[1], rel=1e-12, abs=0)

    # the sampled particles, pushed by the oracle alone in the same field
    o = orc.Oracle(wl, capacity=(4 * N_SAMPLE, 4 * N_SAMPLE), set_particles=False)
    for s in (0, 1):
        o.set_particles(s, _particles(pre[s], np.arange(N_SAMPLE)))
    o.set_field("Er", E_pre[0])
    o.set_field("Ez", E_pre[1])
    o.set_step(k_step)
    o.particle_phase()
    post_o = [o.get_particles(s) for s in (0, 1)]
    flipped, st = classify(wl, E_pre, k_step, pre, post_d, post_o, 1e-5)
    assert st["max_dpos"] <= 1e-5 and st["max_dvel"] <= 1e-5, st
    assert st["n"] <= 1e-4 * 2 * N_SAMPLE + 2, st
    assert sum(len(p["id"]) for p in post_d) >= 1.9 * N_SAMPLE  # the sample survived the step on the device

    # the step's field solve, repeated by the oracle on the device's own charge
    of = orc.Oracle(wl, capacity=(16, 16), set_particles=False)
    of.init_fields()
    for name in ("dep_e", "dep_i", "sigma"):
        of.set_field(name, d.field(name))
    of.set_ceq(ceq_solve)
    of.set_circuit_state(np.array([sd[f"y{k}"] for k in range(6)]))
    of.assemble()
    st_o, _, rel_o = of.field_solve()
    assert st_o == 0 and rel_o <= wl.pcg_tol
    assert sd["pcg_relres"] <= wl.pcg_tol
    assert rel_l2(d.field("rho"), of.field("rho")) <= 1e-13
    assert rel_l2(d.field("chi"), of.field("chi")) <= 1e-13
    assert phi_err(d.field("phi"), of.field("phi"), wl.V_src) <= 1e-8
    assert rel_l2(d.field("Ez"), of.field("Ez")) <= 1e-8
