"""Host logic of the batched sweep: the seeded Latin-hypercube design."""
import numpy as np

from paper_2310_04957_gb300 import sweep


def test_latin_hypercube_strata():
    u = sweep.latin_hypercube(64, 5, seed=4)
    assert u.shape == (64, 5)
    assert (u >= 0).all() and (u < 1).all()
    for d in range(5):
        strata = np.floor(u[:, d] * 64).astype(int)
        assert sorted(strata.tolist()) == list(range(64))  # one point per stratum
    np.testing.assert_array_equal(u, sweep.latin_hypercube(64, 5, seed=4))
    assert not np.array_equal(u, sweep.latin_hypercube(64, 5, seed=5))


def test_design_ranges_and_uneven_sizes():
    pts = sweep.design(64, seed=4)
    assert len(pts) == 64
    V = np.array([p["V"] for p in pts])
    pr = np.array([p["p_mtorr"] for p in pts])
    cm = np.array([p["cm2"] for p in pts])
    n = np.array([p["n_per_species"] for p in pts])
    assert V.min() >= 50 and V.max() < 300 and pr.min() >= 5 and pr.max() < 100
    assert cm.min() >= 100e-12 and cm.max() < 400e-12
    assert n.min() >= 200_000 and n.max() <= 4_000_000
    grids = {(p["nr"], p["nz"]) for p in pts}
    assert grids == {(g, g // 2) for g in sweep.GRID_STEPS}  # every grid size occurs
    # Latin property carries over: every eighth of the voltage range holds 8 points
    counts = np.bincount(((V - 50) / 250 * 8).astype(int), minlength=8)
    assert (counts == 8).all()
