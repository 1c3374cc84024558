"""Checkpoint and resume (pic_save / pic_load) through the C ABI: k steps,
save, k more steps equals load + k steps, bit for bit, in FP64 and FP32, on
the GEC-like cell with the matching network.  The span crosses RF-window ends
(C_eq refresh) and a rebuild of the multigrid hierarchy, so the state that
carries over between steps (circuit, C_eq, surface charge, window sums,
multigrid hierarchy, particle store with its overflow region) is all covered.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import pic
from parity_tools import by_id
from paper_2310_04957_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "Er", "Ez", "chi", "dep_e", "dep_i", "sigma", "rho", "ne_avg", "ni_avg")


def snapshot(d):
    out = {f"p{s}": by_id(d.get_particles(s)) for s in (0, 1)}
    for f in FIELDS:
        out[f] = d.field(f)
    out["scalars"] = d.scalars()
    out["store"] = d.store_stats()
    return out


@pytest.mark.parametrize("precision,split", [(1, 0), (0, 0), (0, 8)], ids=["fp64", "fp32", "fp32-weighted"])
def test_save_load_continues_bit_for_bit(precision, split, tmp_path):
    P = pic()
    wl = dataclasses.replace(W.gec_case(128, 64, 30.0, 150.0, n_per_species=100_000, seed_index=22,
                                        split_cells=split),
                             steps_per_rf=5, phase_src=0.4)
    d = P.Discharge(wl, precision=precision, solver=P.PIC_SOLVER_MG, bin_slack=0.05)
    d.start()
    d.step(8)
    path = str(tmp_path / "state.picrst")
    d.save(path)
    d.step(8)
    a = snapshot(d)
    d.close()
    e = P.Discharge.load(path, wl)
    e.step(8)
    b = snapshot(e)
    assert a["scalars"]["windows"] == 3
    for s in (0, 1):
        for k, v in a[f"p{s}"].items():
            assert np.array_equal(v, b[f"p{s}"][k]), (s, k)
    for f in FIELDS:
        assert np.array_equal(a[f], b[f], equal_nan=True), f
    for k, v in a["scalars"].items():
        assert v == b["scalars"][k] or (np.isnan(v) and np.isnan(b["scalars"][k])), (k, v, b["scalars"][k])
    assert e.status() == 0
    e.close()


def test_load_rejects_truncated_file(tmp_path):
    P = pic()
    wl = W.gec_case(64, 32, 30.0, 150.0, n_per_species=10_000)
    d = P.Discharge(wl)
    d.start()
    path = tmp_path / "state.picrst"
    d.save(str(path))
    raw = path.read_bytes()
    (tmp_path / "cut").write_bytes(raw[: len(raw) // 2])
    with pytest.raises(P.PicError) as ei:
        P.Discharge.load(str(tmp_path / "cut"), wl)
    assert ei.value.code == P.PIC_EIO
    (tmp_path / "long").write_bytes(raw + b"x")
    with pytest.raises(P.PicError) as ei:
        P.Discharge.load(str(tmp_path / "long"), wl)
    assert ei.value.code == P.PIC_EIO


@pytest.mark.parametrize("precision", [1, 0], ids=["fp64", "fp32"])
def test_runs_reproduce_bit_for_bit_with_a_busy_overflow_region(precision, tmp_path):
    """Two runs from one saved state agree bit for bit while many particles
    pass through the overflow region.  The capacity leaves no room for bin
    slack, so every bin gets exactly its last count and each step's net inflow
    overflows; which particles overflow depends on the order of the slot
    claims, which differs between the runs, and must not change any result."""
    P = pic()
    wl = dataclasses.replace(W.gec_case(128, 64, 30.0, 150.0, n_per_species=100_000, seed_index=23),
                             steps_per_rf=5, phase_src=0.4)
    n = max(len(p.r) for p in wl.particles)
    wl = dataclasses.replace(wl, capacity=(int(1.3 * n), int(1.3 * n)))
    d = P.Discharge(wl, precision=precision, solver=P.PIC_SOLVER_MG)
    d.start()
    d.step(2)
    path = str(tmp_path / "state.picrst")
    d.save(path)
    d.close()
    runs = []
    for _ in range(2):
        e = P.Discharge.load(path, wl)
        e.step(6)
        runs.append((snapshot(e), e.status()))
        e.close()
    (a, sa), (b, sb) = runs
    assert sa == 0 and sb == 0
    # electrons cross cells every step; ions barely move, and overflow only by births
    assert a["store"][0]["overflow"] > 1000 and a["store"][1]["overflow"] > 0, a["store"]
    for s in (0, 1):
        for k, v in a[f"p{s}"].items():
            assert np.array_equal(v, b[f"p{s}"][k]), (s, k)
    for f in FIELDS:
        assert np.array_equal(a[f], b[f], equal_nan=True), f
