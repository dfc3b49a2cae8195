"""CUDA path vs the CPU oracle on larger and degenerate inputs, through the C ABI.

* The 64x64x16 slab of the refined 64x64x256 cylinder: the full-size case's
  cross-section, grid spacing, bands, time step and wall-point density (about
  160k leaf cells, 2000 points, thousands of bricks, a five-level multigrid
  hierarchy), two steps, every field of every step against the oracle: FP64
  path relative L2 <= 1e-10, mixed path <= 1e-6.
* A square duct without an immersed boundary (M = 0; Eq. 9, Eq. 12 and the
  velocity correction alone, pressure-driven as in Sec. 3.1), the case the
  oracle pins against the closed-form duct flow.
* A reduced copy of the synthetic aorta (arched, tapered, three branches,
  five ports on two faces, the cardiac inflow waveform): 40x40x60 coarse
  cells, one level, 3k wall points, two steps.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ibfe
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-6

CASES = {
    "slab": (W.cylinder_refined_slab_64x64x16, 2),
    "duct_no_ib": (lambda: W.square_duct_case(n=(8, 8, 32), dt=0.5), 3),
    "aorta_small": (lambda: W.aorta_case(n=(40, 40, 60), max_level=1, M=3000, seed=44, dt=0.002,
                                         name="aorta_40x40x60_L1"), 2),
}
_ORACLE = {}


def oracle_hist(name):
    if name not in _ORACLE:
        make, steps = CASES[name]
        case = make()
        o = ibfe.Oracle(case)
        hist = []
        for _ in range(steps):
            o.step()
            hist.append({"u": o.u.copy(), "p": o.p.copy(), "phi": o.phi.copy(), "ut": o.ut.copy(),
                         "uib": o.u_ib.copy(), "F": o.F.copy(), "BF": o.BF.copy()})
        _ORACLE[name] = (case, o, hist)
    return _ORACLE[name]


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_every_field_every_step(name):
    from paper_2007_02082_gb300 import IBGrid
    case, o, hist = oracle_hist(name)
    g = IBGrid(case, precision="fp64")
    info = g.ib_grid_info()
    assert info["n_nodes"] == o.mesh.n_nodes and info["n_points"] == len(case["X"])
    if name == "slab":
        assert info["mg_levels"] >= 4
    fields = ["ut", "uib", "u", "p", "phi"] + (["F", "BF"] if len(case["X"]) else [])
    for k in range(len(hist)):
        g.ipcs_step(1)
        got = {"u": g.ib_fields_get("U"), "p": g.ib_fields_get("P"), "phi": g.ib_fields_get("PHI"),
               "ut": g.ib_fields_get("U_TENT"), "uib": g.ib_fields_get("U_IB")}
        if len(case["X"]):
            got["F"], got["BF"] = g.ib_fields_get("F_LAG"), g.ib_fields_get("B_F")
        for key in fields:
            e = rel_l2(got[key], hist[k][key])
            assert e <= TOL64, f"step {k + 1} {key}: rel L2 {e:.3e}"
    if not len(case["X"]):
        # no immersed boundary: the correction step changes nothing
        assert np.array_equal(g.ib_fields_get("U_IB"), g.ib_fields_get("U_TENT"))
    g.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_within_1e6(name):
    from paper_2007_02082_gb300 import IBGrid
    case, o, hist = oracle_hist(name)
    g = IBGrid(case, precision="mixed")
    g.ipcs_step(len(hist))
    ref = hist[-1]
    pairs = [("u", "U"), ("p", "P"), ("phi", "PHI")] + ([("F", "F_LAG")] if len(case["X"]) else [])
    for key, field in pairs:
        e = rel_l2(g.ib_fields_get(field), ref[key])
        assert e <= TOLMIX, f"{key}: rel L2 {e:.3e}"
    g.close()
