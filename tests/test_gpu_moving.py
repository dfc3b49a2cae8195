"""Moving wall (ib_set_points): the device rebuild of the supports (Eq. 17),
delta weights (Eq. 18), A_F (Eq. 22) and spreading lists (Eq. 19) after the
Lagrangian points move, against a fresh host build at the new positions and
against the oracle stepping the same motion.

Tolerances: structures bit-exact; a rebuilt handle and a fresh one step
bitwise alike from the same state (every list is sorted); FP64 fields within
relative L2 1e-10 of the oracle per step, the mixed path within 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ibfe
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _refined():
    return W.cylinder_case(n=(8, 8, 8), length=1.0, half_width=0.6, M=300, seed=51, max_level=1, refine_band=1,
                           reduce_band=1, nu=0.02, dt=0.01, b=(0.5,))


def _uniform():
    return W.cylinder_case(n=(8, 8, 16), length=2.0, M=250, seed=3, nu=0.1, dt=0.01)


def _hf(case):
    return np.array(case["extent"]) / (np.array(case["n"]) * 2 ** case["max_level"])


def test_rebuild_equals_fresh_build():
    """A deforming wall: the points that stay in their coarse cell move by
    0.3 / -0.2 finest cells in x / y (so the refinement and domain reduction,
    built from the point cells, are those of a fresh build at the new
    positions); the rebuilt structures equal the fresh build's bit for bit and
    the two handles step bitwise alike."""
    from paper_2007_02082_gb300 import IBGrid
    case = _refined()
    X = np.asarray(case["X"])
    x0, h0 = np.array(case["origin"]), np.array(case["extent"]) / np.array(case["n"])
    Xs = X + _hf(case) * np.array([0.3, -0.2, 0.0])
    keep = np.all(np.floor((Xs - x0) / h0) == np.floor((X - x0) / h0), axis=1)
    X1 = np.where(keep[:, None], Xs, X)
    hf = _hf(case)
    assert (np.floor((X1 - x0) / hf) != np.floor((X - x0) / hf)).any(axis=1).sum() > 10
    g = IBGrid(case, precision="fp64")
    g.ib_set_points(X1)
    c1 = dict(case, X=X1)
    h = IBGrid(c1, precision="fp64")
    for f in ("LEVEL", "ACTIVE"):
        assert np.array_equal(g.ib_fields_get(f), h.ib_fields_get(f)), f
    for f in ("IB_ORIGIN", "IB_FREE", "IB_WEIGHTS"):
        assert np.array_equal(g.ib_fields_get(f), h.ib_fields_get(f)), f
    g.ipcs_step(2)
    h.ipcs_step(2)
    for f in ("U", "P", "F_LAG"):
        assert np.array_equal(g.ib_fields_get(f), h.ib_fields_get(f)), f
    g.close()
    h.close()


@pytest.mark.parametrize("name", ["uniform", "refined"])
def test_translating_wall_matches_oracle(name):
    """The tube wall translates by delta per step along x with wall velocity
    delta / dt; before each step both sides move the points to t^{n+1}."""
    from paper_2007_02082_gb300 import IBGrid
    case = _uniform() if name == "uniform" else _refined()
    steps = 3
    # the wall stays inside the box (0.1 from its side in the uniform case)
    delta = np.array([0.1, 0.05, 0.0] if name == "uniform" else [0.3, 0.1, 0.0]) * _hf(case)
    UB = np.tile(delta / case["dt"], (len(case["X"]), 1))
    X0 = np.asarray(case["X"])
    o = ibfe.Oracle(case)
    g = IBGrid(case, precision="fp64")
    gm = IBGrid(case, precision="mixed")
    for n in range(steps):
        Xn = X0 + (n + 1) * delta
        o.set_points(Xn, UB)
        o.step()
        g.ib_set_points(Xn, UB)
        gm.ib_set_points(Xn, UB)
        g.ipcs_step(1)
        gm.ipcs_step(1)
        for key, f in (("u", "U"), ("p", "P"), ("F", "F_LAG")):
            e = rel_l2(g.ib_fields_get(f), getattr(o, key))
            assert e <= 1e-10, f"step {n + 1} {f}: {e:.3e}"
        assert np.array_equal(g.ib_fields_get("IB_ORIGIN"), o.ib.origin.astype(np.int32))
    for key, f in (("u", "U"), ("p", "P")):
        assert rel_l2(gm.ib_fields_get(f), getattr(o, key)) <= 1e-6, f
    # the wall moves: the corrected velocity at the points is the wall velocity
    assert np.abs(o.ib.W @ o.u_ib - UB).max() < 1e-9
    g.close()
    gm.close()


def test_leaving_the_refined_band_is_rejected():
    from paper_2007_02082_gb300 import IBError, IBGrid
    case = _refined()
    g = IBGrid(case, precision="fp64")
    org = g.ib_fields_get("IB_ORIGIN")
    X = np.asarray(case["X"])
    inward = X * np.array([0.5, 0.5, 1.0])   # into the coarse cells inside the tube
    with pytest.raises(IBError) as ei:
        g.ib_set_points(inward)
    assert ei.value.status == 1
    assert np.array_equal(g.ib_fields_get("IB_ORIGIN"), org)
    g.ipcs_step(1)
    assert g.ib_grid_info()["status_ib"] == 0
    with pytest.raises(IBError):
        g.ib_set_points(X[:-1])
    g.close()


def test_device_points_equal_host_points():
    import torch
    from paper_2007_02082_gb300 import IBGrid
    case = _uniform()
    X1 = np.asarray(case["X"]) + _hf(case) * np.array([-0.4, 0.25, 0.0])
    a = IBGrid(case, precision="fp64")
    b = IBGrid(case, precision="fp64")
    a.ib_set_points(X1)
    b.ib_set_points(torch.tensor(X1, device="cuda"))
    for f in ("IB_ORIGIN", "IB_FREE", "IB_WEIGHTS"):
        assert np.array_equal(a.ib_fields_get(f), b.ib_fields_get(f)), f
    a.close()
    b.close()
