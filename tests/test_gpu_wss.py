"""Wall shear stress at the Lagrangian points (ib_wss, Sec. 2.6): second-order
DC-PSE derivatives over the finest-level fluid nodes around each wall point.

The Poiseuille case checks the kernel on its own (a quadratic field is
differentiated exactly, WSS = 2 mu U / R); the refined case compares it with
the oracle's wall_shear_stress, first on the library's own velocity field
(only the DC-PSE arithmetic differs: relative 1e-10), then on the oracle's run
(FP64 step parity included: relative 1e-8).
"""
import numpy as np
import pytest

import workloads as W
from oracle import ibfe
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _normals(X):
    n = np.zeros_like(X)
    r = np.hypot(X[:, 0], X[:, 1])
    n[:, 0], n[:, 1] = X[:, 0] / r, X[:, 1] / r
    return n


def test_poiseuille_wss_exact():
    from paper_2007_02082_gb300 import IBGrid
    case = W.cylinder_uniform_16x16x64()
    g = IBGrid(case, precision="fp64")
    q = g.ib_fields_get("NODE_Q").astype(float)
    h = np.array(case["extent"]) / np.array(case["n"])
    x = np.array(case["origin"]) + q * h
    u = np.zeros((len(q), 3))
    u[:, 2] = 1.0 - 4.0 * (x[:, 0] ** 2 + x[:, 1] ** 2)
    g.ib_fields_set("U", u)
    X = np.asarray(case["X"])
    wss, grad = g.ib_wss(_normals(X), with_grad=True)
    assert np.abs(wss - 2 * case["nu"] * 1.0 / 0.5).max() <= 1e-9
    exact = np.zeros_like(grad)
    exact[:, 2, 0], exact[:, 2, 1] = -8.0 * X[:, 0], -8.0 * X[:, 1]
    assert np.abs(grad - exact).max() <= 1e-8
    g.close()


def test_wss_matches_oracle_on_a_refined_run():
    from paper_2007_02082_gb300 import IBGrid
    case = W.cylinder_refined_small(n=(16, 16, 8), seed=21)
    g = IBGrid(case, precision="fp64")
    g.ipcs_step(3)
    X = np.asarray(case["X"])
    nrm = _normals(X)
    wss = g.ib_wss(nrm)
    assert np.all(np.isfinite(wss)) and wss.max() > 0
    m = ibfe.build_mesh(case)
    ref_own, _ = ibfe.wall_shear_stress(m, g.ib_fields_get("U"), X, case["UB"], nrm, case["nu"], case["rho"])
    assert rel_l2(wss, ref_own) <= 1e-10
    o = ibfe.Oracle(case).run(3)
    ref, _ = ibfe.wall_shear_stress(m, o.u, X, case["UB"], nrm, case["nu"], case["rho"])
    assert rel_l2(wss, ref) <= 1e-8
    g.close()
