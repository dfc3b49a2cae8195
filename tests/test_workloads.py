"""Properties of the synthetic inputs that stand in for the paper's vessels
(CPU only).  The aorta-like case (arched centreline, taper, three branches,
cardiac inflow) has no analytic solution; what its generator must fix is
checked here: the waveform's stated properties and the geometry's."""
import math

import numpy as np

import workloads as W


def _waveform(t, wf):
    u = wf["a0"] + 0 * t
    for k, (a, b) in enumerate(zip(wf["a"], wf["b"]), start=1):
        u = u + a * np.cos(2 * math.pi * k * t / wf["period"]) + b * np.sin(2 * math.pi * k * t / wf["period"])
    return u


def test_aorta_waveform_is_cardiac_like():
    """Five harmonics of period 1, peak 1, a brief reverse flow (minimum about
    -0.1, below zero for less than 15 % of the period), peak Reynolds number
    1500 on the inlet diameter with the case's viscosity."""
    wf = W.aorta_waveform()
    assert len(wf["a"]) == len(wf["b"]) == 5 and wf["period"] == 1.0
    t = np.linspace(0.0, 1.0, 20001)
    u = _waveform(t, wf)
    assert abs(u.max() - 1.0) < 5e-3
    assert -0.15 < u.min() < -0.05
    frac = np.mean(u < 0)
    assert 0.02 < frac < 0.15
    # one contiguous reverse-flow interval (brief, not scattered)
    neg = u[:-1] < 0
    assert np.count_nonzero(neg[1:] != neg[:-1]) <= 2
    c = W.aorta_case(n=(40, 40, 60), max_level=1, M=3000, seed=44)
    assert math.isclose(1.0 * wf["inlet_diameter"] / c["nu"], wf["peak_reynolds"])
    # the inlet port carries exactly this waveform
    p = c["ports"][0]
    assert p["kind"] == W.INLET and p["a0"] == wf["a0"] and p["a"] == tuple(wf["a"]) and p["b"] == tuple(wf["b"])


def test_aorta_geometry():
    """Points on the wall inside the box, ports on box faces inside the
    vessel, wall area close to the analytic one, taper and branches present."""
    c = W.aorta_case(n=(40, 40, 60), max_level=1, M=3000, seed=44)
    X, dS = c["X"], c["dS"]
    lo = np.array(c["origin"])
    hi = lo + np.array(c["extent"])
    assert np.all(X >= lo) and np.all(X <= hi)
    Rc, ld, ri, ro, rb = 3.0, 6.0, 1.0, 0.7, 0.25
    L_arc = math.pi * Rc
    area = (2 * math.pi * 0.5 * (ri + ri + (ro - ri) * L_arc / (L_arc + ld)) * L_arc
            + 2 * math.pi * 0.5 * (ri + (ro - ri) * L_arc / (L_arc + ld) + ro) * ld + 2 * math.pi * ri * ld)
    # three branches from the arch centreline to the top face
    area += sum(2 * math.pi * rb * (hi[2] - Rc * math.sin(math.radians(d))) for d in (110.0, 90.0, 70.0))
    # less the parts of each tube inside the other (the openings of the junctions)
    assert 0.95 < dS.sum() / area < 1.02
    # inlet, descending outlet and three branch outlets on the box faces
    ports = c["ports"]
    assert [p["kind"] for p in ports] == [W.INLET] + [W.OUTLET] * 4
    assert ports[0]["center"][2] == lo[2] and ports[1]["center"][2] == lo[2]
    assert all(math.isclose(p["center"][2], hi[2]) for p in ports[2:])
    assert ports[0]["radius"] == ri and ports[1]["radius"] == ro and all(p["radius"] == rb for p in ports[2:])
    # the radius tapers: wall points of the descent are closer to its axis than those of the inflow limb
    down = X[(X[:, 2] < -1.0) & (X[:, 0] > 0)]
    up = X[(X[:, 2] < -1.0) & (X[:, 0] < 0)]
    r_down = np.hypot(down[:, 0] - Rc, down[:, 1])
    r_up = np.hypot(up[:, 0] + Rc, up[:, 1])
    assert np.allclose(r_up, ri) and r_down.max() < ri - 0.15 and r_down.min() > ro - 1e-9
    # the inside mask holds the port discs' cells and the branches
    h = c["extent"][0] / c["n"][0]
    ins = c["inside"]
    for p in ports:
        i = int((p["center"][0] - lo[0]) / h)
        k = 0 if p["side"] == 0 else c["n"][2] - 1
        assert ins[k, c["n"][1] // 2, i] == 1
