"""Seeded synthetic inputs for the IB-FE-IPCS step (geometry only).

This module makes the inputs that both the CUDA path and the CPU oracle consume:
the box and its coarse grid, the Lagrangian points X_i on the vessel wall with
their area elements dS_i and prescribed velocities U_B, the coarse-cell inside
mask, the inflow/outflow ports and the physical parameters.  It holds none of
the method's arithmetic (no delta kernel, no element integrals, no solver).

Conventions shared by every consumer:
  * coarse-cell arrays are numpy arrays shaped [nz, ny, nx] (x fastest);
  * a port is a disc on a box face: axis (0/1/2), side (0 = low face, 1 = high
    face), centre, radius, kind ('inlet' | 'pinlet' | 'outlet') and a waveform
    w(t) = a0 + sum_k a_k cos(2 pi k t / T) + b_k sin(2 pi k t / T): the peak
    of the parabolic profile of a velocity inlet ('inlet'), the imposed
    pressure of a pressure inlet ('pinlet'); an outlet holds zero pressure;
  * the area element follows the paper's uniform rule (Sec. 2.5): every point
    carries dS = (wall area) / M.
Point sampling is stratified jitter: M equal-area strata in (theta, z), one
seeded point per stratum, displaced by at most +-0.35 of a stratum, which keeps
the spacing close to uniform as Sec. 2.5 asks.
"""
from __future__ import annotations

import math

import numpy as np

INLET = "inlet"
PINLET = "pinlet"
OUTLET = "outlet"


def _port(axis, side, center, radius, kind, a0=0.0, a=(), b=(), period=1.0):
    return {
        "axis": int(axis), "side": int(side),
        "center": tuple(float(c) for c in center), "radius": float(radius),
        "kind": kind, "a0": float(a0), "a": tuple(float(v) for v in a),
        "b": tuple(float(v) for v in b), "period": float(period),
    }


def cylinder_wall_points(R, z0, z1, M, seed, jitter=0.35):
    """Stratified-jitter points on the wall r = R, z0 <= z <= z1 of a z-aligned tube."""
    circ = 2.0 * math.pi * R
    length = z1 - z0
    n_th = max(1, int(round(math.sqrt(M * circ / length))))
    n_z = max(1, int(round(M / n_th)))
    rng = np.random.default_rng(seed)
    jt = rng.uniform(-jitter, jitter, size=(n_z, n_th))
    jz = rng.uniform(-jitter, jitter, size=(n_z, n_th))
    i_th = np.arange(n_th)[None, :] + 0.5 + jt
    i_z = np.arange(n_z)[:, None] + 0.5 + jz
    theta = i_th * (2.0 * math.pi / n_th)
    z = z0 + i_z * (length / n_z)
    X = np.stack([R * np.cos(theta), R * np.sin(theta), z], axis=-1).reshape(-1, 3)
    m = X.shape[0]
    dS = np.full(m, circ * length / m)
    return np.ascontiguousarray(X, dtype=np.float64), dS


def cell_centres(origin, extent, n):
    """Coarse-cell centre coordinates, each shaped [nz, ny, nx]."""
    h = [extent[a] / n[a] for a in range(3)]
    xs = [origin[a] + (np.arange(n[a]) + 0.5) * h[a] for a in range(3)]
    zc, yc, xc = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return xc, yc, zc


def cylinder_case(n=(16, 16, 64), R=0.5, length=4.0, half_width=0.6, M=2000,
                  seed=1, max_level=0, refine_band=2, reduce_band=-1,
                  nu=0.1, dt=0.01, steps=50, a0=1.0, b=(), period=1.0,
                  name=None, inlet=INLET, viscous="grad"):
    """Straight tube of radius R along z, immersed in [-w, w]^2 x [0, length].

    Defaults: the uniform 16x16x64 cylinder, nu = 0.1, dt = 0.01, steady
    parabolic inlet of peak 1, and M = 2000 wall points, which puts the spacing
    ratio a = sqrt(dS)/h at 1.06 (x, y) and 1.27 (z), the regime of the paper's
    Table 1 (a = 0.98).  At M = 4000 (a = 0.75) the force matrix A_F of Eq. 22 is
    numerically rank-deficient on this grid (Sec. 2.5 warns of exactly this).
    inlet = PINLET drives the flow by the inlet pressure a0 (+ harmonics)
    instead; a0 = 16 nu L / R^2 (6.4 with the defaults) gives the same
    Poiseuille flow of peak 1 (the pressure-driven tube of Sec. 3.1).
    viscous = "sym" selects the symmetric viscous form 2 nu (eps(u), eps(v)).
    """
    origin = (-half_width, -half_width, 0.0)
    extent = (2.0 * half_width, 2.0 * half_width, float(length))
    X, dS = cylinder_wall_points(R, 0.0, length, M, seed)
    xc, yc, zc = cell_centres(origin, extent, n)
    inside = (np.hypot(xc, yc) < R).astype(np.uint8)
    ports = [
        _port(2, 0, (0.0, 0.0, 0.0), R, inlet, a0=a0, b=b, period=period),
        _port(2, 1, (0.0, 0.0, length), R, OUTLET),
    ]
    return {
        "name": name or f"cylinder_{n[0]}x{n[1]}x{n[2]}_L{max_level}",
        "origin": origin, "extent": extent, "n": tuple(int(v) for v in n),
        "max_level": int(max_level), "refine_band": int(refine_band),
        "reduce_band": int(reduce_band),
        "nu": float(nu), "rho": 1.0, "dt": float(dt), "steps": int(steps),
        "ports": ports, "X": X, "dS": dS, "UB": np.zeros_like(X),
        "inside": inside, "viscous": viscous,
    }


def cylinder_uniform_16x16x64(**kw):
    """Uniform 16x16x64 cylinder, Re 10, dt 0.01, 50 steps, FP64."""
    return cylinder_case(**kw)


def aneurysm_128x128x256_L2(**kw):
    """Tube R = 0.5 along z (length 4) fused with a sphere R = 0.6 centred 0.7
    off the axis at mid-length, box [-0.6, 1.4] x [-1, 1] x [0, 4] on
    128x128x256 coarse cells (h0 = 1/64), two refinement levels, domain
    reduction, ~60k points (spacing 4.3 finest cells), pulsatile inflow
    u_max(t) = 1 + 0.5 sin(2 pi t), nu = 0.01, dt = 0.001, 2000 steps."""
    args = dict(R=0.5, length=4.0, Rs=0.6, offset=0.7, h=1.0 / 64, spacing=4.31, seed=3, max_level=2,
                refine_band=2, reduce_band=2, nu=0.01, dt=0.001, steps=2000, a0=1.0, b=(0.5,),
                box=((-0.6, -1.0, 0.0), (2.0, 2.0, 4.0)))
    args.update(kw)
    c = aneurysm_case(**args)
    c["name"] = "aneurysm_128x128x256_L2"
    return c


def cylinder_refined_64x64x256(**kw):
    """64x64x256 cylinder, one refinement level in a 2h band around the wall,
    cells more than 2h outside the wall dropped, 32k points, pulsatile inflow
    u_max(t) = 1 + 0.5 sin(2 pi t), nu = 0.02, dt = 0.002, 1000 steps."""
    args = dict(n=(64, 64, 256), M=32000, seed=2, max_level=1, refine_band=2,
                reduce_band=2, nu=0.02, dt=0.002, steps=1000, a0=1.0, b=(0.5,),
                period=1.0, name="cylinder_64x64x256_L1")
    args.update(kw)
    return cylinder_case(**args)


def paper_tube_sec31(p_in=1.0, M=1632, seed=31, port_tangential="zero", dt=2.5e-3, steps=400):
    """The pressure-driven tube of Sec. 3.1 in SI units: radius 5 mm, length
    50 mm, box -6..6 mm across (Table 1's box), the 12x12x50 grid of Table 1's
    first row (h = 1 mm) with its 1632 wall points, blood density 1050 and
    viscosity 0.00345 (kinematic nu = mu / rho), inlet pressure p_in Pa over a
    zero-pressure outlet (kinematic pressure p_in / rho).  The exact flow has
    U_max = R^2 p_in / (4 mu L) = 0.0362 m/s for p_in = 1."""
    rho, mu = 1050.0, 0.00345
    c = cylinder_case(n=(12, 12, 50), R=0.005, length=0.05, half_width=0.006, M=M, seed=seed, nu=mu / rho, dt=dt,
                      steps=steps, inlet=PINLET, a0=p_in / rho, name=f"paper_tube_p{p_in:g}_12x12x50")
    c["port_tangential"] = port_tangential
    return c


def cylinder_refined_slab_64x64x16(**kw):
    """A slab of the refined 64x64x256 cylinder: the same cross-section, grid
    spacing, bands, viscosity, time step and wall-point density over 16 of its
    256 coarse cells along the axis (length 0.25, 2000 points).  The oracle
    steps it in seconds; it still spans thousands of bricks and a five-level
    multigrid hierarchy."""
    length = 4.0 * 16 / 256
    args = dict(n=(64, 64, 16), length=length, M=2000, seed=2, max_level=1, refine_band=2, reduce_band=2,
                nu=0.02, dt=0.002, steps=2, a0=1.0, b=(0.5,), period=1.0, name="cylinder_64x64x16_L1_slab")
    args.update(kw)
    return cylinder_case(**args)


def square_duct_case(n=(8, 8, 32), L=4.0, nu=0.1, p_in=1.0, dt=1.0, steps=15, name=None):
    """Square duct [-1/2, 1/2]^2 x [0, L] without an immersed boundary (M = 0):
    no-slip box walls, a pressure inlet and an outlet (discs just inside the
    walls) on the end faces, the whole box active."""
    ports = [_port(2, 0, (0.0, 0.0, 0.0), 0.499, PINLET, a0=p_in), _port(2, 1, (0.0, 0.0, L), 0.499, OUTLET)]
    return _case(name or f"duct_{n[0]}x{n[1]}x{n[2]}", (-0.5, -0.5, 0.0), (1.0, 1.0, float(L)), n,
                 np.zeros((0, 3)), np.zeros(0), np.ones((n[2], n[1], n[0]), np.uint8), ports, nu, dt, steps,
                 0, 2, -1)


def cylinder_refined_small(n=(16, 16, 32), M=None, seed=7, **kw):
    """A reduced copy of the refined cylinder: same geometry rules and bands,
    a coarse grid small enough for the oracle's direct solves in seconds."""
    length = 4.0 * n[2] / 64.0 if "length" not in kw else kw.pop("length")
    if M is None:
        # keep sqrt(dS)/h_fine close to the refined 64x64x256 case (about 2.3)
        hf = min(1.2 / n[0], length / n[2]) / 2.0
        area = 2.0 * math.pi * 0.5 * length
        M = max(64, int(round(area / (2.3 * hf) ** 2)))
    args = dict(n=n, length=length, M=M, seed=seed, max_level=1, refine_band=2,
                reduce_band=2, nu=0.02, dt=0.002, steps=5, a0=1.0, b=(0.5,),
                period=1.0, name=f"cylinder_{n[0]}x{n[1]}x{n[2]}_L1")
    args.update(kw)
    return cylinder_case(**args)



# ---------------------------------------------------------------------------
# Further synthetic vessels (serving mix and the aneurysm case)
# ---------------------------------------------------------------------------
def _box(lo, hi):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return tuple(float(v) for v in lo), tuple(float(v) for v in (hi - lo))


def _grid_for(extent, h):
    return tuple(max(2, int(math.ceil(e / h))) for e in extent)


def _case(name, origin, extent, n, X, dS, inside, ports, nu, dt, steps, max_level, refine_band, reduce_band):
    return {
        "name": name, "origin": origin, "extent": extent, "n": tuple(int(v) for v in n),
        "max_level": int(max_level), "refine_band": int(refine_band), "reduce_band": int(reduce_band),
        "nu": float(nu), "rho": 1.0, "dt": float(dt), "steps": int(steps), "ports": ports,
        "X": np.ascontiguousarray(X, dtype=np.float64), "dS": np.ascontiguousarray(dS, dtype=np.float64),
        "UB": np.zeros((len(X), 3)), "inside": inside.astype(np.uint8),
    }


def aneurysm_case(R=0.5, length=4.0, Rs=0.6, offset=0.7, h=1.0 / 32, spacing=2.3, seed=3, max_level=1,
                  refine_band=2, reduce_band=2, nu=0.01, dt=0.001, steps=2000, a0=1.0, b=(0.5,), box=None):
    """Saccular aneurysm: a tube of radius R along z fused with a sphere of
    radius Rs centred `offset` off the axis at mid-length.  Points: stratified
    jitter on the tube wall outside the sphere and on the sphere outside the
    tube (equal-area strata in (cos phi, theta)); dS = stratum area.  `box`
    (origin, extent) fixes the domain; by default it is the vessel plus 4h."""
    zc = 0.5 * length
    margin = 4.0 * h
    if box is None:
        origin, extent = _box((-R - margin, -max(R, Rs) - margin, 0.0),
                              (offset + Rs + margin, max(R, Rs) + margin, length))
    else:
        origin, extent = tuple(box[0]), tuple(box[1])
    n = _grid_for(extent, h)
    extent = tuple(n[a] * h for a in range(3))
    hf = h / (1 << max_level)
    rng = np.random.default_rng(seed)
    # tube wall
    ds_target = (spacing * hf) ** 2
    circ = 2 * math.pi * R
    n_th = max(8, int(round(circ / math.sqrt(ds_target))))
    n_z = max(4, int(round(length / math.sqrt(ds_target))))
    th = (np.arange(n_th)[None, :] + 0.5 + rng.uniform(-0.35, 0.35, (n_z, n_th))) * (2 * math.pi / n_th)
    zz = (np.arange(n_z)[:, None] + 0.5 + rng.uniform(-0.35, 0.35, (n_z, n_th))) * (length / n_z)
    Xt = np.stack([R * np.cos(th), R * np.sin(th), zz], -1).reshape(-1, 3)
    keep = np.linalg.norm(Xt - np.array([offset, 0.0, zc]), axis=1) > Rs
    Xt = Xt[keep]
    dSt = np.full(len(Xt), circ * length / (n_th * n_z))
    # sphere
    area_s = 4 * math.pi * Rs * Rs
    n_s = max(16, int(round(area_s / ds_target)))
    n_mu = max(4, int(round(math.sqrt(n_s / 2))))
    n_ph = max(8, int(round(n_s / n_mu)))
    mu = -1 + (np.arange(n_mu)[:, None] + 0.5 + rng.uniform(-0.35, 0.35, (n_mu, n_ph))) * (2.0 / n_mu)
    ph = (np.arange(n_ph)[None, :] + 0.5 + rng.uniform(-0.35, 0.35, (n_mu, n_ph))) * (2 * math.pi / n_ph)
    sr = np.sqrt(np.clip(1 - mu * mu, 0, 1))
    Xs = np.stack([offset + Rs * sr * np.cos(ph), Rs * sr * np.sin(ph), zc + Rs * mu], -1).reshape(-1, 3)
    Xs = Xs[np.hypot(Xs[:, 0], Xs[:, 1]) > R]
    dSs = np.full(len(Xs), area_s / (n_mu * n_ph))
    X = np.concatenate([Xt, Xs])
    dS = np.concatenate([dSt, dSs])
    xc, yc, zcc = cell_centres(origin, extent, n)
    inside = (np.hypot(xc, yc) < R) | (np.sqrt((xc - offset) ** 2 + yc ** 2 + (zcc - zc) ** 2) < Rs)
    ports = [_port(2, 0, (0.0, 0.0, 0.0), R, INLET, a0=a0, b=b, period=1.0),
             _port(2, 1, (0.0, 0.0, length), R, OUTLET)]
    return _case(f"aneurysm_{n[0]}x{n[1]}x{n[2]}_L{max_level}", origin, extent, n, X, dS, inside, ports, nu, dt,
                 steps, max_level, refine_band, reduce_band)


def aneurysm_slab_128x128x16_L2(nz=16, **kw):
    """A slab of `nz` coarse cells of the 128x128x256 aneurysm, centred on the
    sac (mid-length): the same box cross-section, coarse spacing, levels,
    bands, viscosity, time step and wall points (those inside the slab), with
    a velocity inlet and an outlet on the tube's disc at the slab's end faces.
    The oracle steps it in seconds to a minute."""
    c = aneurysm_128x128x256_L2(**kw)
    h = c["extent"][2] / c["n"][2]
    k0 = c["n"][2] // 2 - nz // 2
    z0, z1 = k0 * h, (k0 + nz) * h
    X, dS = c["X"], c["dS"]
    keep = (X[:, 2] >= z0) & (X[:, 2] <= z1)
    X = X[keep].copy()
    X[:, 2] -= z0
    n = (c["n"][0], c["n"][1], nz)
    origin = (c["origin"][0], c["origin"][1], 0.0)
    extent = (c["extent"][0], c["extent"][1], nz * h)
    R = c["ports"][0]["radius"]
    ports = [_port(2, 0, (0.0, 0.0, 0.0), R, INLET, a0=1.0, b=(0.5,), period=1.0),
             _port(2, 1, (0.0, 0.0, extent[2]), R, OUTLET)]
    inside = np.ascontiguousarray(c["inside"][k0:k0 + nz])
    return _case(f"aneurysm_128x128x{nz}_L2_slab", origin, extent, n, X, dS[keep], inside, ports, c["nu"], c["dt"],
                 2, c["max_level"], c["refine_band"], c["reduce_band"])


def bent_tube_case(R=0.5, Rc=1.5, l_in=1.5, l_out=1.5, h=1.0 / 16, spacing=2.3, seed=5, max_level=0,
                   refine_band=2, reduce_band=2, nu=0.02, dt=0.005, steps=200, a0=1.0, b=()):
    """90-degree bend in the xz-plane: a straight inflow leg along +z from the
    low z face, a quarter torus of centreline radius Rc, and a straight outflow
    leg along +x to the high x face.  Points: stratified jitter in (arclength,
    angle) with each point's dS the local area element times the stratum size
    (the torus area element varies with the angle)."""
    margin = 4.0 * h
    zb = l_in                                        # start of the bend
    # centreline: (0,0,s) for s<zb; arc centre (Rc, 0, zb); outflow along +x at z = zb + Rc
    xmax = Rc + l_out
    origin, extent = _box((-R - margin, -R - margin, 0.0), (xmax, R + margin, zb + Rc + R + margin))
    n = _grid_for(extent, h)
    extent = (xmax - origin[0], n[1] * h, n[2] * h)
    n = (max(2, int(round(extent[0] / h))), n[1], n[2])
    extent = (n[0] * h, extent[1], extent[2])
    xmax = origin[0] + extent[0]
    l_out = xmax - Rc
    hf = h / (1 << max_level)
    rng = np.random.default_rng(seed)
    ds_target = (spacing * hf) ** 2
    L_arc = 0.5 * math.pi * Rc
    L_tot = zb + L_arc + l_out
    n_s = max(8, int(round(L_tot / math.sqrt(ds_target))))
    n_th = max(8, int(round(2 * math.pi * R / math.sqrt(ds_target))))
    s = (np.arange(n_s)[:, None] + 0.5 + rng.uniform(-0.35, 0.35, (n_s, n_th))) * (L_tot / n_s)
    th = (np.arange(n_th)[None, :] + 0.5 + rng.uniform(-0.35, 0.35, (n_s, n_th))) * (2 * math.pi / n_th)
    s, th = s.ravel(), th.ravel()
    X = np.zeros((len(s), 3))
    w = np.ones(len(s))                               # local area factor
    # frame: binormal e_y; normal in the xz-plane
    for k in range(len(s)):
        sk, tk = s[k], th[k]
        if sk < zb:
            c, t, nrm = np.array([0.0, 0.0, sk]), np.array([0, 0, 1.0]), np.array([-1.0, 0, 0])
        elif sk < zb + L_arc:
            a = (sk - zb) / Rc
            c = np.array([Rc - Rc * math.cos(a), 0.0, zb + Rc * math.sin(a)])
            t = np.array([math.sin(a), 0.0, math.cos(a)])
            nrm = np.array([-math.cos(a), 0.0, math.sin(a)])          # away from the bend centre
            w[k] = 1.0 + (R / Rc) * math.cos(tk)
        else:
            c = np.array([Rc + (sk - zb - L_arc), 0.0, zb + Rc])
            t, nrm = np.array([1.0, 0, 0]), np.array([0, 0, 1.0])
        X[k] = c + R * (math.cos(tk) * nrm + math.sin(tk) * np.array([0, 1.0, 0]))
    dS = w * (L_tot / n_s) * (2 * math.pi * R / n_th)
    xc, yc, zcc = cell_centres(origin, extent, n)
    # distance to the centreline
    d_in = np.where(zcc < zb, np.hypot(xc, yc), np.inf)
    rr = np.hypot(xc - Rc, zcc - zb)
    ang_ok = (zcc >= zb) & (xc <= Rc)
    d_arc = np.where(ang_ok, np.hypot(rr - Rc, yc), np.inf)
    d_out = np.where(xc > Rc, np.hypot(zcc - (zb + Rc), yc), np.inf)
    inside = np.minimum(np.minimum(d_in, d_arc), d_out) < R
    ports = [_port(2, 0, (0.0, 0.0, 0.0), R, INLET, a0=a0, b=b, period=1.0),
             _port(0, 1, (xmax, 0.0, zb + Rc), R, OUTLET)]
    return _case(f"bend_{n[0]}x{n[1]}x{n[2]}_L{max_level}", origin, extent, n, X, dS, inside, ports, nu, dt, steps,
                 max_level, refine_band, reduce_band)


def aorta_waveform():
    """The synthetic aorta's inflow waveform (aorta_waveform.json): period,
    a0, a_k, b_k of the peak velocity, the peak Reynolds number and the inlet
    diameter it refers to."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "aorta_waveform.json")) as f:
        return json.load(f)


def _tube_points(centre, tangent, normal, radius, dradius, s0, s1, ds_target, rng, curvature=0.0):
    """Stratified jitter on a tube of varying radius around a planar
    centreline: strata in (arclength s, angle theta), one point each,
    displaced by at most +-0.35 stratum; theta measured from `normal(s)`
    towards e_y.  dS = the local area element R (1 - kappa R cos theta)
    sqrt(1 + R'^2) times the stratum size."""
    L = s1 - s0
    rmax = max(radius(s0), radius(s1))
    n_s = max(4, int(round(L / math.sqrt(ds_target))))
    n_th = max(8, int(round(2 * math.pi * rmax / math.sqrt(ds_target))))
    s = s0 + (np.arange(n_s)[:, None] + 0.5 + rng.uniform(-0.35, 0.35, (n_s, n_th))) * (L / n_s)
    th = (np.arange(n_th)[None, :] + 0.5 + rng.uniform(-0.35, 0.35, (n_s, n_th))) * (2 * math.pi / n_th)
    s, th = s.ravel(), th.ravel()
    C, N, R, dR = centre(s), normal(s), radius(s), dradius(s)
    ey = np.array([0.0, 1.0, 0.0])
    X = C + R[:, None] * (np.cos(th)[:, None] * N + np.sin(th)[:, None] * ey[None, :])
    dS = R * (1.0 - curvature * R * np.cos(th)) * np.sqrt(1.0 + dR * dR) * (L / n_s) * (2 * math.pi / n_th)
    return X, dS


def aorta_case(n=(256, 256, 384), max_level=2, M=200000, seed=4, Rc=3.0, l_down=6.0, r_in=1.0, r_out=0.7,
               r_branch=0.25, branch_deg=(110.0, 90.0, 70.0), refine_band=2, reduce_band=2, dt=5e-4, steps=2000,
               name=None):
    """Synthetic aorta-like vessel.  The centreline arches over 180 degrees in
    the xz-plane (a circle of radius Rc about the origin, from (-Rc, 0, 0)
    up over (0, 0, Rc) to (Rc, 0, 0)), then descends straight for l_down.
    The radius tapers linearly from r_in to r_out along the arch and the
    descent.  Three branch tubes of radius r_branch rise along +z from the
    arch centreline at the given arch angles to the top of the box.  The
    ascending limb continues straight down, radius r_in, to the low-z face of
    the box at z = -l_down: the inlet and the descending outlet both lie on
    that face and the branch outlets on the high-z face (ports lie on box
    faces).  Box: x and y within +-(Rc + r_in) plus a margin of 4 cubic
    cells, cubic spacing h = 2 (Rc + r_in + 4 h) / n_x, extent n h per axis.
    Inflow: the 5-harmonic waveform of aorta_waveform.json (peak 1);
    nu = U_peak D_in / Re_peak = 2 / 1500."""
    wf = aorta_waveform()
    nu = 1.0 * wf["inlet_diameter"] / wf["peak_reynolds"]
    half = Rc + r_in
    h = 2.0 * half / (n[0] - 8)                          # x: the vessel plus 4 cells each side
    origin = (-half - 4 * h, -0.5 * n[1] * h, -l_down)
    extent = (n[0] * h, n[1] * h, n[2] * h)
    z_top = origin[2] + extent[2]
    hf = h / (1 << max_level)
    L_arc = math.pi * Rc
    L_tot = L_arc + l_down
    rad = lambda s: r_in + (r_out - r_in) * np.clip(s, 0.0, L_tot) / L_tot
    drad = lambda s: np.where((s >= 0) & (s <= L_tot), (r_out - r_in) / L_tot, 0.0)
    # centreline by arclength s: s < 0 the inflow extension, [0, L_arc] the
    # arch, beyond it the descent
    def centre(s):
        s = np.asarray(s, dtype=np.float64)
        phi = math.pi - np.clip(s, 0.0, L_arc) / Rc
        c = np.stack([Rc * np.cos(phi), np.zeros_like(s), Rc * np.sin(phi)], -1)
        c = np.where((s < 0)[..., None], np.stack([-Rc + 0 * s, 0 * s, s], -1), c)
        c = np.where((s > L_arc)[..., None], np.stack([Rc + 0 * s, 0 * s, -(s - L_arc)], -1), c)
        return c
    def normal(s):   # in the xz-plane, away from the arch centre (and -x / +x on the straight limbs)
        s = np.asarray(s, dtype=np.float64)
        phi = math.pi - np.clip(s, 0.0, L_arc) / Rc
        return np.stack([np.cos(phi), np.zeros_like(s), np.sin(phi)], -1)
    rng = np.random.default_rng(seed)
    # area to spread the M points over (estimated), then each part
    A_arch = 2 * math.pi * 0.5 * (r_in + rad(L_arc)) * L_arc
    A_down = 2 * math.pi * 0.5 * (rad(L_arc) + r_out) * l_down
    A_in = 2 * math.pi * r_in * l_down
    br_len = [z_top - Rc * math.sin(math.radians(d)) for d in branch_deg]
    A_br = sum(2 * math.pi * r_branch * L for L in br_len)
    ds_target = (A_arch + A_down + A_in + A_br) / M
    parts = [
        _tube_points(centre, None, normal, rad, drad, 0.0, L_arc, ds_target, rng, curvature=1.0 / Rc),
        _tube_points(centre, None, normal, rad, drad, L_arc, L_tot, ds_target, rng),
        _tube_points(centre, None, normal, rad, drad, -l_down, 0.0, ds_target, rng),
    ]
    bx = []
    for d, L in zip(branch_deg, br_len):
        x0, z0 = Rc * math.cos(math.radians(d)), Rc * math.sin(math.radians(d))
        bx.append(x0)
        cb = lambda s, x0=x0, z0=z0: np.stack([x0 + 0 * np.asarray(s), 0 * np.asarray(s), z0 + np.asarray(s)], -1)
        nb = lambda s: np.stack([np.ones_like(np.asarray(s)), 0 * np.asarray(s), 0 * np.asarray(s)], -1)
        parts.append(_tube_points(cb, None, nb, lambda s: r_branch + 0 * np.asarray(s),
                                  lambda s: 0 * np.asarray(s), 0.0, L, ds_target, rng))
    # signed inside tests: distance to each centreline piece below its radius
    def in_main(P):
        x, y, z = P[..., 0], P[..., 1], P[..., 2]
        # arch: nearest point on the circle in the xz-plane, upper half
        rr = np.hypot(x, z)
        phi = np.arctan2(z, x)
        on_arch = (z >= 0) & (phi >= 0) & (phi <= math.pi)
        s_arch = (math.pi - np.clip(phi, 0, math.pi)) * Rc
        d_arch = np.where(on_arch, np.hypot(rr - Rc, y), np.inf)
        ins = d_arch < rad(s_arch)
        ins |= (z < 0) & (np.hypot(x + Rc, y) < r_in)                              # inflow extension
        s_down = L_arc - z
        ins |= (z < 0) & (np.hypot(x - Rc, y) < rad(s_down))                      # descent
        return ins
    def in_branch(P):
        x, y, z = P[..., 0], P[..., 1], P[..., 2]
        ins = np.zeros(P.shape[:-1], dtype=bool)
        for d, x0 in zip(branch_deg, bx):
            z0 = Rc * math.sin(math.radians(d))
            ins |= (z >= z0) & (np.hypot(x - x0, y) < r_branch)
        return ins
    Xs, dSs = [], []
    for k, (X, dS) in enumerate(parts):
        keep = ~in_branch(X) if k < 3 else ~in_main(X)
        Xs.append(X[keep])
        dSs.append(dS[keep])
    X = np.concatenate(Xs)
    dS = np.concatenate(dSs)
    xc, yc, zc = cell_centres(origin, extent, n)
    P = np.stack([xc, yc, zc], -1)
    inside = in_main(P) | in_branch(P)
    a, b = tuple(wf["a"]), tuple(wf["b"])
    ports = [_port(2, 0, (-Rc, 0.0, origin[2]), r_in, INLET, a0=wf["a0"], a=a, b=b, period=wf["period"]),
             _port(2, 0, (Rc, 0.0, origin[2]), r_out, OUTLET)]
    for x0 in bx:
        ports.append(_port(2, 1, (x0, 0.0, z_top), r_branch, OUTLET))
    return _case(name or f"aorta_{n[0]}x{n[1]}x{n[2]}_L{max_level}", origin, extent, n, X, dS, inside, ports, nu,
                 dt, steps, max_level, refine_band, reduce_band)


def aorta_256x256x384_L2(**kw):
    """The synthetic aorta on 256x256x384 coarse cells with two refinement
    levels, domain reduction, 200k wall points, the cardiac waveform inflow
    (peak Re 1500), dt = 5e-4, 2000 steps."""
    return aorta_case(**kw)


def serving_requests(n_req=256, rate=None, seed=5, steps=200, cells_lo=32 ** 3, cells_hi=128 ** 3):
    """Poisson-arrival stream of seeded random vessels: kind in {straight,
    bent, aneurysmal}, radius 0.3-1.0, length 3-10, about 32^3 to 128^3 active
    leaf cells (log-uniform target; the coarse spacing is sized for it from an
    estimate of the refined wall band), 0-2 refinement levels, nu 0.01-0.05.
    Returns [(arrival_time, case)], arrival times in units of 1/rate seconds
    (rate None: unit rate)."""
    rng = np.random.default_rng(seed)
    lam = 1.0 if rate is None else float(rate)
    t = np.cumsum(rng.exponential(1.0 / lam, n_req))
    out = []
    for k in range(n_req):
        kind = ["straight", "bent", "aneurysm"][int(rng.integers(0, 3))]
        R = float(rng.uniform(0.3, 1.0))
        L = float(rng.uniform(3.0, 10.0))
        target = float(np.exp(rng.uniform(np.log(cells_lo), np.log(cells_hi))))
        levels = int(rng.integers(0, 3))
        nu = float(rng.uniform(0.01, 0.05))
        sub = int(rng.integers(1 << 20))
        if kind == "straight":
            vol = math.pi * (R * 1.25) ** 2 * L
        elif kind == "bent":
            vol = math.pi * (R * 1.25) ** 2 * (0.6 * L + 0.5 * math.pi * 3 * R)
        else:
            vol = math.pi * (R * 1.25) ** 2 * L + 4.0 / 3.0 * math.pi * (1.2 * R * 1.2) ** 3
        # leaf cells: the wall band (2 coarse cells each side) is refined 8^levels
        # times, the next band 8^(levels-1) times; size the coarse spacing h so
        # that coarse cells x this factor meet the target (fixed point in h)
        wall = vol / (math.pi * (R * 1.25) ** 2) * 2 * math.pi * R   # wall area of the vessel
        h = (vol / target) ** (1.0 / 3.0)
        for _ in range(20):
            f = 1.0
            if levels >= 1:
                inner = min(1.0, wall * 5 * h / vol)              # level `levels` band
                outer = min(1.0 - inner, wall * 4 * h / vol) if levels == 2 else 0.0
                f = 1.0 + inner * (8 ** levels - 1) + outer * (8 ** (levels - 1) - 1)
            h = (vol * f / target) ** (1.0 / 3.0)
        h = max(h, 2.0 * R / 28)
        dt = 0.25 * h / (1 << levels)
        if kind == "straight":
            n_ax = max(8, int(round(L / h)))
            nxy = max(8, int(round(2 * (R + 4 * h) / h)))
            Rl = R
            pts = (2 * math.pi * R * L) / (2.3 * h / (1 << levels)) ** 2
            c = cylinder_case(n=(nxy, nxy, n_ax), R=Rl, length=L, half_width=nxy * h / 2, M=max(64, int(pts)),
                              seed=sub, max_level=levels, refine_band=2, reduce_band=2, nu=nu, dt=dt, steps=steps,
                              name=f"req{k}_straight")
        elif kind == "bent":
            c = bent_tube_case(R=R, Rc=3 * R, l_in=0.3 * L, l_out=0.3 * L, h=h, seed=sub, max_level=levels,
                               nu=nu, dt=dt, steps=steps)
            c["name"] = f"req{k}_bent"
        else:
            c = aneurysm_case(R=R, length=L, Rs=1.2 * R, offset=1.4 * R, h=h, seed=sub, max_level=levels, nu=nu,
                              dt=dt, steps=steps, b=())
            c["name"] = f"req{k}_aneurysm"
        out.append((float(t[k]), c))
    return out
