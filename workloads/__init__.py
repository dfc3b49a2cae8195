"""Seeded synthetic inputs for the IB-FE-IPCS step (geometry only).

This module makes the inputs that both the CUDA path and the CPU oracle consume:
the box and its coarse grid, the Lagrangian points X_i on the vessel wall with
their area elements dS_i and prescribed velocities U_B, the coarse-cell inside
mask, the inflow/outflow ports and the physical parameters.  It holds none of
the method's arithmetic (no delta kernel, no element integrals, no solver).

Conventions shared by every consumer:
  * coarse-cell arrays are numpy arrays shaped [nz, ny, nx] (x fastest);
  * a port is a disc on a box face: axis (0/1/2), side (0 = low face, 1 = high
    face), centre, radius, kind ('inlet' | 'outlet'), and for an inlet a
    parabolic profile of peak u_max(t) = a0 + sum_k a_k cos(2 pi k t / T)
    + b_k sin(2 pi k t / T);
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
                  name=None):
    """Straight tube of radius R along z, immersed in [-w, w]^2 x [0, length].

    Defaults: the uniform 16x16x64 cylinder, nu = 0.1, dt = 0.01, steady
    parabolic inlet of peak 1, and M = 2000 wall points, which puts the spacing
    ratio a = sqrt(dS)/h at 1.06 (x, y) and 1.27 (z), the regime of the paper's
    Table 1 (a = 0.98).  At M = 4000 (a = 0.75) the force matrix A_F of Eq. 22 is
    numerically rank-deficient on this grid (Sec. 2.5 warns of exactly this).
    """
    origin = (-half_width, -half_width, 0.0)
    extent = (2.0 * half_width, 2.0 * half_width, float(length))
    X, dS = cylinder_wall_points(R, 0.0, length, M, seed)
    xc, yc, zc = cell_centres(origin, extent, n)
    inside = (np.hypot(xc, yc) < R).astype(np.uint8)
    ports = [
        _port(2, 0, (0.0, 0.0, 0.0), R, INLET, a0=a0, b=b, period=period),
        _port(2, 1, (0.0, 0.0, length), R, OUTLET),
    ]
    return {
        "name": name or f"cylinder_{n[0]}x{n[1]}x{n[2]}_L{max_level}",
        "origin": origin, "extent": extent, "n": tuple(int(v) for v in n),
        "max_level": int(max_level), "refine_band": int(refine_band),
        "reduce_band": int(reduce_band),
        "nu": float(nu), "rho": 1.0, "dt": float(dt), "steps": int(steps),
        "ports": ports, "X": X, "dS": dS, "UB": np.zeros_like(X),
        "inside": inside,
    }


def cylinder_uniform_16x16x64(**kw):
    """Uniform 16x16x64 cylinder, Re 10, dt 0.01, 50 steps, FP64."""
    return cylinder_case(**kw)


def cylinder_refined_64x64x256(**kw):
    """64x64x256 cylinder, one refinement level in a 2h band around the wall,
    cells more than 2h outside the wall dropped, 32k points, pulsatile inflow
    u_max(t) = 1 + 0.5 sin(2 pi t), nu = 0.02, dt = 0.002, 1000 steps."""
    args = dict(n=(64, 64, 256), M=32000, seed=2, max_level=1, refine_band=2,
                reduce_band=2, nu=0.02, dt=0.002, steps=1000, a0=1.0, b=(0.5,),
                period=1.0, name="cylinder_64x64x256_L1")
    args.update(kw)
    return cylinder_case(**args)


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

