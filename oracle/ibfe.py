"""CPU FP64 oracle of the IB-FE-IPCS time step (immersed boundary finite elements).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU legs of
bench.py (cpu_baseline and --impl reference) import this module.  The product
path (the CUDA library and its Python binding) never imports or calls it, and it
shares no code, table or helper with that path.

What it computes, in the paper's order and notation:

  Step 1 (Sec. 2.2, Eq. 9)   tentative velocity u~ from the semi-implicit Oseen
                             problem with the old pressure p^n;
  Steps 2-4 (Sec. 2.3-2.4)   BCE-IB correction: delta kernel of Eq. 18, the
                             force system A_F F = B_F of Eq. 21-24, spreading of
                             Eq. 19 and the velocity update of Eq. 14;
  Step 5 (Eq. 12)            pressure-increment Poisson problem for Phi;
  Step 6 (Sec. 2.2)          velocity correction and p^{n+1} = p^n + Phi.

Discretisation: P1/P1 tetrahedra (Sec. 4, element pair) on a Cartesian box whose
cells are split into the six Kuhn tetrahedra around the (0,0,0)-(1,1,1)
diagonal (the box-mesh vertex grid of Sec. 3.1; Table 1's node and element
counts), with optional nested local refinement near the wall (Sec. 3.2) and
domain reduction (Sec. 4.3).  Matrices are assembled element by element with
generic P1 shape functions (inverse of the 4x4 vertex matrix); hanging nodes are
removed by the constraint matrix P (A_c = P^T A P); linear systems are solved
directly (SuperLU) or, for large systems, by CG/BiCGStab to stagnation.

Readings taken where the paper is silent, ambiguous or garbled (each is listed
with its reason in the project's design notes):
  R1  velocity update u^{n+1} = u - dt grad Phi (the printed '+' contradicts
      Eq. 10-12), done as the consistent-mass L2 projection;
  R2  Eq. 14: u = u~ + dt f / rho (the printed step 4 divides u~ by rho too);
  R3  the predictor is Eq. 9 (semi-implicit), not the explicit Eq. 13;
  R4  A_F[i,k] = (dt/rho) h^-3 dS_k sum_j w_ij w_kj (dS on the columns, as
      Eq. 19 implies); identical to Eq. 22 when dS is uniform;
  R5  per-axis spacing h_x, h_y, h_z in the 1-D kernel factors, h^3 -> hx hy hz
      of the finest level;
  R6  kinematic pressure (rho = 1 in every synthetic case);
  R7  viscous term nu (grad u, grad v) (equal to div 2 nu eps(u) for a
      divergence-free field; do-nothing outlet); with case["viscous"] ==
      "sym" the symmetric form 2 nu (eps(u), eps(v)) of Eq. 1 and Eq. 9, minus
      the boundary term nu ((grad u)^T n, v) on the outlet and pressure-inlet
      faces, which keeps the do-nothing condition of the gradient form;
  R9  Phi = 0 on outlet-port nodes; on pressure-inlet nodes Phi takes the
      increment p_in(t^{n+1}) - p^n that brings p^{n+1} to the imposed inlet
      pressure; homogeneous Neumann elsewhere;
  R10 port nodes: on the port face with dx^2 + dy^2 <= R^2 in FP64, no FMA;
      other boundary nodes of the active region are no-slip walls; outlet and
      pressure-inlet nodes carry no velocity condition (the natural condition
      nu du/dn = 0 of the gradient-form viscous term, as at a do-nothing
      outlet); opt-in case["port_tangential"] = "zero" holds their tangential
      components at zero instead (the paper is silent on them);
  R11 refinement level per coarse cell from the Chebyshev distance d to a
      point-containing coarse cell, hanging nodes constrained to the mean of the
      two ends of the coarse edge (cube edge or Kuhn face diagonal) they bisect;
  R12 active coarse cells: inside, or d <= reduce_band;
  R13 missing support nodes weigh zero; the force is spread only to free nodes
      (not Dirichlet, not hanging) and A_F uses those free nodes;
  R16 initial state u = 0, p = 0 unless given;
  R17 the Poisson right-hand side uses the IB-corrected velocity (step 5).
Dirichlet conditions apply to non-hanging nodes only: a hanging node always
takes the mean of its parents.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# The six Kuhn tetrahedra of a cell: the path v0 -> v0+e_a -> +e_b -> +e_c for
# every permutation (a, b, c) of the axes.
KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))

DIRECT_MAX_DOF = 60_000        # above this, Krylov solves replace SuperLU
DENSE_AF_MAX = 8_000           # the paper's direct solver for A_F up to this M


# --------------------------------------------------------------------------
# Eq. 18: the 4-point kernel of Lai and Peskin
# --------------------------------------------------------------------------
def delta4(r):
    """delta(r) of Eq. 18, vectorised."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    m1 = r <= 1.0
    m2 = (r > 1.0) & (r <= 2.0)
    a = r[m1]
    out[m1] = (3.0 - 2.0 * a + np.sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0
    a = r[m2]
    out[m2] = (5.0 - 2.0 * a - np.sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0
    return out


def inflow_peak(port, t):
    """Port waveform a0 + sum_k a_k cos(k w t) + b_k sin(k w t): the peak inlet
    speed u_max(t) of a velocity inlet, the pressure p_in(t) of a pressure
    inlet."""
    w = 2.0 * math.pi / port["period"]
    u = port["a0"]
    for k, ak in enumerate(port["a"], start=1):
        u += ak * math.cos(k * w * t)
    for k, bk in enumerate(port["b"], start=1):
        u += bk * math.sin(k * w * t)
    return u


# --------------------------------------------------------------------------
# Grid: level map, active cells, leaf cells, nodes, hanging nodes, flags
# --------------------------------------------------------------------------
def _shift(a, d, fill):
    """out[z,y,x] = a[z+dz, y+dy, x+dx] (fill outside)."""
    out = np.full_like(a, fill)
    src = []
    dst = []
    for ax, s in zip((0, 1, 2), (d[2], d[1], d[0])):
        n = a.shape[ax]
        if s >= 0:
            src.append(slice(s, n))
            dst.append(slice(0, n - s))
        else:
            src.append(slice(0, n + s))
            dst.append(slice(-s, n))
    out[tuple(dst)] = a[tuple(src)]
    return out


def chebyshev_distance(seed_mask, rmax):
    """Chebyshev (26-neighbour) distance in cells to the nearest seed cell,
    capped at rmax + 1."""
    cap = rmax + 1
    d = np.where(seed_mask, 0, cap).astype(np.int32)
    reached = seed_mask.copy()
    for r in range(1, rmax + 1):
        grown = reached.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == dy == dz == 0:
                        continue
                    grown |= _shift(reached, (dx, dy, dz), False)
        new = grown & ~reached
        d[new] = r
        reached = grown
    return d


@dataclass
class Mesh:
    """The composite (refined, reduced) mesh and its node bookkeeping."""
    case: dict
    L: int
    n: np.ndarray                 # coarse cells per axis (x, y, z)
    origin: np.ndarray
    h0: np.ndarray                # coarse spacing per axis
    hf: np.ndarray                # finest spacing per axis
    point_cell: np.ndarray        # (M, 3) coarse cell of each point
    dist: np.ndarray              # [nz, ny, nx] Chebyshev distance
    level: np.ndarray             # [nz, ny, nx] level map
    active: np.ndarray            # [nz, ny, nx] bool
    leaf_corner: np.ndarray       # (C, 3) finest-index lower corner of leaf cells
    leaf_size: np.ndarray         # (C,) edge length in finest index units
    node_q: np.ndarray            # (N, 3) finest integer coordinates, canonical order
    node_x: np.ndarray            # (N, 3) physical coordinates
    tets: np.ndarray              # (T, 4) node indices (Kuhn path order)
    hanging: np.ndarray           # (N,) bool
    parents: np.ndarray           # (N, 2) parent nodes of hanging nodes (-1 else)
    boundary: np.ndarray          # (N,) bool, on the boundary of the active region
    inlet: np.ndarray             # (N,) port index + 1 of a velocity-inlet port, 0 else
    pinlet: np.ndarray            # (N,) port index + 1 of a pressure-inlet port, 0 else
    outlet: np.ndarray            # (N,) bool
    node_level: np.ndarray        # (N,) coarsest level among leaf cells touching the node
    dof: np.ndarray               # (N,) DOF index of non-hanging nodes (-1 for hanging)
    P: sp.csr_matrix = field(repr=False, default=None)   # (N, Ndof)

    @property
    def n_nodes(self):
        return self.node_q.shape[0]

    @property
    def n_dof(self):
        return int(self.P.shape[1])

    def key(self, q):
        nf = self.n * (1 << self.L) + 1
        q = np.asarray(q, dtype=np.int64)
        return (q[..., 2] * nf[1] + q[..., 1]) * nf[0] + q[..., 0]

    def lookup(self, q):
        """Node index of finest coordinates q (..., 3); -1 where there is no node."""
        keys = self.key(q)
        sorted_keys = self._keys
        pos = np.searchsorted(sorted_keys, keys)
        pos = np.clip(pos, 0, len(sorted_keys) - 1)
        ok = sorted_keys[pos] == keys
        inb = np.all((np.asarray(q) >= 0) & (np.asarray(q) <= self.n * (1 << self.L)), axis=-1)
        return np.where(ok & inb, pos, -1)


def level_map(case):
    """Coarse-cell maps of the grid generation (Sec. 3.2 refinement, Sec. 4.3
    domain reduction; readings R11-R12): the point cell of every Lagrangian
    point, the Chebyshev distance to the nearest point cell, the 2:1-balanced
    refinement level and the active mask, all [nz][ny][nx]."""
    L = int(case["max_level"])
    n = np.array(case["n"], dtype=np.int64)
    origin = np.array(case["origin"], dtype=np.float64)
    extent = np.array(case["extent"], dtype=np.float64)
    h0 = extent / n
    X = np.asarray(case["X"], dtype=np.float64)
    nx, ny, nz = (int(v) for v in n)

    # coarse cell of every Lagrangian point
    pc = np.floor((X - origin) / h0).astype(np.int64) if len(X) else np.zeros((0, 3), np.int64)
    if len(X) and (np.any(pc < 0) or np.any(pc >= n)):
        raise ValueError("a Lagrangian point lies outside the box")
    seed = np.zeros((nz, ny, nx), dtype=bool)
    if len(X):
        seed[pc[:, 2], pc[:, 1], pc[:, 0]] = True

    B = max(1, int(case["refine_band"]))
    rb = int(case["reduce_band"])
    rmax = max(B * L + 1, rb, 1)
    dist = chebyshev_distance(seed, rmax)

    # R11: level map, then 2:1 balance over the 26-neighbourhood
    k = np.where(dist <= B, 0, -((-(dist - B)) // B))
    level = np.maximum(0, L - k).astype(np.int32)
    while True:
        nb = level.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    nb = np.maximum(nb, _shift(level, (dx, dy, dz), 0))
        bal = np.maximum(level, nb - 1)
        if np.array_equal(bal, level):
            break
        level = bal

    # R12: domain reduction
    inside = np.asarray(case["inside"]).astype(bool)
    active = np.ones_like(inside) if rb < 0 else (inside | (dist <= rb))
    return pc, dist, level, active


def build_mesh(case):
    """Grid generation of Sec. 3 on the structured box (readings R10-R12)."""
    L = int(case["max_level"])
    n = np.array(case["n"], dtype=np.int64)
    origin = np.array(case["origin"], dtype=np.float64)
    extent = np.array(case["extent"], dtype=np.float64)
    h0 = extent / n
    hf = extent / (n * (1 << L)).astype(np.float64)
    pc, dist, level, active = level_map(case)

    # leaf cells (finest-index corners)
    corners = []
    sizes = []
    cz, cy, cx = np.nonzero(active)
    lev = level[cz, cy, cx]
    for l in range(L + 1):
        sel = lev == l
        if not np.any(sel):
            continue
        s = 1 << (L - l)
        base = np.stack([cx[sel], cy[sel], cz[sel]], axis=1) * (1 << L)
        m = 1 << l
        sub = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
        c = (base[:, None, :] + s * sub[None, :, :]).reshape(-1, 3)
        corners.append(c)
        sizes.append(np.full(len(c), s, dtype=np.int64))
    leaf_corner = np.concatenate(corners) if corners else np.zeros((0, 3), np.int64)
    leaf_size = np.concatenate(sizes) if sizes else np.zeros(0, np.int64)

    # nodes: distinct vertices of leaf cells, canonical order (z, y, x)
    off8 = np.array([[dx, dy, dz] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], dtype=np.int64)
    verts = (leaf_corner[:, None, :] + leaf_size[:, None, None] * off8[None]).reshape(-1, 3)
    nf = n * (1 << L) + 1
    vkeys = (verts[:, 2] * nf[1] + verts[:, 1]) * nf[0] + verts[:, 0]
    keys = np.unique(vkeys)
    node_q = np.stack([keys % nf[0], (keys // nf[0]) % nf[1], keys // (nf[0] * nf[1])], axis=1)
    node_x = origin + node_q * hf

    mesh = Mesh(case=case, L=L, n=n, origin=origin, h0=h0, hf=hf, point_cell=pc,
                dist=dist, level=level, active=active, leaf_corner=leaf_corner,
                leaf_size=leaf_size, node_q=node_q, node_x=node_x, tets=None,
                hanging=None, parents=None, boundary=None, inlet=None, pinlet=None, outlet=None,
                node_level=None, dof=None)
    mesh._keys = keys

    # Kuhn tetrahedra of every leaf cell
    tets = []
    for perm in KUHN_PERMS:
        v = [leaf_corner.copy()]
        cur = leaf_corner.copy()
        for ax in perm:
            cur = cur.copy()
            cur[:, ax] += leaf_size
            v.append(cur)
        tets.append(np.stack([mesh.lookup(q) for q in v], axis=1))
    tets = np.concatenate(tets) if len(leaf_corner) else np.zeros((0, 4), np.int64)
    assert np.all(tets >= 0)
    mesh.tets = tets

    # coarsest level touching each node
    node_level = np.full(len(keys), L + 1, dtype=np.int32)
    leaf_lev = (L - np.log2(leaf_size).round().astype(np.int32)) if len(leaf_size) else np.zeros(0, np.int32)
    vidx = mesh.lookup(verts).reshape(-1, 8)
    np.minimum.at(node_level, vidx.ravel(), np.repeat(leaf_lev, 8))
    mesh.node_level = node_level

    # R11: hanging nodes = midpoints of edges (12 cube edges, 6 Kuhn face
    # diagonals) of leaf cells that are themselves nodes
    hanging = np.zeros(len(keys), dtype=bool)
    parents = np.full((len(keys), 2), -1, dtype=np.int64)
    big = leaf_size >= 2
    bc, bs = leaf_corner[big], leaf_size[big]
    edges = []
    for a in range(3):
        o1, o2 = [b for b in range(3) if b != a]
        for s1 in (0, 1):
            for s2 in (0, 1):
                e0 = np.zeros(3, np.int64)
                e0[o1], e0[o2] = s1, s2
                e1 = e0.copy()
                e1[a] += 1
                edges.append((e0, e1))
    for c in range(3):                      # face normal axis c
        a, b = [x for x in range(3) if x != c]
        for side in (0, 1):
            e0 = np.zeros(3, np.int64)
            e0[c] = side
            e1 = e0.copy()
            e1[a] += 1
            e1[b] += 1
            edges.append((e0, e1))
    for e0, e1 in edges:
        q0 = bc + bs[:, None] * e0
        q1 = bc + bs[:, None] * e1
        mid = (q0 + q1) // 2
        hit = mesh.lookup(mid)
        sel = hit >= 0
        if np.any(sel):
            h = hit[sel]
            hanging[h] = True
            parents[h, 0] = mesh.lookup(q0[sel])
            parents[h, 1] = mesh.lookup(q1[sel])
    if np.any(hanging):
        hp = parents[hanging]
        if np.any(hp < 0) or np.any(hanging[hp.ravel()]):
            raise ValueError("hanging node with a missing or hanging parent")
    mesh.hanging = hanging
    mesh.parents = parents

    # boundary of the active region: a node is interior iff the 8 coarse cells
    # around it (one per octant) are all active
    Lf = 1 << L
    boundary = np.zeros(len(keys), dtype=bool)
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                s = np.array([sx, sy, sz])
                c = (2 * node_q + s) // (2 * Lf)
                inb = np.all((c >= 0) & (c < n), axis=1)
                cc = np.clip(c, 0, n - 1)
                act = active[cc[:, 2], cc[:, 1], cc[:, 0]]
                boundary |= ~(inb & act)
    mesh.boundary = boundary

    # R10: port nodes
    inlet = np.zeros(len(keys), dtype=np.int32)
    pinlet = np.zeros(len(keys), dtype=np.int32)
    outlet = np.zeros(len(keys), dtype=bool)
    nfine = n * Lf
    for pi, port in enumerate(case["ports"]):
        a = port["axis"]
        plane = 0 if port["side"] == 0 else nfine[a]
        on = node_q[:, a] == plane
        o = [b for b in range(3) if b != a]
        d0 = node_x[:, o[0]] - port["center"][o[0]]
        d1 = node_x[:, o[1]] - port["center"][o[1]]
        r2 = d0 * d0
        r2 = r2 + d1 * d1
        sel = on & boundary & (r2 <= port["radius"] * port["radius"]) & (inlet == 0) & (pinlet == 0) & ~outlet
        if port["kind"] == "inlet":
            inlet[sel] = pi + 1
        elif port["kind"] == "pinlet":
            pinlet[sel] = pi + 1
        else:
            outlet[sel] = True
    inlet[hanging] = 0
    pinlet[hanging] = 0
    outlet[hanging] = False
    mesh.inlet = inlet
    mesh.pinlet = pinlet
    mesh.outlet = outlet

    # DOFs and the constraint matrix P (hanging node = mean of its parents)
    dof = np.full(len(keys), -1, dtype=np.int64)
    nh = ~hanging
    dof[nh] = np.arange(int(nh.sum()))
    rows = [np.nonzero(nh)[0]]
    cols = [dof[nh]]
    vals = [np.ones(int(nh.sum()))]
    hidx = np.nonzero(hanging)[0]
    for j in (0, 1):
        rows.append(hidx)
        cols.append(dof[parents[hidx, j]])
        vals.append(np.full(len(hidx), 0.5))
    mesh.P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(len(keys), int(nh.sum())))
    mesh.dof = dof
    return mesh


def velocity_dirichlet(mesh):
    """Non-hanging nodes with a velocity condition: walls and velocity inlets
    (R10)."""
    return (mesh.boundary & ~mesh.outlet & (mesh.pinlet == 0) & ~mesh.hanging) | (mesh.inlet > 0)


def velocity_dirichlet_components(mesh):
    """(N, 3) bool: the velocity condition per component.  Every component of a
    wall or velocity-inlet node (R10).  With case["port_tangential"] == "zero"
    also the components tangential to an outlet or pressure-inlet port on its
    nodes (held at zero): Sec. 3.1 imposes the pressure on the ports and says
    nothing of the tangential velocity there; the default ("free") leaves
    every component of a port node free, as R10 reads it."""
    d = np.repeat(velocity_dirichlet(mesh)[:, None], 3, axis=1)
    if mesh.case.get("port_tangential", "free") != "zero":
        return d
    taken = np.zeros(mesh.n_nodes, dtype=bool)
    for pi, port in enumerate(mesh.case["ports"]):
        a = port["axis"]
        plane = 0 if port["side"] == 0 else int(mesh.n[a]) << mesh.L
        o = [b for b in range(3) if b != a]
        d0 = mesh.node_x[:, o[0]] - port["center"][o[0]]
        d1 = mesh.node_x[:, o[1]] - port["center"][o[1]]
        r2 = d0 * d0
        r2 = r2 + d1 * d1
        sel = (mesh.node_q[:, a] == plane) & (r2 <= port["radius"] * port["radius"]) & ~taken
        sel &= mesh.outlet | (mesh.pinlet > 0) | (mesh.inlet > 0)
        taken |= sel
        if port["kind"] == "inlet":
            continue
        for k in o:
            d[sel & ~mesh.hanging, k] = True
    return d


def pressure_dirichlet(mesh):
    """Nodes where Phi is prescribed: outlets and pressure inlets (R9)."""
    return mesh.outlet | (mesh.pinlet > 0)


def phi_dirichlet_values(mesh, t, p):
    """Prescribed Phi at time t given the old pressure p (R9): p_in(t) - p on
    pressure-inlet nodes, so that p^{n+1} = p^n + Phi equals p_in there; zero
    on outlet nodes (and zero elsewhere)."""
    g = np.zeros(mesh.n_nodes)
    for pi, port in enumerate(mesh.case["ports"]):
        sel = mesh.pinlet == pi + 1
        if np.any(sel):
            g[sel] = inflow_peak(port, t) - p[sel]
    return g


def dirichlet_velocity_values(mesh, t):
    """Prescribed velocity at every node at time t: the parabolic inlet profile
    along the inward port normal, zero on walls (and zero elsewhere)."""
    g = np.zeros((mesh.n_nodes, 3))
    for pi, port in enumerate(mesh.case["ports"]):
        sel = mesh.inlet == pi + 1
        if not np.any(sel) or port["kind"] != "inlet":
            continue
        a = port["axis"]
        o = [b for b in range(3) if b != a]
        d0 = mesh.node_x[sel, o[0]] - port["center"][o[0]]
        d1 = mesh.node_x[sel, o[1]] - port["center"][o[1]]
        r2 = d0 * d0 + d1 * d1
        prof = inflow_peak(port, t) * (1.0 - r2 / (port["radius"] ** 2))
        g[sel, a] = prof if port["side"] == 0 else -prof
    return g


# --------------------------------------------------------------------------
# P1 element matrices, assembled element by element
# --------------------------------------------------------------------------
def tet_geometry(mesh):
    """Gradients of the 4 barycentric functions (T, 4, 3) and volumes (T,)."""
    xyz = mesh.node_x[mesh.tets]                         # (T, 4, 3)
    A = np.concatenate([np.ones(xyz.shape[:2] + (1,)), xyz], axis=2)   # rows [1, x_a]
    inv = np.linalg.inv(A)                               # phi_a coefficients in column a
    grads = np.transpose(inv[:, 1:, :], (0, 2, 1))       # (T, 4, 3)
    vol = np.abs(np.linalg.det(A)) / 6.0
    return grads, vol


def _assemble(mesh, Ke):
    T = mesh.tets
    r = np.repeat(T, 4, axis=1).ravel()
    c = np.tile(T, (1, 4)).ravel()
    N = mesh.n_nodes
    return sp.csr_matrix((Ke.ravel(), (r, c)), shape=(N, N))


class Operators:
    """Assembled all-node matrices: mass M, stiffness K, gradients G_k, and the
    convection matrix C(u) on demand."""

    def __init__(self, mesh):
        self.mesh = mesh
        grads, vol = tet_geometry(mesh)
        self.grads, self.vol = grads, vol
        eye = np.eye(4)
        self.M = _assemble(mesh, vol[:, None, None] * (1.0 + eye)[None] / 20.0)
        self.K = _assemble(mesh, vol[:, None, None] * np.einsum("tak,tbk->tab", grads, grads))
        # (d_k p, v_a) = sum_b p_b d_k phi_b |T| / 4
        self.G = [_assemble(mesh, np.broadcast_to((vol / 4.0)[:, None, None] * grads[:, None, :, k],
                                                  (len(vol), 4, 4)).copy()) for k in range(3)]
        self.P = mesh.P
        self.PT = mesh.P.T.tocsr()

    def transpose_blocks(self):
        """Kt[i][j][a, b] = int (d_j phi_a)(d_i phi_b): the blocks of
        (grad u^T : grad v) for test phi_a e_i and trial phi_b e_j, so that
        2 (eps(u), eps(v)) = (grad u, grad v) + sum_ij Kt[i][j] (Eq. 1 read with
        the symmetric strain rate)."""
        if not hasattr(self, "_kt"):
            g, v = self.grads, self.vol
            self._kt = [[_assemble(self.mesh, v[:, None, None] * np.einsum("ta,tb->tab", g[:, :, j], g[:, :, i]))
                         for j in range(3)] for i in range(3)]
        return self._kt

    def natural_boundary_blocks(self):
        """Bn[i][j][a, b] = int_F n_j (d_i phi_b) phi_a over the tetrahedron faces
        F lying in the plane of an outlet or pressure-inlet port (outward normal
        n = -e_axis on the low face, +e_axis on the high face), so that
        sum_ij Bn[i][j] u_j is the boundary term ((grad u)^T n, v).  Rows of
        nodes with a velocity condition are eliminated by the solve."""
        if hasattr(self, "_bn"):
            return self._bn
        m = self.mesh
        N = m.n_nodes
        rows = {(i, j): ([], [], []) for i in range(3) for j in range(3)}
        Lf = 1 << m.L
        for port in m.case["ports"]:
            if port["kind"] == "inlet":
                continue
            ax = port["axis"]
            plane = 0 if port["side"] == 0 else int(m.n[ax]) * Lf
            nrm = -1.0 if port["side"] == 0 else 1.0
            on = m.node_q[m.tets][:, :, ax] == plane                 # (T, 4)
            for t in np.nonzero(on.sum(axis=1) == 3)[0]:
                face = m.tets[t][on[t]]
                x = m.node_x[face]
                area = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
                for a in face:
                    for bi, b in enumerate(m.tets[t]):
                        for i in range(3):
                            r, cidx, val = rows[(i, ax)]
                            r.append(a)
                            cidx.append(b)
                            val.append(nrm * self.grads[t, bi, i] * area / 3.0)
        self._bn = [[sp.csr_matrix((np.asarray(rows[(i, j)][2], float),
                                    (np.asarray(rows[(i, j)][0], np.int64), np.asarray(rows[(i, j)][1], np.int64))),
                                   shape=(N, N)) for j in range(3)] for i in range(3)]
        return self._bn

    def convection(self, u):
        """C(u)[a, b] = int_T (u_h . grad phi_b) phi_a, u_h the P1 interpolant."""
        uT = u[self.mesh.tets]                                  # (T, 4, 3)
        s = uT.sum(axis=1, keepdims=True)                       # sum_c u_c
        ubar = (self.vol / 20.0)[:, None, None] * (s + uT)      # sum_c u_c |T| (1+d_ac)/20
        Ce = np.einsum("tak,tbk->tab", ubar, self.grads)
        return _assemble(self.mesh, Ce)

    def condense(self, A):
        return (self.PT @ A @ self.P).tocsr()


# --------------------------------------------------------------------------
# Linear solves with Dirichlet elimination
# --------------------------------------------------------------------------
def _krylov(A, b, symmetric, rtol=1e-13):
    d = A.diagonal()
    Minv = sp.diags(1.0 / d)
    x = np.zeros_like(b)
    for j in range(b.shape[1]):
        if symmetric:
            xj, info = spla.cg(A, b[:, j], rtol=rtol, atol=0.0, maxiter=20000, M=Minv)
        else:
            xj, info = spla.bicgstab(A, b[:, j], rtol=rtol, atol=0.0, maxiter=20000, M=Minv)
        x[:, j] = xj
    return x


def solve_dirichlet(A, b, dmask, g, symmetric, factor_cache=None, key=None):
    """Solve A x = b for the free DOFs with x = g on the Dirichlet DOFs
    (symmetric elimination).  b, g: (Ndof, k)."""
    F = ~dmask
    D = dmask
    x = np.array(g, dtype=np.float64, copy=True)
    AFF = A[F][:, F].tocsc()
    rhs = b[F] - A[F][:, D] @ g[D]
    if AFF.shape[0] == 0:
        return x
    if AFF.shape[0] <= DIRECT_MAX_DOF:
        lu = None
        if factor_cache is not None and key in factor_cache:
            lu = factor_cache[key]
        if lu is None:
            lu = spla.splu(AFF, permc_spec="MMD_AT_PLUS_A")
            if factor_cache is not None and key is not None:
                factor_cache[key] = lu
        x[F] = lu.solve(np.ascontiguousarray(rhs))
    else:
        x[F] = _krylov(AFF, rhs, symmetric)
    return x


# --------------------------------------------------------------------------
# BCE-IB (Sec. 2.3): weights, interpolation, force system, spreading
# --------------------------------------------------------------------------
class IB:
    """Interpolation matrix W (M x N, all existing support nodes), its free-node
    part W_f, and the force matrix A_F (Eq. 22, reading R4)."""

    def __init__(self, mesh, case, free):
        X = np.asarray(case["X"], dtype=np.float64)
        self.dS = np.asarray(case["dS"], dtype=np.float64)
        self.UB = np.asarray(case["UB"], dtype=np.float64)
        self.M = len(X)
        hf = mesh.hf
        self.h3 = hf[0] * hf[1] * hf[2]
        # support origin: floor((X - x0)/h) - 1 on the finest grid (R13)
        self.origin = (np.floor((X - mesh.origin) / hf).astype(np.int64) - 1) if self.M else np.zeros((0, 3), np.int64)
        off = np.array([[a, b, c] for c in range(4) for b in range(4) for a in range(4)], dtype=np.int64)
        q = self.origin[:, None, :] + off[None]                         # (M, 64, 3)
        idx = mesh.lookup(q)                                            # -1 = missing
        xn = mesh.origin + q * hf
        w = (delta4((xn[..., 0] - X[:, None, 0]) / hf[0])
             * delta4((xn[..., 1] - X[:, None, 1]) / hf[1])
             * delta4((xn[..., 2] - X[:, None, 2]) / hf[2]))
        exists = idx >= 0
        if np.any(exists):
            sup = idx[exists]
            if np.any(mesh.hanging[sup]) or np.any(mesh.node_level[sup] != mesh.L):
                raise ValueError("an IB support crosses a hanging or coarser-level node")
        self.support_idx = idx
        self.weights = np.where(exists, w, 0.0)
        rows = np.repeat(np.arange(self.M), 64)[exists.ravel()]
        cols = idx.ravel()[exists.ravel()]
        vals = w.ravel()[exists.ravel()]
        N = mesh.n_nodes
        self.W = sp.csr_matrix((vals, (rows, cols)), shape=(self.M, N))
        fsel = free[cols]
        self.Wf = sp.csr_matrix((vals[fsel], (rows[fsel], cols[fsel])), shape=(self.M, N))
        dt, rho = case["dt"], case["rho"]
        # A_F[i,k] = (dt/rho) h^-3 dS_k sum_j w_ij w_kj
        S = (self.Wf @ self.Wf.T).tocsr() * (dt / (rho * self.h3))
        self.AF = (S @ sp.diags(self.dS)).tocsr()
        self._lu = None

    def solve_force(self, BF):
        """Solve A_F F = B_F (the paper's direct solver, Sec. 2.3)."""
        if self.M == 0:
            return np.zeros((0, 3))
        if self.M <= DENSE_AF_MAX:
            if self._lu is None:
                self._lu = sla.lu_factor(self.AF.toarray())
            return sla.lu_solve(self._lu, BF)
        if self._lu is None:
            self._lu = spla.splu(self.AF.tocsc())
        return self._lu.solve(np.ascontiguousarray(BF))

    def spread(self, F):
        """f(x_j) = sum_i F_i D_ij dS_i on free nodes (Eq. 19), D = w / h^3."""
        return (self.Wf.T @ (F * self.dS[:, None])) / self.h3


# --------------------------------------------------------------------------
# Sec. 2.6: wall shear stress by DC-PSE derivatives at the wall points
# --------------------------------------------------------------------------
# monomials z^alpha with 1 <= |alpha| <= 2, the first-degree ones first
_DCPSE_ALPHA = ((1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2))


def _monomials(z):
    return np.stack([z[:, 0] ** a[0] * z[:, 1] ** a[1] * z[:, 2] ** a[2] for a in _DCPSE_ALPHA], axis=1)


def finest_nodes(mesh):
    """Nodes that are vertices of a finest-level leaf cell."""
    flag = np.zeros(mesh.n_nodes, dtype=bool)
    fine = mesh.leaf_size == 1
    if np.any(fine):
        c = mesh.leaf_corner[fine]
        off = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)])
        idx = mesh.lookup((c[:, None, :] + off[None]).reshape(-1, 3))
        flag[idx[idx >= 0]] = True
    return flag


def wall_shear_stress(mesh, u, X, UB, normals, nu, rho=1.0, radius=3.5):
    """WSS at the wall points (Sec. 2.6): |t - (t.n) n| with t = 2 mu eps(u) n,
    eps_ij = (d_j u_i + d_i u_j) / 2, mu = rho nu, n the unit outward normal.

    The derivatives are DC-PSE operators (the method Sec. 2.6 cites) of second
    order: d_j f(X_p) = (1/e) sum_q (f_q - f_p) eta_j(z_q), z_q = (x_q - X_p)/e,
    eta_j(z) = sum_alpha a_alpha z^alpha exp(-|z|^2) over the nine monomials
    1 <= |alpha| <= 2, the coefficients from the discrete moment conditions
    sum_q z_q^beta eta_j(z_q) = delta(beta, e_j), so polynomials of degree 2
    are differentiated exactly.  Readings: e = the largest finest spacing; the
    point cloud is the finest-level nodes q with |x_q - X_p| <= radius e on the
    fluid side, (x_q - X_p).n < 0, distances and projections summed x, y, z
    without fused multiply-add; f_p = U_B (no-slip at the wall).
    Returns wss (M,) and grad (M, 3, 3), grad[p, i, j] = d u_i / d x_j."""
    X = np.asarray(X, dtype=np.float64)
    UB = np.asarray(UB, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    e = float(np.max(mesh.hf))
    rc2 = (radius * e) * (radius * e)
    cand = np.nonzero(finest_nodes(mesh))[0]
    cx = mesh.node_x[cand]
    M = len(X)
    grad = np.zeros((M, 3, 3))
    for p in range(M):
        d = cx - X[p]
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        r2 = r2 + d[:, 2] * d[:, 2]
        dn = d[:, 0] * nrm[p, 0] + d[:, 1] * nrm[p, 1]
        dn = dn + d[:, 2] * nrm[p, 2]
        sel = (r2 <= rc2) & (dn < 0.0)
        z = d[sel] / e
        P = _monomials(z)
        w = np.exp(-(z * z).sum(axis=1))
        A = (P * w[:, None]).T @ P
        coef = np.linalg.solve(A, np.eye(9)[:, :3])              # (9, 3): eta_1, eta_2, eta_3
        eta = (P @ coef) * w[:, None]                             # (n, 3)
        du = u[cand[sel]] - UB[p]                                 # (n, 3)
        grad[p] = du.T @ eta / e
    S = 0.5 * (grad + np.transpose(grad, (0, 2, 1)))
    t = 2.0 * rho * nu * np.einsum("pij,pj->pi", S, nrm)
    ts = t - np.einsum("pi,pi->p", t, nrm)[:, None] * nrm
    return np.sqrt((ts * ts).sum(axis=1)), grad


# --------------------------------------------------------------------------
# The IPCS step with the BCE-IB correction (Sec. 2.4)
# --------------------------------------------------------------------------
class Oracle:
    """Runs the combined algorithm of Sec. 2.4 on one synthetic case."""

    def __init__(self, case, u0=None, p0=None):
        self.case = case
        self.mesh = build_mesh(case)
        self.ops = Operators(self.mesh)
        m = self.mesh
        self.vdir_node = velocity_dirichlet(m)
        self.vdir = self.vdir_node[~m.hanging]
        # per component: differs from vdir only on pressure ports when their
        # tangential velocity is held at zero
        vdir_c = velocity_dirichlet_components(m)
        self.vdir_c = vdir_c[~m.hanging]
        self.split = not all(np.array_equal(self.vdir_c[:, k], self.vdir) for k in range(3))
        if self.split:
            self.vdir_node = vdir_c.any(axis=1)   # the force spreads to nodes free in every component
        self.pdir = pressure_dirichlet(m)[~m.hanging]
        free = ~self.vdir_node & ~m.hanging
        self.ib = IB(m, case, free)
        N = m.n_nodes
        self.u = np.zeros((N, 3)) if u0 is None else np.array(u0, dtype=np.float64)
        self.p = np.zeros(N) if p0 is None else np.array(p0, dtype=np.float64)
        self.F = np.zeros((self.ib.M, 3))
        self.phi = np.zeros(N)
        self.t = 0.0
        self.nstep = 0
        self._cache = {}
        self.Kc = self.ops.condense(self.ops.K)
        self.Mc = self.ops.condense(self.ops.M)

    def _dof(self, v):
        return v[~self.mesh.hanging]

    def set_points(self, X, UB=None):
        """Moving or deforming wall: the Lagrangian points take positions X
        (M, 3) and prescribed velocities U_B (zero if None) for the following
        steps; the supports, W, W_f and A_F are rebuilt there (Eq. 17-22 at the
        new positions; the area elements dS stay).  The IB method's reason to
        exist is that the Eulerian grid does not follow the wall (Sec. 1)."""
        X = np.asarray(X, dtype=np.float64)
        if X.shape != (self.ib.M, 3):
            raise ValueError("set_points keeps the number of points")
        case = dict(self.case)
        case["X"] = X
        case["UB"] = np.zeros_like(X) if UB is None else np.asarray(UB, dtype=np.float64)
        self.case = case
        self.ib = IB(self.mesh, case, ~self.vdir_node & ~self.mesh.hanging)

    def step(self):
        m, ops, c = self.mesh, self.ops, self.case
        dt, nu, rho = c["dt"], c["nu"], c["rho"]
        t1 = self.t + dt
        g_all = dirichlet_velocity_values(m, t1)
        g = self._dof(g_all)

        # Step 1, Eq. 9: (M + dt C(u^n) + dt nu K) u~ = M u^n - dt G p^n
        Am = ops.M + dt * ops.convection(self.u) + (dt * nu) * ops.K
        b = np.stack([ops.PT @ (ops.M @ self.u[:, k] - dt * (ops.G[k] @ self.p)) for k in range(3)], 1)
        if c.get("viscous", "grad") == "sym":
            ut = self._momentum_sym(Am, b, g, dt * nu)
        else:
            Ac = ops.condense(Am)
            ut = ops.P @ self._solve_velocity(Ac, b, g, symmetric=False)

        # Steps 2-3: B_F = U_B - h^3 D^T u~ (Eq. 23), A_F F = B_F (Eq. 21)
        BF = self.ib.UB - self.ib.W @ ut
        F = self.ib.solve_force(BF)
        # Step 4, Eq. 14 (R2): u = u~ + dt f / rho, f from Eq. 19
        u = ut + (dt / rho) * self.ib.spread(F)

        # Step 5, Eq. 12: (grad Phi, grad q) = -(1/dt) (div u, q), Phi = 0 at
        # outlets and p_in(t^{n+1}) - p^n at pressure inlets (R9)
        div = sum(ops.G[k] @ u[:, k] for k in range(3))
        bp = (ops.PT @ (-(1.0 / dt) * div))[:, None]
        gp = self._dof(phi_dirichlet_values(m, t1, self.p))[:, None]
        phi = ops.P @ solve_dirichlet(self.Kc, bp, self.pdir, gp, symmetric=True,
                                      factor_cache=self._cache, key="K")[:, 0]

        # Step 6 (R1): (u^{n+1}, v) = (u, v) - dt (grad Phi, v); p^{n+1} = p^n + Phi
        bc = np.stack([ops.PT @ (ops.M @ u[:, k] - dt * (ops.G[k] @ phi)) for k in range(3)], 1)
        un = ops.P @ self._solve_velocity(self.Mc, bc, g, symmetric=True, key="M")
        self.ut, self.u_ib, self.BF = ut, u, BF
        self.u = un
        self.p = self.p + phi
        self.phi = phi
        self.F = F
        self.t = t1
        self.nstep += 1

    def _solve_velocity(self, A, b, g, symmetric, key=None):
        """The three velocity components with their Dirichlet rows; one solve
        for all three when every component has the same condition."""
        cache = self._cache if key is not None else None
        if not self.split:
            return solve_dirichlet(A, b, self.vdir, g, symmetric, factor_cache=cache, key=key)
        return np.stack([solve_dirichlet(A, b[:, k:k + 1], self.vdir_c[:, k], g[:, k:k + 1], symmetric,
                                         factor_cache=cache, key=None if key is None else f"{key}{k}")[:, 0]
                         for k in range(3)], axis=1)

    def _momentum_sym(self, Am, b, g, dtnu):
        """Eq. 9 with the symmetric viscous form (R7): the three components
        couple through dt nu (Kt - Bn); one block system on 3 Ndof unknowns,
        component-major."""
        ops = self.ops
        Kt, Bn = ops.transpose_blocks(), ops.natural_boundary_blocks()
        blocks = [[ops.condense((Am if i == j else 0 * Am) + dtnu * (Kt[i][j] - Bn[i][j])) for j in range(3)]
                  for i in range(3)]
        A3 = sp.bmat(blocks, format="csr")
        nd = b.shape[0]
        d3 = np.concatenate([self.vdir_c[:, k] for k in range(3)])
        x3 = solve_dirichlet(A3, b.T.reshape(-1, 1), d3, g.T.reshape(-1, 1), symmetric=False)[:, 0]
        return ops.P @ x3.reshape(3, nd).T

    def run(self, steps):
        for _ in range(steps):
            self.step()
        return self
