"""Host-side multigrid hierarchy of the Poisson preconditioner (csrc/mg.cpp).

Compiled with a small driver (tests/mg_probe.cpp); no GPU needed.  The
hierarchy is pinned against what the discretisation fixes independently of
the builder:

  * G0 operator = P0^T K P0 with K the oracle's own element-by-element
    stiffness over all nodes (hanging nodes expanded as the mean of their
    parents): the Galerkin identity of nested P1 spaces (Sec. 3.2 refinement
    keeps the spaces nested);
  * every coarser operator = P^T A P of the level below (Galerkin);
  * both identities hold exactly away from the outlet nodes (Phi = 0, Eq. 12);
    next to them the coarse Dirichlet rule (injection, where the outlet lies on
    the coarse lattice) is an approximation, so those rows are skipped;
  * where the outlet plane falls between coarse lattice planes (odd cell
    count) a coarse node is removed when its interpolation reaches a finer
    outlet node: the coarse space is nested and the identity holds on every
    row;
  * prolongation is P1 interpolation: it reproduces linear functions;
  * restriction is the transpose of prolongation on owner copies;
  * operators are symmetric with zero row sums away from Dirichlet nodes.
"""
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import ibfe
from tests.test_host_setup import _desc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_02082_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("mgprobe")
    exe = d / "mg_probe"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, os.path.join(CSRC, "setup.cpp"), os.path.join(CSRC, "mg.cpp"),
                    os.path.join(ROOT, "tests", "mg_probe.cpp"), "-o", str(exe)], check=True)
    return exe, d


def run_probe(probe, case):
    exe, d = probe
    inp, out = d / "in.bin", d / "out.bin"
    with open(inp, "wb") as f:
        f.write(bytes(_desc(case)))
        f.write(np.int64(len(case["X"])).tobytes())
        for k in ("X", "dS", "UB"):
            f.write(np.ascontiguousarray(case[k], np.float64).tobytes())
        f.write(np.ascontiguousarray(case["inside"], np.uint8).tobytes())
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    b = open(out, "rb").read()
    pos = [0]

    def take(n, dt):
        dt = np.dtype(dt)
        v = np.frombuffer(b, dt, count=n, offset=pos[0])
        pos[0] += n * dt.itemsize
        return v

    ok, nlev, small, ns, N = (int(v) for v in take(5, np.int64))
    res = {"ok": ok, "small": small, "ns": ns, "canon_slot": take(N, np.int32),
           "slot_q": take(3 * ns, np.int32).reshape(ns, 3), "lev": []}
    for _ in range(nlev):
        nn, nd, nr, npe, n0, n1, n2 = (int(v) for v in take(7, np.int64))
        L = {"nn": nn, "n": (n0, n1, n2), "h": take(3, np.float64)}
        L["coord"] = take(3 * nn, np.int32).reshape(nn, 3)
        L["dir"] = take(3 * nd, np.int32).reshape(nd, 3)
        L["nbr"] = take(6 * nn, np.int32).reshape(nn, 6)
        L["offd"] = take(6 * nn, np.float64).reshape(nn, 6)
        L["diag"] = take(nn, np.float64)
        rptr = take(nn + 1, np.int32)
        L["R"] = (rptr, take(nr, np.int32), take(nr, np.float64))
        prow = int(take(1, np.int64)[0])
        pptr = take(prow, np.int32)
        L["P"] = (pptr, take(npe, np.int32), take(npe, np.float64))
        res["lev"].append(L)
    if ok:
        nb = int(take(1, np.int64)[0])
        wf = {"meta": take(ns, np.uint16), "blev": take(nb, np.int32), "bco": take(3 * nb, np.int32).reshape(nb, 3)}
        wf["lat_n"] = tuple(int(v) for v in take(3, np.int64))
        nl = int(take(1, np.int64)[0])
        wf["lat0"] = take(nl, np.int32)
        wf["npart"] = int(take(1, np.int64)[0])
        nn0 = res["lev"][0]["nn"]
        wf["pbase"] = take(nb, np.int32)
        wf["r0slot"] = take(nn0, np.int32)
        wf["r0ptr"] = take(nn0 + 1, np.int32)
        ni = int(take(1, np.int64)[0])
        wf["r0idx"] = take(ni, np.int32)
        res["wf"] = wf
    return res


def level_matrix(L):
    nn = L["nn"]
    rows, cols, vals = [np.arange(nn)], [np.arange(nn)], [L["diag"]]
    m = L["nbr"] >= 0
    r = np.repeat(np.arange(nn)[:, None], 6, axis=1)
    rows.append(r[m]), cols.append(L["nbr"][m]), vals.append(L["offd"][m])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nn, nn))


def csr(ptr, col, w, ncol):
    return sp.csr_matrix((w, col, ptr), shape=(len(ptr) - 1, ncol))


def far_from(coords, dirs, dist):
    if len(dirs) == 0:
        return np.ones(len(coords), bool)
    far = np.ones(len(coords), bool)
    for d in dirs:
        far &= np.abs(coords - d[None, :]).max(axis=1) > dist
    return far


CASES = {
    "uniform": W.cylinder_uniform_16x16x64(),
    "refined": W.cylinder_refined_small(n=(16, 16, 8), seed=21),
    "two_levels": W.cylinder_case(n=(24, 24, 8), length=1.0, half_width=0.75, M=1500, seed=12, max_level=2,
                                  refine_band=1, reduce_band=3, nu=0.02, dt=0.002, b=(0.5,)),
    # odd cell count along the outlet axis: the outlet plane falls between the
    # lattice planes of every coarser level
    "odd_outlet": W.cylinder_case(n=(12, 12, 37), length=3.7, half_width=0.6, M=800, seed=14, max_level=1,
                                  refine_band=1, reduce_band=2, nu=0.05, dt=0.005),
    # no immersed boundary (M = 0), Phi prescribed on a pressure inlet and an outlet
    "duct_no_points": {"name": "duct_8x8x24", "origin": (-0.5, -0.5, 0.0), "extent": (1.0, 1.0, 3.0),
                       "n": (8, 8, 24), "max_level": 0, "refine_band": 2, "reduce_band": -1, "nu": 0.1,
                       "rho": 1.0, "dt": 0.01,
                       "ports": [W._port(2, 0, (0.0, 0.0, 0.0), 0.499, W.PINLET, a0=1.0),
                                 W._port(2, 1, (0.0, 0.0, 3.0), 0.499, W.OUTLET)],
                       "X": np.zeros((0, 3)), "dS": np.zeros(0), "UB": np.zeros((0, 3)),
                       "inside": np.ones((24, 8, 8), np.uint8)},
    # the reduced synthetic aorta: five ports on two faces, branches, one level
    "aorta_small": W.aorta_case(n=(40, 40, 60), max_level=1, M=3000, seed=44, dt=0.002),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mg_levels_symmetric_and_galerkin(probe, name):
    case = CASES[name]
    res = run_probe(probe, case)
    assert res["ok"] == 1
    levs = res["lev"]
    assert len(levs) >= 2
    assert levs[-1]["nn"] <= 1024
    checked = 0
    for k, L in enumerate(levs):
        A = level_matrix(L)
        assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
        far = far_from(L["coord"], L["dir"], 1)
        rs = np.asarray(A.sum(axis=1)).ravel()
        assert np.abs(rs[far]).max() <= 1e-12 * abs(A).max()
        if k == 0:
            continue
        F = levs[k - 1]
        P = csr(*L["P"], L["nn"])                                # G(k) -> G(k-1)
        assert P.shape == (F["nn"], L["nn"])
        R = csr(*L["R"], F["nn"])
        assert abs(R - P.T).max() == 0.0
        Ag = (P.T @ level_matrix(F) @ P).tocsr()
        if name == "odd_outlet" and k == 1:   # G0 -> G1 by interpolation (37 cells): nested, every row
            assert abs(Ag - A).max() <= 1e-12 * abs(A).max(), (name, k)
            checked += 1
        else:
            far2 = np.nonzero(far_from(L["coord"], L["dir"], 2))[0]
            if len(far2):   # short domains: every node of the coarsest levels is near the outlet
                D = (Ag - A)[far2][:, far2]
                assert abs(D).max() <= 1e-12 * abs(A).max(), (name, k)
                checked += 1
        # P1 interpolation reproduces linear functions (rows away from Dirichlet)
        lin = lambda c, h: (c * h[None, :]) @ np.array([0.3, -1.1, 0.7])
        fine = P @ lin(L["coord"].astype(float), L["h"])
        full = np.asarray(P.sum(axis=1)).ravel() == 1.0
        assert full.sum() > 0.5 * F["nn"]
        assert np.abs(fine - lin(F["coord"].astype(float), F["h"]))[full].max() < 1e-12
    assert checked >= 1


@pytest.mark.parametrize("name", sorted(CASES))
def test_mg_g0_is_galerkin_of_oracle_stiffness(probe, name):
    case = CASES[name]
    res = run_probe(probe, case)
    L0 = res["lev"][0]
    m = ibfe.build_mesh(case)
    ops = ibfe.Operators(m)
    N = m.n_nodes
    P0 = csr(*L0["P"], L0["nn"])                                 # composite slot -> G0
    slot = res["canon_slot"]
    V = P0[slot].tolil()
    V[np.nonzero(m.outlet)[0], :] = 0
    V = V.tocsr()
    h = np.nonzero(m.hanging)[0]
    if len(h):
        par = m.parents[h]
        E = sp.identity(N, format="lil")
        for i, (a, b) in zip(h, par):
            E[i, i] = 0.0
            E[i, a] = 0.5
            E[i, b] = 0.5
        V = (E.tocsr() @ V).tocsr()
    A0 = level_matrix(L0)
    Ag = (V.T @ ops.K @ V).tocsr()
    far = np.nonzero(far_from(L0["coord"], L0["dir"], 2))[0]
    D = (Ag - A0)[far][:, far]
    assert abs(D).max() <= 1e-12 * abs(A0).max()
    # linear reproduction at every composite node (away from the outlet)
    h0 = L0["h"]
    hf = np.array(case["extent"]) / (np.array(case["n"]) * 2 ** case["max_level"])
    f = np.array([0.3, -1.1, 0.7])
    coarse = (L0["coord"] * h0[None, :]) @ f
    got = P0 @ coarse
    rows = np.nonzero(np.diff(P0.indptr) > 0)[0]
    full = np.asarray(P0[rows].sum(axis=1)).ravel() == 1.0
    want = (res["slot_q"][rows] * hf[None, :]) @ f
    assert np.abs(got[rows] - want)[full].max() < 1e-12
    # restriction = transpose of prolongation on owner copies
    R = csr(*L0["R"], res["ns"])
    owner = np.zeros(res["ns"], bool)
    owner[slot] = True
    Pown = P0.multiply(owner[:, None]).tocsr()
    assert abs(R - Pown.T).max() == 0.0


M_VALID, M_HANG, M_DUP, M_PDIR = 1 << 8, 1 << 9, 1 << 10, 1 << 12


def _hat(e, sc):
    """The G0 hat function of the Kuhn mesh at lattice offset e (level units,
    sc per coarse cell): 1 - (max(0, e) - min(0, e)) / sc, clipped at 0."""
    span = np.maximum(0, e.max(axis=-1)) - np.minimum(0, e.min(axis=-1))
    return np.clip(sc - span, 0, None) / sc


@pytest.mark.parametrize("name", sorted(CASES))
def test_weight_free_transfers_equal_the_stored_ones(probe, name):
    """The device computes the composite <-> G0 transfers from lattice
    positions instead of reading stored weights.  Rebuilt here from the
    tables the builder gives it (the G0 lattice map, each fine brick's
    partial sums and the G0 nodes they feed, the level-0 owner slots) with the
    hat-function weight, both transfers equal the stored CSR exactly."""
    res = run_probe(probe, CASES[name])
    assert res["ok"] == 1
    wf, L0 = res["wf"], res["lev"][0]
    ns, nn0 = res["ns"], L0["nn"]
    meta, blev, bco = wf["meta"].astype(np.int64), wf["blev"], wf["bco"].astype(np.int64)
    nx, ny, nz = wf["lat_n"]
    lat = wf["lat0"].reshape(nz, ny, nx)
    t = np.arange(512)
    local = np.stack([t & 7, (t >> 3) & 7, t >> 6], -1)
    owner = ((meta & M_VALID) != 0) & ((meta & (M_HANG | M_DUP | M_PDIR)) == 0)
    kept = ((meta & M_VALID) != 0) & ((meta & (M_HANG | M_PDIR)) == 0)
    # restriction
    rows, cols, vals = [], [], []
    for j in np.nonzero(wf["r0slot"] >= 0)[0]:
        rows.append([j]), cols.append([wf["r0slot"][j]]), vals.append([1.0])
    fine = np.nonzero(wf["pbase"] >= 0)[0]
    owner_brick = np.searchsorted(wf["pbase"][fine], np.arange(wf["npart"]), side="right") - 1
    for j in range(nn0):
        for p in wf["r0idx"][wf["r0ptr"][j]:wf["r0ptr"][j + 1]]:
            b = fine[owner_brick[p]]
            l = int(blev[b]); sc = 1 << l; T = (6 + sc) // sc + 1
            k = p - wf["pbase"][b]
            tq = np.array([k % T, (k // T) % T, k // (T * T)])
            Q = bco[b] * 8 // sc + tq
            assert lat[Q[2], Q[1], Q[0]] == j
            pos = bco[b] * 8 + local
            w = _hat(pos - sc * Q, sc)
            sl = b * 512 + t
            m = owner[sl] & (w > 0)
            rows.append(np.full(m.sum(), j)), cols.append(sl[m]), vals.append(w[m])
    Rwf = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nn0, ns))
    R = csr(*L0["R"], ns)
    assert abs(Rwf - R).max() == 0.0
    # prolongation: the hat weights of the eight corners of the G0 cell holding each kept slot
    s = np.nonzero(kept)[0]
    b = s // 512
    sc = (1 << blev[b].astype(np.int64))[:, None]
    pos = bco[b] * 8 + local[s % 512]
    c = np.minimum(pos // sc, np.array([nx, ny, nz]) - 2)
    rows, cols, vals = [], [], []
    for bits in range(8):
        corner = c + np.array([bits & 1, (bits >> 1) & 1, (bits >> 2) & 1])
        w = _hat(pos - sc * corner, sc[:, 0])
        id_ = lat[corner[:, 2], corner[:, 1], corner[:, 0]]
        m = (w > 0) & (id_ >= 0)
        assert np.all(id_[w > 0] != -2)     # a weight never falls on an absent node
        rows.append(s[m]), cols.append(id_[m]), vals.append(w[m])
    Pwf = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(ns, nn0))
    P = csr(*L0["P"], nn0)
    assert abs(Pwf - P).max() == 0.0


KUHN_DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (1, 1, 1)]


def _one_level(w):
    """Transpose of one-level Kuhn interpolation from a coarse array of
    w // 2 + 1 nodes per axis to the fine array of w: a coarse node at fine
    position 2t takes the fine value there and half of each Kuhn-direction
    neighbour."""
    wo = w // 2 + 1
    R = np.zeros((wo ** 3, w ** 3))
    for tz in range(wo):
        for ty in range(wo):
            for tx in range(wo):
                j = (tz * wo + ty) * wo + tx
                for (dx, dy, dz), wt in [((0, 0, 0), 1.0)] + [((s * a, s * b, s * c), 0.5) for (a, b, c) in KUHN_DIRS
                                                              for s in (1, -1)]:
                    x, y, z = 2 * tx + dx, 2 * ty + dy, 2 * tz + dz
                    if 0 <= x < w and 0 <= y < w and 0 <= z < w:
                        R[j, (z * w + y) * w + x] += wt
    return R


@pytest.mark.parametrize("level", [1, 2, 3])
def test_brick_restriction_by_levels_equals_the_hat_function(level):
    """The device restricts a level-l brick to its G0 footprint by l one-level
    Kuhn restrictions (8 -> 5 -> 3 -> 2 nodes per axis).  Nested P1 spaces make
    that product the direct hat-function weight of every brick node for every
    G0 node of the footprint."""
    R = np.eye(512)
    w = 8
    for _ in range(level):
        R = _one_level(w) @ R
        w = w // 2 + 1
    sc = 1 << level
    T = (6 + sc) // sc + 1
    assert w == T
    t = np.arange(512)
    pos = np.stack([t & 7, (t >> 3) & 7, t >> 6], -1)
    for j in range(T ** 3):
        q = np.array([j % T, (j // T) % T, j // (T * T)])
        assert np.array_equal(R[j], _hat(pos - sc * q, sc)), (level, j)
