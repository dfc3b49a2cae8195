"""Incident-cell-mask weights of the P1 Kuhn operators (csrc/kuhn_weights.hpp).

The library derives the consistent-mass and stiffness couplings of a node from
the 8-bit mask of its active incident cells by closed formulas.  This test
enumerates, for every mask, the six Kuhn tetrahedra of every active incident
cell (one per axis order, Sec. 3.1 box mesh) and counts directly which of them
hold the node and each neighbour, and sums the neighbours' barycentric
gradients and the products (d_j phi_node)(d_i phi_neighbour) of the symmetric
viscous form: the counts and sums must equal the library's formulas.
"""
import itertools
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_02082_gb300", "csrc")

OFFSETS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
           (0, 1, 1), (0, -1, -1), (1, 0, 1), (-1, 0, -1), (1, 1, 1), (-1, -1, -1)]


def brute_force(mask):
    mass = np.zeros(15, int)
    edge = np.zeros(6, int)
    grad = np.zeros((15, 3), int)
    trans = np.zeros((15, 3, 3), int)
    for c in range(8):
        if not (mask >> c) & 1:
            continue
        d = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        lower = d - 1                                  # cell lower corner relative to the node
        for perm in itertools.permutations(range(3)):
            v = [lower.copy()]
            for a in perm:
                w = v[-1].copy()
                w[a] += 1
                v.append(w)
            verts = [tuple(x) for x in v]
            if (0, 0, 0) not in verts:
                continue
            # barycentric gradients in units 1/h: lambda_0 = 1 - x_a1, lambda_1 = x_a1 - x_a2, ...
            gvec = np.zeros((4, 3), int)
            gvec[0, perm[0]] = -1
            gvec[1, perm[0]], gvec[1, perm[1]] = 1, -1
            gvec[2, perm[1]], gvec[2, perm[2]] = 1, -1
            gvec[3, perm[2]] = 1
            ia = verts.index((0, 0, 0))
            for k, o in enumerate(OFFSETS):
                if o in verts:
                    mass[k] += 2 if k == 0 else 1
                    grad[k] += gvec[verts.index(o)]
                    trans[k] += np.outer(gvec[verts.index(o)], gvec[ia])   # [i][j] = d_i phi_o * d_j phi_node
            for i in range(3):                         # axis edges of the tetrahedron
                p, q = verts[i], verts[i + 1]
                if (0, 0, 0) in (p, q):
                    other = q if p == (0, 0, 0) else p
                    a = perm[i]
                    s = other[a]
                    edge[2 * a + (0 if s > 0 else 1)] += 1
    return mass, edge, grad, trans


def test_mask_weights_match_tetrahedron_enumeration(tmp_path):
    exe = tmp_path / "kw"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "kuhn_weights_probe.cpp"),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for mask in range(256):
        got = np.array([int(v) for v in out[mask].split()])
        mass, edge, grad, trans = brute_force(mask)
        assert np.array_equal(got[:15], mass), (mask, got[:15], mass)
        assert np.array_equal(got[15:21], edge), (mask, got[15:21], edge)
        assert np.array_equal(got[21:66].reshape(15, 3), grad), mask
        assert np.array_equal(got[66:].reshape(15, 3, 3), trans), mask
    # interior node: row of the mass matrix sums to the cell volume (120 units)
    assert sum(int(v) for v in out[255].split()[:15]) == 120


def test_transpose_couplings_match_oracle_assembly():
    """The oracle assembles (grad u^T, grad v) element by element with generic
    P1 shape functions; on an anisotropic box every node's row equals
    (V/6)/(h_i h_j) times the enumerated coupling of its incident-cell mask."""
    import sys
    sys.path.insert(0, ROOT)
    from oracle import ibfe
    n, h = (3, 3, 3), np.array([0.5, 0.7, 0.9])
    case = {"origin": (0.0, 0.0, 0.0), "extent": tuple(np.array(n) * h), "n": n, "max_level": 0, "refine_band": 2,
            "reduce_band": -1, "nu": 0.1, "rho": 1.0, "dt": 0.01, "ports": [], "X": np.zeros((0, 3)),
            "dS": np.zeros(0), "UB": np.zeros((0, 3)), "inside": np.ones((3, 3, 3), np.uint8)}
    m = ibfe.build_mesh(case)
    Kt = ibfe.Operators(m).transpose_blocks()
    V = h.prod()
    for a in range(m.n_nodes):
        q = m.node_q[a]
        mask = 0
        for c in range(8):
            d = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
            cell = q + d - 1
            if np.all(cell >= 0) and np.all(cell < n):
                mask |= 1 << c
        trans = brute_force(mask)[3]
        for k, o in enumerate(OFFSETS):
            qb = q + np.array(o)
            if not (np.all(qb >= 0) and np.all(qb <= n)):
                continue
            b = m.lookup(qb[None, :])[0]
            for i in range(3):
                for j in range(3):
                    want = V / 6.0 / (h[i] * h[j]) * trans[k, i, j]
                    assert abs(Kt[i][j][a, b] - want) <= 1e-12, (a, k, i, j)
