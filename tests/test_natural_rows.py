"""Natural-boundary rows of the symmetric viscous form (csrc/setup.cpp).

The library builds, per stored slot, the rows of ((grad u)^T n, phi_a) over the
tetrahedron faces in outlet and pressure-inlet planes; the oracle assembles the
same term over all faces with generic P1 shape functions.  Mapping each slot
to its node (interface copies and hanging nodes included) and summing, the two
must agree on every row without a velocity condition.  No GPU needed.
"""
import os
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import ibfe
from tests.test_host_setup import _desc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_02082_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("natprobe")
    exe = d / "nat_probe"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(CSRC, "setup.cpp"), os.path.join(ROOT, "tests", "natural_rows_probe.cpp"),
                    "-o", str(exe)], check=True)
    return exe, d


def host_rows(probe, case):
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
    pos = 0

    def i64(n):
        nonlocal pos
        v = np.frombuffer(b, np.int64, count=n, offset=pos)
        pos += 8 * n
        return v

    rows = []
    for _ in range(int(i64(1)[0])):
        q = i64(3)
        ents = []
        for _ in range(int(i64(1)[0])):
            qb = i64(3)
            comp = int(i64(1)[0])
            w = float(np.frombuffer(b, np.float64, count=1, offset=pos)[0])
            pos += 8
            ents.append((qb, comp, w))
        rows.append((q, ents))
    return rows


CASES = {
    "uniform_outlet": lambda: W.cylinder_uniform_16x16x64(viscous="sym"),
    "refined_pressure_inlet": lambda: W.cylinder_refined_small(n=(16, 16, 8), seed=23, inlet=W.PINLET, a0=0.16,
                                                               viscous="sym"),
    "two_levels": lambda: W.cylinder_case(n=(24, 24, 8), length=1.0, half_width=0.75, M=1500, seed=12, max_level=2,
                                          refine_band=1, reduce_band=3, viscous="sym"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_natural_rows_match_oracle(probe, name):
    case = CASES[name]()
    rows = host_rows(probe, case)
    m = ibfe.build_mesh(case)
    Bn = ibfe.Operators(m).natural_boundary_blocks()
    N = m.n_nodes
    vdir = ibfe.velocity_dirichlet(m)
    import scipy.sparse as sp
    trip = {(i, j): ([], [], []) for i in range(3) for j in range(3)}
    for q, ents in rows:
        a = m.lookup(q[None, :])[0]
        assert a >= 0 and not vdir[a]
        for qb, comp, w in ents:
            bnode = m.lookup(qb[None, :])[0]
            assert bnode >= 0
            r, c, v = trip[(comp // 3, comp % 3)]
            r.append(a)
            c.append(bnode)
            v.append(w)
    keep = np.nonzero(~vdir)[0]
    assert len(rows) > 50
    scale = max(abs(Bn[i][j]).max() for i in range(3) for j in range(3))
    for i in range(3):
        for j in range(3):
            r, c, v = trip[(i, j)]
            H = sp.csr_matrix((np.asarray(v, float), (np.asarray(r, int), np.asarray(c, int))), shape=(N, N))
            D = (H - Bn[i][j])[keep]
            assert (abs(D).max() if D.nnz else 0.0) <= 1e-12 * scale, (name, i, j)
