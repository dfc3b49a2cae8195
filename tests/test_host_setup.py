"""Host-side logic of the library, checked on the CPU.

* The library builds and exports every function include/ib.h declares.
* The host grid builder (level map, active cells, canonical nodes, hanging
  nodes, boundary/port flags, IB supports) agrees bit for bit with the oracle.
  It is compiled with a small driver (tests/host_grid_probe.cpp), so no GPU is
  needed.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import ibfe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_02082_gb300", "csrc")


@pytest.fixture(scope="module")
def lib_path():
    from paper_2007_02082_gb300.build import build
    return build()


def test_library_exports_every_declared_function(lib_path):
    hdr = open(os.path.join(ROOT, "include", "ib.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"^\s*(?:ib_status|const char\*|void)\s+(\w+)\s*\(", hdr, flags=re.M))
    assert {"ib_grid_create", "ib_set_boundary", "ipcs_step", "ib_fields_get"} <= names
    lib = C.CDLL(lib_path)
    for n in names:
        assert hasattr(lib, n), n
    from paper_2007_02082_gb300 import _abi
    assert set(_abi.EXPORTS) == names


def test_abi_struct_sizes_match_header(tmp_path):
    """The ctypes mirror has the same layout as the C structs."""
    from paper_2007_02082_gb300 import _abi
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "ib.h"\nint main(){printf("%zu %zu %zu\\n",'
                   'sizeof(ib_port),sizeof(ib_grid_desc),sizeof(ib_info));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [C.sizeof(_abi.IbPort), C.sizeof(_abi.IbGridDesc), C.sizeof(_abi.IbInfo)]


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("probe")
    exe = d / "probe"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, os.path.join(CSRC, "setup.cpp"), os.path.join(ROOT, "tests", "host_grid_probe.cpp"),
                    "-o", str(exe)], check=True)
    return exe, d


def _desc(case):
    from paper_2007_02082_gb300 import _abi
    from paper_2007_02082_gb300 import _port_struct
    d = _abi.IbGridDesc()
    for a in range(3):
        d.origin[a] = case["origin"][a]
        d.extent[a] = case["extent"][a]
        d.n[a] = case["n"][a]
    d.max_level, d.refine_band, d.reduce_band = case["max_level"], case["refine_band"], case["reduce_band"]
    d.nu, d.rho, d.dt = case["nu"], case["rho"], case["dt"]
    d.viscous_form = 1 if case.get("viscous", "grad") == "sym" else 0
    d.port_tangential = _abi.IB_TANGENTIAL_ZERO if case.get("port_tangential") == "zero" else _abi.IB_TANGENTIAL_FREE
    d.n_ports = len(case["ports"])
    for k, p in enumerate(case["ports"]):
        d.ports[k] = _port_struct(p)
    return d


def run_probe(probe, case):
    exe, d = probe
    inp, out = d / "in.bin", d / "out.bin"
    desc = _desc(case)
    M = len(case["X"])
    with open(inp, "wb") as f:
        f.write(bytes(desc))
        f.write(np.int64(M).tobytes())
        f.write(np.ascontiguousarray(case["X"], np.float64).tobytes())
        f.write(np.ascontiguousarray(case["dS"], np.float64).tobytes())
        f.write(np.ascontiguousarray(case["UB"], np.float64).tobytes())
        f.write(np.ascontiguousarray(case["inside"], np.uint8).tobytes())
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True)
    if r.returncode != 0:
        return r.returncode, r.stderr
    b = open(out, "rb").read()
    hdr = np.frombuffer(b[:48], np.int64)
    N, M, nc = (int(v) for v in hdr[:3])
    o = 48
    res = {"n_hang": int(hdr[3]), "n_if": int(hdr[4]), "nbricks": int(hdr[5])}
    for name, cnt, dt in (("q", 3 * N, np.int32), ("flags", N, np.uint8), ("active", nc, np.uint8),
                          ("level", nc, np.uint8), ("ib_origin", 3 * M, np.int32), ("ib_free", 64 * M, np.uint8)):
        nb = cnt * np.dtype(dt).itemsize
        res[name] = np.frombuffer(b[o:o + nb], dt)
        o += nb
    res["q"] = res["q"].reshape(N, 3)
    res["ib_origin"] = res["ib_origin"].reshape(M, 3)
    res["ib_free"] = res["ib_free"].reshape(M, 64)
    return 0, res


def oracle_structures(case):
    m = ibfe.build_mesh(case)
    vdir = ibfe.velocity_dirichlet(m)
    # the force spreads to nodes free in every component (a pressure port's
    # tangential components are Dirichlet under the zero-tangential option)
    free = ~ibfe.velocity_dirichlet_components(m).any(axis=1) & ~m.hanging
    ib = ibfe.IB(m, case, free)
    flags = (m.hanging * 1 + vdir * 2 + ibfe.pressure_dirichlet(m) * 4 + ((m.inlet > 0) | (m.pinlet > 0)) * 8
             + m.boundary * 16).astype(np.uint8)
    exists = ib.support_idx >= 0
    fr = np.where(exists, np.where(free[np.maximum(ib.support_idx, 0)], 1, 2), 0).astype(np.uint8)
    return m, flags, ib.origin, fr


def _duct_no_points():
    """A pressure-driven square duct without an immersed boundary (M = 0)."""
    n = (6, 6, 12)
    return {"name": "duct_6x6x12", "origin": (-0.5, -0.5, 0.0), "extent": (1.0, 1.0, 2.0), "n": n,
            "max_level": 0, "refine_band": 2, "reduce_band": -1, "nu": 0.1, "rho": 1.0, "dt": 0.01,
            "ports": [W._port(2, 0, (0.0, 0.0, 0.0), 0.499, W.PINLET, a0=1.0),
                      W._port(2, 1, (0.0, 0.0, 2.0), 0.499, W.OUTLET)],
            "X": np.zeros((0, 3)), "dS": np.zeros(0), "UB": np.zeros((0, 3)),
            "inside": np.ones((n[2], n[1], n[0]), np.uint8)}


CASES = {
    "duct_no_points": _duct_no_points,
    "uniform_16x16x64": lambda: W.cylinder_uniform_16x16x64(),
    "refined_16x16x32": lambda: W.cylinder_refined_small(),
    "refined_reduced_20x20x12": lambda: W.cylinder_case(n=(20, 20, 12), length=1.5, half_width=0.75, M=900,
                                                         seed=11, max_level=1, refine_band=2, reduce_band=2),
    "two_levels_24x24x8": lambda: W.cylinder_case(n=(24, 24, 8), length=1.0, half_width=0.75, M=1500, seed=12,
                                                  max_level=2, refine_band=1, reduce_band=3),
    "aneurysm_L1": lambda: W.aneurysm_case(length=1.5, h=1.0 / 12, seed=13),
    "bend_L0": lambda: W.bent_tube_case(R=0.4, Rc=1.0, l_in=0.5, l_out=0.5, h=1.0 / 10, seed=14),
    # pressure inlet on a refined face: port nodes next to hanging nodes
    "pressure_inlet_refined": lambda: W.cylinder_refined_small(n=(16, 16, 8), seed=23, inlet=W.PINLET, a0=0.16),
    # the reduced copy of the synthetic aorta: arch, taper, three branches,
    # five ports on two box faces, one refinement level
    "aorta_40x40x60_L1": lambda: W.aorta_case(n=(40, 40, 60), max_level=1, M=3000, seed=44),
    # zero tangential velocity on the pressure ports: the force is not spread
    # onto their nodes
    "pressure_inlet_tangential_zero": lambda: dict(W.cylinder_refined_small(n=(16, 16, 8), seed=23, inlet=W.PINLET,
                                                                             a0=0.16), port_tangential="zero"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_grid_matches_oracle_bit_exact(probe, name):
    case = CASES[name]()
    rc, res = run_probe(probe, case)
    assert rc == 0, res
    m, flags, org, fr = oracle_structures(case)
    assert np.array_equal(res["active"], m.active.astype(np.uint8).ravel())
    assert np.array_equal(res["level"], m.level.astype(np.uint8).ravel())
    assert np.array_equal(res["q"], m.node_q.astype(np.int32))
    assert res["n_hang"] == int(m.hanging.sum())
    assert np.array_equal(res["flags"], flags)
    assert np.array_equal(res["ib_origin"], org.astype(np.int32))
    assert np.array_equal(res["ib_free"], fr)


def test_point_outside_box_is_rejected(probe):
    case = W.cylinder_uniform_16x16x64()
    case["X"] = case["X"].copy()
    case["X"][5] = (10.0, 0.0, 1.0)
    rc, err = run_probe(probe, case)
    assert rc == 10 + 1 and "outside" in err


def test_invalid_points_and_ports_are_rejected(probe):
    """The host grid builder refuses, with IB_EINVAL and a message, a
    non-finite point, a non-positive area element and an outlet whose disc
    meets no boundary node (the Poisson problem would be singular)."""
    base = W.cylinder_uniform_16x16x64()

    def bad(edit, msg):
        c = dict(base, X=base["X"].copy(), dS=base["dS"].copy(), ports=[dict(p) for p in base["ports"]])
        edit(c)
        rc, err = run_probe(probe, c)
        assert rc == 10 + 1 and msg in err, (rc, err)

    bad(lambda c: c["X"].__setitem__((7, 1), np.nan), "non-finite")
    bad(lambda c: c["dS"].__setitem__(3, 0.0), "positive")
    bad(lambda c: c["ports"][1].update(center=(5.0, 5.0, 4.0)), "singular")


def test_binding_maps_the_case_options():
    """The viscous form and the tangential port condition map to their
    descriptor values; an unknown value is refused rather than ignored."""
    from paper_2007_02082_gb300 import _abi, _port_tangential, _viscous_form
    assert _viscous_form({}) == _abi.IB_VISCOUS_GRAD
    assert _viscous_form({"viscous": "sym", "port_tangential": "free"}) == _abi.IB_VISCOUS_SYM
    assert _port_tangential({}) == _abi.IB_TANGENTIAL_FREE
    assert _port_tangential({"port_tangential": "zero"}) == _abi.IB_TANGENTIAL_ZERO
    with pytest.raises(ValueError):
        _port_tangential({"port_tangential": "slip"})
    with pytest.raises(ValueError):
        _viscous_form({"viscous": "cubic"})


def test_grid_create_rejects_invalid_descriptions(lib_path):
    """ib_grid_create validates the description before it touches the device:
    every invalid field returns IB_EINVAL and no handle (no GPU needed)."""
    from paper_2007_02082_gb300 import _abi
    lib = _abi.bind(C.CDLL(lib_path))
    case = W.cylinder_case(n=(8, 8, 16), M=100)

    def create(edit):
        d = _desc(case)
        d.precision, d.poisson_pc = _abi.IB_MIXED, 0
        edit(d)
        h = C.c_void_p(0)
        st = lib.ib_grid_create(C.byref(d), C.byref(h))
        return st, h.value

    def port0(field, v):
        return lambda d: setattr(d.ports[0], field, v)

    bad = [
        port0("profile", 1),                                   # only the parabolic inlet profile exists
        port0("axis", 3),
        port0("side", 2),
        port0("radius", 0.0),
        port0("kind", 7),
        port0("n_harm", _abi.IB_MAX_HARMONICS + 1),
        lambda d: setattr(d, "n_ports", 0),
        lambda d: setattr(d.ports[1], "kind", _abi.IB_INLET_VELOCITY),   # no port fixes Phi
        lambda d: setattr(d, "precision", 2),
        lambda d: setattr(d, "viscous_form", 2),
        lambda d: setattr(d, "nu", 0.0),
        lambda d: setattr(d, "dt", -1.0),
        lambda d: setattr(d, "max_level", 9),
        lambda d: (setattr(d, "max_level", 1), setattr(d, "refine_band", 0)),
        # launch choices outside their ranges
        lambda d: d.tune.__setitem__(_abi.TUNE_INDEX["poisson_kernel"], 4),
        lambda d: d.tune.__setitem__(_abi.TUNE_INDEX["stream_chunk"], 5),
        lambda d: d.tune.__setitem__(_abi.TUNE_INDEX["mg_small"], 10),
        lambda d: d.tune.__setitem__(_abi.TUNE_INDEX["mg_sweeps"], 5),
        lambda d: d.tune.__setitem__(_abi.TUNE_INDEX["mg_persist"], 3),
        lambda d: setattr(d, "port_tangential", 2),
    ]
    for k, edit in enumerate(bad):
        st, h = create(edit)
        assert st == _abi.IB_EINVAL and not h, k


def test_null_handles_are_rejected(lib_path):
    """Every entry point checks its handle before any device work: a null grid
    or batch gives IB_EINVAL (or a message / no-op for the error and destroy
    calls), as include/ib.h states."""
    from paper_2007_02082_gb300 import _abi
    lib = _abi.bind(C.CDLL(lib_path))
    E = _abi.IB_EINVAL
    buf = (C.c_double * 8)()
    info = _abi.IbInfo()
    assert lib.ib_set_boundary(None, 1, buf, buf, None, None) == E
    assert lib.ipcs_step(None, 1) == E
    assert lib.ib_fields_get(None, 0, buf, 8, 0) == E
    assert lib.ib_fields_get_noalloc(None, 0, buf, 8, 0) == E
    assert lib.ib_fields_set(None, 0, buf, 8, 0) == E
    assert lib.ib_set_points(None, 1, buf, None, 0) == E
    assert lib.ib_wss(None, buf, buf, None, 0) == E
    assert lib.ib_grid_info(None, C.byref(info)) == E
    assert lib.ib_last_error(None) == b"null handle"
    lib.ib_grid_destroy(None)
    out = C.c_void_p(0)
    assert lib.ib_batch_create(None, 1, C.byref(out)) == E and not out.value
    members = (C.c_void_p * 1)(None)
    assert lib.ib_batch_create(members, 0, C.byref(out)) == E and not out.value
    assert lib.ib_batch_step(None, 1, None) == E
    assert lib.ib_batch_fields_get(None, 0, 0, buf, 8, 0) == E
    assert lib.ib_batch_info(None, 0, C.byref(info)) == E
    assert lib.ib_batch_last_error(None) == b"null batch"
    lib.ib_batch_destroy(None)


def test_fields_get_writes_into_a_host_array():
    """Marshalling of ib_fields_get(out=numpy array): the library receives the
    array's own pointer and byte count with the host flag and writes into it
    (no intermediate copy); a destination of the wrong shape, dtype or layout
    is refused before the call."""
    from paper_2007_02082_gb300 import IBGrid, _abi

    class FakeLib:
        calls = []

        def ib_fields_get(self, h, field, ptr, nbytes, on_dev):
            self.calls.append((field, ptr, nbytes, on_dev))
            src = np.arange(nbytes // 8, dtype=np.float64)
            C.memmove(ptr, src.ctypes.data, nbytes)
            return 0

        def ib_last_error(self, h):
            return b""

    g = object.__new__(IBGrid)
    g.lib, g.h, g.case = FakeLib(), None, {"n": (2, 2, 2)}
    g.ib_grid_info = lambda: {"n_nodes": 5, "n_points": 2}
    out = np.zeros((5, 3))
    assert g.ib_fields_get("U", out=out) is out
    assert g.lib.calls[-1] == (_abi.FIELD["U"], out.ctypes.data, out.nbytes, 0)
    assert np.array_equal(out.ravel(), np.arange(15.0))
    p = g.ib_fields_get("P")
    assert p.shape == (5,) and np.array_equal(p, np.arange(5.0))
    for bad in (np.zeros((5, 2)), np.zeros((5, 3), np.float32), np.zeros((3, 5)).T):
        with pytest.raises(ValueError):
            g.ib_fields_get("U", out=bad)
