"""Host logic of the autotuner (paper_2007_02082_gb300.tune) on the CPU: the
workload-class key, the choice among timed candidates, the JSON cache, and
that a cached class is not timed again (library handles and GPU timing are
replaced by fakes)."""
import json

import pytest

from paper_2007_02082_gb300 import tune as T


def test_class_key_groups_by_precision_depth_and_size():
    a = T.class_key({"n_slots": 1 << 26}, "mixed", 2)
    assert a == "mixed:L2:s26"
    assert T.class_key({"n_slots": int(1.2 * (1 << 26))}, "mixed", 2) == a      # same order of magnitude
    assert T.class_key({"n_slots": 1 << 24}, "mixed", 2) != a
    assert T.class_key({"n_slots": 1 << 26}, "fp64", 2) != a
    assert T.class_key({"n_slots": 1 << 26}, "mixed", 1) != a


def test_choose_fastest_and_keep_defaults():
    choice, ms = T.choose([({}, 10.0), ({"mg_sweeps": 3}, 8.5), ({"stream_chunk": 4}, 9.0)])
    assert ms == 8.5 and choice == dict(T.DEFAULTS, mg_sweeps=3)
    # a failed candidate (None) is skipped; ties keep the earlier one
    choice, ms = T.choose([({}, 5.0), ({"poisson_kernel": 2}, None), ({"mg_small": 2048}, 5.0)])
    assert choice == T.DEFAULTS and ms == 5.0
    with pytest.raises(ValueError):
        T.choose([({}, None)])


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    c = T.TuneCache(p)
    assert c.get("k") is None
    c.put("k", dict(T.DEFAULTS, mg_sweeps=1), 7.5, [({}, 8.0), ({"mg_sweeps": 1}, 7.5)])
    d = T.TuneCache(p)
    assert d.get("k") == dict(T.DEFAULTS, mg_sweeps=1)
    raw = json.load(open(p))
    assert raw["k"]["ms_per_step"] == 7.5 and len(raw["k"]["candidates"]) == 2


class FakeGrid:
    def __init__(self, case, precision="mixed", device=0, deferred=False, **kw):
        self.case = case

    def ib_grid_info(self):
        return {"n_slots": self.case["slots"]}

    def close(self):
        pass


def test_tune_case_times_each_candidate_once_per_class(monkeypatch, tmp_path):
    import paper_2007_02082_gb300 as pkg
    monkeypatch.setattr(pkg, "IBGrid", FakeGrid)
    calls = []

    def timer(over):
        calls.append(dict(over))
        return 10.0 - len(over) - over.get("mg_sweeps", 0)   # fastest: mg_sweeps 3

    cache = T.TuneCache(str(tmp_path / "c.json"))
    case = {"slots": 1 << 20, "max_level": 1}
    choice, key, hit, timings = T.tune_case(case, "mixed", cache=cache, timer=timer)
    assert not hit and len(calls) == len(T.CANDIDATES) and choice["mg_sweeps"] == 3
    # the same class again (a slightly different size): from the cache, nothing timed
    choice2, key2, hit2, _ = T.tune_case({"slots": (1 << 20) + 4096, "max_level": 1}, "mixed", cache=cache,
                                         timer=timer)
    assert hit2 and key2 == key and choice2 == choice and len(calls) == len(T.CANDIDATES)


def test_every_candidate_is_a_valid_description():
    """The tuner's defaults and every candidate pass the library's own check of
    the launch choices: ib_grid_create does not answer IB_EINVAL for them (on a
    machine without a GPU it stops at the device with IB_ECUDA; with one it
    returns a handle), while an out-of-range value of each choice is refused."""
    import ctypes as C

    import workloads as W
    from paper_2007_02082_gb300 import _abi
    from paper_2007_02082_gb300.build import build
    from tests.test_host_setup import _desc
    lib = _abi.bind(C.CDLL(build()))
    case = W.cylinder_case(n=(8, 8, 16), M=100)

    def status(choice):
        d = _desc(case)
        d.precision = _abi.IB_MIXED
        for k, v in choice.items():
            d.tune[_abi.TUNE_INDEX[k]] = v
        h = C.c_void_p(0)
        st = lib.ib_grid_create(C.byref(d), C.byref(h))
        if h.value:
            lib.ib_grid_destroy(h)
        return st

    assert set(T.DEFAULTS) == set(_abi.TUNE_INDEX)
    for over in T.CANDIDATES:
        assert set(over) <= set(_abi.TUNE_INDEX), over
        assert status(dict(T.DEFAULTS, **over)) != _abi.IB_EINVAL, over
    for bad in ({"poisson_kernel": 4}, {"stream_chunk": 5}, {"mg_small": 10}, {"mg_sweeps": 5}, {"mg_persist": 3}):
        assert status(dict(T.DEFAULTS, **bad)) == _abi.IB_EINVAL, bad
