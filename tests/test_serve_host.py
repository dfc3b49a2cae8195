"""Host logic of the continuous-batching loop (paper_2007_02082_gb300.serve)
on the CPU: the library handles are replaced by fakes that count steps, so the
admission by device footprint, joins and leaves between epochs, the cap on
members and the early exit of a failed request are checked without a GPU."""
import numpy as np
import pytest

from paper_2007_02082_gb300 import serve as S


class FakeGrid:
    live = 0

    def __init__(self, case, precision="mixed", deferred=False):
        assert deferred
        self.case = case
        self.steps = 0
        self.closed = False
        self.batch = None
        FakeGrid.live += 1

    def ib_grid_info(self):
        c = self.case
        return {"n_slots": c["slots"], "n_points": c["points"], "af_nnz": c["nnz"], "n_leaf_cells": c["cells"],
                "device_bytes": c.get("snap", 0)}

    def close(self):
        assert not self.closed and self.batch is None
        self.closed = True
        FakeGrid.live -= 1


class FakeBatch:
    log = []

    def __init__(self, handles):
        for h in handles:
            assert h.batch is None and not h.closed
            h.batch = self
        self.handles = list(handles)
        FakeBatch.log.append([h.case["rid"] for h in handles])

    def step(self, k):
        st = []
        for h in self.handles:
            h.steps += k
            fail_at = h.case.get("fail_at")
            st.append(5 if fail_at is not None and h.steps >= fail_at else 0)
        return st

    def info(self, i):
        # a batch engine reporting `engine_factor` times the estimated bytes
        est = sum(S.footprint(h.ib_grid_info(), "mixed") for h in self.handles)
        return {"device_bytes": int(est * max(h.case.get("engine_factor", 1.0) for h in self.handles))}

    def close(self):
        for h in self.handles:
            h.batch = None


@pytest.fixture(autouse=True)
def fakes(monkeypatch):
    monkeypatch.setattr(S, "IBGrid", FakeGrid)
    monkeypatch.setattr(S, "IBBatch", FakeBatch)
    FakeGrid.live = 0
    FakeBatch.log = []
    yield


def _case(rid, steps, cells=1000, slots=2000, points=100, nnz=5000, **kw):
    return dict(rid=rid, steps=steps, cells=cells, slots=slots, points=points, nnz=nnz, **kw)


def test_every_request_runs_its_steps_and_is_released():
    stream = [(0.0, _case(k, 3 + 2 * (k % 3), cells=100 * (k + 1))) for k in range(7)]
    got = {}
    res = S.serve(stream, epoch_steps=2, setup_workers=3, keep=lambda rid, h: got.__setitem__(rid, h.steps))
    s = res.summary()
    assert s["requests"] == 7 and s["failed"] == 0
    assert got == {k: c["steps"] for k, (_, c) in enumerate(stream)}
    assert res.cell_steps == sum(c["cells"] * c["steps"] for _, c in stream)
    assert FakeGrid.live == 0
    assert len(res.batch_sizes) == res.epochs and all(b >= 1 for b in res.batch_sizes)
    assert all(lat >= 0 for lat in res.latencies)
    # an epoch never runs past the end of any member
    for members in FakeBatch.log:
        assert len(set(members)) == len(members)


def test_footprint_budget_bounds_the_batch():
    c = _case(0, 4)
    one = S.footprint({"n_slots": c["slots"], "n_points": c["points"], "af_nnz": c["nnz"]}, "mixed")
    stream = [(0.0, _case(k, 4)) for k in range(6)]
    res = S.serve(stream, hbm_budget=2 * one + 1, epoch_steps=2, setup_workers=6)
    assert res.summary()["failed"] == 0
    assert max(res.batch_sizes) <= 2
    assert FakeGrid.live == 0


def test_request_above_the_budget_runs_alone():
    stream = [(0.0, _case(0, 3, slots=10 ** 7)), (0.0, _case(1, 3))]
    res = S.serve(stream, hbm_budget=10 ** 8, epoch_steps=1, setup_workers=2)
    assert res.summary()["requests"] == 2 and res.summary()["failed"] == 0
    for members in FakeBatch.log:
        if 0 in members:
            assert members == [0]


def test_member_cap():
    stream = [(0.0, _case(k, 2)) for k in range(9)]
    res = S.serve(stream, max_members=4, epoch_steps=2, setup_workers=9)
    assert max(res.batch_sizes) <= 4 and res.summary()["requests"] == 9


def test_failed_request_leaves_early_and_others_finish():
    stream = [(0.0, _case(0, 10, fail_at=4)), (0.0, _case(1, 10)), (0.0, _case(2, 6))]
    got = {}
    res = S.serve(stream, epoch_steps=2, setup_workers=3, keep=lambda rid, h: got.__setitem__(rid, h.steps))
    assert res.summary()["failed"] == 1
    assert got[0] == 4 and got[1] == 10 and got[2] == 6
    assert sorted(res.statuses) == [0, 0, 5]
    assert FakeGrid.live == 0


def test_footprint_counts_the_mixed_force_solve():
    info = {"n_slots": 0, "n_points": 256, "af_nnz": 1000}
    d = S.footprint(info, "mixed") - S.footprint(info, "fp64")
    assert d == 256 * (24 + 84 + 4) + 1000 * 4
    # the coarsest multigrid level's dense inverse, in the Krylov precision
    mg = dict(info, mg_levels=3, mg_coarsest=100)
    assert S.footprint(mg, "fp64") - S.footprint(info, "fp64") == 8 * 100 * 100
    assert S.footprint(mg, "mixed") - S.footprint(info, "mixed") == 4 * 100 * 100
    assert np.all([S.footprint(dict(info, n_slots=n), "fp64") > 0 for n in (0, 512)])


def test_snapshots_of_built_requests_count_against_the_budget():
    """Each built request holds a device snapshot until it leaves: with the
    budget at two footprints plus a snapshot's worth, snapshots as large as a
    footprint leave room for one member at a time."""
    c = _case(0, 4)
    one = S.footprint({"n_slots": c["slots"], "n_points": c["points"], "af_nnz": c["nnz"]}, "mixed")
    stream = [(0.0, _case(k, 4, snap=one)) for k in range(4)]
    res = S.serve(stream, hbm_budget=3 * one + 1, epoch_steps=2, setup_workers=4)
    assert res.summary()["failed"] == 0 and res.summary()["requests"] == 4
    assert max(res.batch_sizes) == 1
    assert FakeGrid.live == 0


def test_ready_backlog_is_bounded():
    """At most max_ready requests are built ahead of admission."""
    peak = [0]
    orig = FakeGrid.__init__

    def counting(self, *a, **k):
        orig(self, *a, **k)
        peak[0] = max(peak[0], FakeGrid.live)

    FakeGrid.__init__ = counting
    try:
        stream = [(0.0, _case(k, 6)) for k in range(10)]
        res = S.serve(stream, max_members=2, max_ready=2, epoch_steps=2, setup_workers=10)
    finally:
        FakeGrid.__init__ = orig
    assert res.summary()["requests"] == 10 and FakeGrid.live == 0
    assert peak[0] <= 4          # two members and two built ahead


def test_admission_follows_the_reported_batch_bytes():
    """A batch engine that reports more device bytes than the estimate scales
    the footprint used for admission from then on."""
    c = _case(0, 4)
    one = S.footprint({"n_slots": c["slots"], "n_points": c["points"], "af_nnz": c["nnz"]}, "mixed")
    stream = [(0.0, _case(k, 4, engine_factor=3.0)) for k in range(6)]
    res = S.serve(stream, hbm_budget=4 * one, epoch_steps=2, setup_workers=1)
    assert res.summary()["failed"] == 0
    assert res.footprint_scale == pytest.approx(3.0)
    assert max(res.batch_sizes[1:]) <= 1       # 3 x one each: one member fits the budget
