"""Batched (continuously batched) steps: several problems side by side.

Each member's kernels touch only its own bricks and every Krylov reduction is
segmented per member, so a member's result is bitwise the same alone and in any
mix (the served path's correctness condition); state carries across batches
through the members' snapshots.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    return [
        W.cylinder_case(n=(8, 8, 16), length=2.0, M=250, seed=31, nu=0.05, dt=0.01),
        W.cylinder_refined_small(n=(16, 16, 8), seed=32),
        W.cylinder_case(n=(12, 12, 24), length=3.0, half_width=0.7, M=500, seed=33, nu=0.02, dt=0.005,
                        b=(0.5,), max_level=1, refine_band=2, reduce_band=2),
        # pressure-driven member: its port indices and times are offset in the mix
        W.cylinder_case(n=(8, 8, 16), length=2.0, M=250, seed=34, nu=0.05, dt=0.01, inlet=W.PINLET, a0=0.8,
                        b=(0.2,)),
    ]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_member_bitwise_alone_and_in_mix(precision):
    from paper_2007_02082_gb300 import IBBatch, IBGrid
    cases = _cases()
    steps = 3
    alone = []
    for c in cases:
        g = IBGrid(c, precision=precision, deferred=True)
        b = IBBatch([g])
        st = b.step(steps)
        assert np.all(st == 0)
        alone.append((g.ib_fields_get("U"), g.ib_fields_get("P")))
        b.close()
        g.close()
    mem = [IBGrid(c, precision=precision, deferred=True) for c in cases]
    batch = IBBatch(mem)
    st = batch.step(steps)
    assert np.all(st == 0)
    for i, m in enumerate(mem):
        assert np.array_equal(m.ib_fields_get("U"), alone[i][0]), i
        assert np.array_equal(m.ib_fields_get("P"), alone[i][1]), i
        assert batch.info(i)["step"] == steps
    batch.close()
    # a standalone handle runs the same kernels: the same bits again
    s = IBGrid(cases[1], precision=precision)
    s.ipcs_step(steps)
    assert np.array_equal(s.ib_fields_get("U"), alone[1][0])
    s.close()
    for m in mem:
        m.close()


def test_symmetric_form_members_alone_and_in_mix():
    """Members of the symmetric viscous form (coupled momentum components,
    natural boundary rows) keep their bits alone and in a mix; a batch cannot
    mix the two viscous forms."""
    from paper_2007_02082_gb300 import IBBatch, IBError, IBGrid
    cases = [W.cylinder_case(n=(8, 8, 8), length=1.0, half_width=0.6, M=300, seed=61, max_level=1, refine_band=1,
                             reduce_band=1, nu=0.02, dt=0.002, b=(0.5,), viscous="sym"),
             W.cylinder_case(n=(8, 8, 16), length=2.0, M=250, seed=62, nu=0.05, dt=0.01, inlet=W.PINLET, a0=0.8,
                             viscous="sym")]
    alone = []
    for c in cases:
        g = IBGrid(c, precision="mixed", deferred=True)
        b = IBBatch([g])
        assert np.all(b.step(2) == 0)
        alone.append(g.ib_fields_get("U"))
        b.close()
        g.close()
    mem = [IBGrid(c, precision="mixed", deferred=True) for c in cases]
    batch = IBBatch(mem)
    assert np.all(batch.step(2) == 0)
    for i, m in enumerate(mem):
        assert np.array_equal(m.ib_fields_get("U"), alone[i]), i
    batch.close()
    other = IBGrid(_cases()[0], precision="mixed", deferred=True)
    with pytest.raises(IBError):
        IBBatch([mem[0], other])
    for m in mem + [other]:
        m.close()


def test_state_carries_across_batches():
    """Member B steps 2 times with A, then 2 times with C: bitwise B stepped 4
    times alone (u, p and the warm starts Phi, F travel in the snapshot)."""
    from paper_2007_02082_gb300 import IBBatch, IBGrid
    a, b, c = _cases()[:3]
    ref = IBGrid(b, precision="mixed", deferred=True)
    rb = IBBatch([ref])
    rb.step(4)
    u_ref = ref.ib_fields_get("U")
    rb.close()
    ga = IBGrid(a, precision="mixed", deferred=True)
    gb = IBGrid(b, precision="mixed", deferred=True)
    gc = IBGrid(c, precision="mixed", deferred=True)
    b1 = IBBatch([ga, gb])
    b1.step(2)
    b1.close()
    assert gb.ib_grid_info()["step"] == 2
    b2 = IBBatch([gb, gc])
    b2.step(2)
    assert np.array_equal(gb.ib_fields_get("U"), u_ref)
    b2.close()
    for g in (ref, ga, gb, gc):
        g.close()


def test_deferred_handle_rules():
    from paper_2007_02082_gb300 import IBBatch, IBError, IBGrid
    c = _cases()[0]
    g = IBGrid(c, precision="fp64", deferred=True)
    with pytest.raises(IBError):
        g.ipcs_step(1)            # deferred handles step only inside a batch
    b = IBBatch([g])
    with pytest.raises(IBError):
        IBBatch([g])              # already held by a batch
    b.close()
    s = IBGrid(c, precision="fp64")
    with pytest.raises(IBError):
        IBBatch([s])              # standalone handles cannot join
    s.close()
    g.close()


def test_serving_loop_results_match_alone():
    """Continuous batching: requests join and leave between epochs; every
    request's final velocity is bitwise the one it gets alone."""
    from paper_2007_02082_gb300 import IBBatch, IBGrid
    from paper_2007_02082_gb300.serve import serve
    cases = _cases()
    stream = []
    for k in range(6):
        # the first request, the pressure-driven tube (a slowly accelerating
        # flow), runs for about 30 epochs so that the others join while it is
        # active; short requests spaced in time may never overlap
        c = dict(cases[3] if k == 0 else cases[k % 4])
        c["steps"] = 61 if k == 0 else 3 + (k % 3) * 2
        stream.append((0.0, c))
    got = {}
    # every request arrives at once and is set up concurrently
    res = serve(stream, precision="mixed", epoch_steps=2, setup_workers=6,
                keep=lambda rid, h: got.__setitem__(rid, h.ib_fields_get("U")))
    s = res.summary()
    assert s["requests"] == 6 and s["failed"] == 0
    assert res.epochs >= 3 and max(res.batch_sizes) >= 2
    for rid, (_, c) in enumerate(stream):
        g = IBGrid(c, precision="mixed", deferred=True)
        b = IBBatch([g])
        b.step(c["steps"])
        assert np.array_equal(g.ib_fields_get("U"), got[rid]), rid
        b.close()
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_serving_footprint_covers_the_batch_bytes(precision):
    """The serving loop admits requests by footprint(): for single members and
    for a mix, the estimate is at least the device bytes the batch engine
    reports holding (ib_batch_info), so admission never plans with less memory
    than the library takes."""
    from paper_2007_02082_gb300 import IBBatch, IBGrid
    from paper_2007_02082_gb300.serve import footprint
    cases = _cases() + [W.aneurysm_case(R=0.4, length=3.0, Rs=0.5, offset=0.55, h=1.0 / 12, max_level=2, seed=35,
                                        dt=0.002, b=())]
    mem = [IBGrid(c, precision=precision, deferred=True) for c in cases]
    for group in [[m] for m in mem] + [mem]:
        b = IBBatch(group)
        est = sum(footprint(m.ib_grid_info(), precision) for m in group)
        measured = b.info(0)["device_bytes"]
        b.close()
        assert measured <= est <= 1.6 * measured, (len(group), measured, est)
    for m in mem:
        m.close()
