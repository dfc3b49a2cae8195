"""Host arithmetic of bench.py on the CPU: the per-class and whole-step
bandwidth figures use the same byte model as the dominant kernel's roofline."""
import math


def test_timed_class_bandwidth_matches_the_roofline_formula():
    import bench
    n_valid = 2_824_181
    peak = 6788.6
    vb = 4
    dms = [0.0] * 12
    dn = [0] * 12
    # momentum apply, mass apply, Poisson stencil and the V-cycle transfers
    for k, ms, n in ((6, 4.63, 60), (3, 2.89, 40), (0, 0.94, 20), (11, 4.6, 300)):
        dms[k], dn[k] = ms, n
    r = bench.timed_class_bandwidth(dms, dn, vb, True, n_valid, peak)
    # the dominant kernel's fraction, as the roofline computes it
    per_launch = bench.class_bytes(6, vb, True) * n_valid
    achieved = per_launch / ((dms[6] / dn[6]) / 1e3) / 1e9
    assert math.isclose(r["per_class_frac"][bench.CLASS_NAMES[6]], round(achieved / peak, 3))
    # the V-cycle transfers have no byte model and are left out of the total
    assert bench.CLASS_NAMES[11] not in r["per_class_frac"]
    total_b = sum(bench.class_bytes(k, vb, True) * n_valid * dn[k] for k in (6, 3, 0))
    assert math.isclose(r["gbs"], total_b / ((4.63 + 2.89 + 0.94) / 1e3) / 1e9)
    assert math.isclose(r["frac"], r["gbs"] / peak)
    assert math.isclose(r["time_share"], (4.63 + 2.89 + 0.94) / sum(dms))


def test_timed_class_bandwidth_without_launches():
    import bench
    r = bench.timed_class_bandwidth([0.0] * 12, [0] * 12, 8, False, 1000, 6800.0)
    assert r["gbs"] is None and r["frac"] is None and r["per_class_frac"] == {}


def test_parse_tune_reads_launch_choices():
    """--batch-tune: "key=value" pairs of the library's launch choices, every
    key one the binding maps; an empty value keeps the library's defaults."""
    import bench
    from paper_2007_02082_gb300 import _abi
    assert bench.parse_tune("") is None
    t = bench.parse_tune("mg_persist=2, poisson_kernel=3")
    assert t == {"mg_persist": 2, "poisson_kernel": 3}
    assert set(t) <= set(_abi.TUNE_INDEX)
