"""ib_fields_get_noalloc: the allocation-free read of a parked problem's fields.

The file sorts last so that it also runs after every other GPU test in the
same process; run alone (`pytest tests/test_zz_no_alloc.py -m gpu`) it is the
first use of the library in a fresh process.  Both reads gather the same stored
values into canonical order, so the test tolerance is exact equality.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _parked(case, steps):
    """A deferred handle stepped inside a batch, then released by it."""
    from paper_2007_02082_gb300 import IBBatch, IBGrid
    g = IBGrid(case, precision="fp64", deferred=True)
    if steps:
        b = IBBatch([g])
        assert np.all(b.step(steps) == 0)
        b.close()
    return g


def test_noalloc_read_matches_fields_get_twice():
    g = _parked(W.cylinder_refined_small(n=(16, 16, 8), seed=41), 2)
    for name in ("U", "P", "PHI"):
        ref = g.ib_fields_get(name)
        assert np.abs(ref).max() > 0, name
        for _ in range(2):                        # two calls in a row
            got = g.ib_fields_get_noalloc(name)
            assert got.shape == ref.shape and got.dtype == ref.dtype
            assert np.array_equal(got, ref), name
    g.close()


def test_noalloc_device_destination():
    import torch
    g = _parked(W.cylinder_uniform_16x16x64(), 1)
    ref = g.ib_fields_get("U")
    out = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.zero_()
        g.ib_fields_get_noalloc("U", out=out)
        assert np.array_equal(out.cpu().numpy(), ref)
    # the binding refuses a destination of the wrong dtype, layout or shape
    with pytest.raises(ValueError):
        g.ib_fields_get_noalloc("U", out=torch.empty(ref.shape, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        g.ib_fields_get_noalloc("U", out=torch.empty((3, ref.shape[0]), dtype=torch.float64, device="cuda").t())
    with pytest.raises(ValueError):
        g.ib_fields_get_noalloc("U", out=torch.empty(ref.size, dtype=torch.float64, device="cuda"))
    g.close()


def test_noalloc_read_allocates_nothing():
    """The defining property: no device allocation, neither through the
    library's allocator callback nor in PyTorch's caching allocator."""
    import torch
    g = _parked(W.cylinder_refined_small(n=(16, 16, 8), seed=43), 1)
    ref = g.ib_fields_get("P")
    out = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    calls = g._alloc.calls
    before = torch.cuda.memory_stats()["allocation.all.allocated"]
    for _ in range(2):
        g.ib_fields_get_noalloc("P", out=out)
        host = g.ib_fields_get_noalloc("P")
    torch.cuda.synchronize()
    assert g._alloc.calls == calls
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == before
    assert np.array_equal(out.cpu().numpy(), ref) and np.array_equal(host, ref)
    # ib_fields_get on the same parked handle does allocate (a temporary gather buffer)
    g.ib_fields_get("P")
    assert g._alloc.calls > calls
    g.close()


def test_noalloc_rejects_oversize_and_non_parked():
    from paper_2007_02082_gb300 import IBBatch, IBError, IBGrid
    # 467k nodes: P (467k values) fits the 1,048,576-value scratch, U (1.4M) does not
    big = _parked(W.cylinder_case(n=(48, 48, 192), length=4.8, M=500, seed=42), 0)
    n = big.ib_grid_info()["n_nodes"]
    assert n <= 1 << 20 < 3 * n
    assert np.array_equal(big.ib_fields_get_noalloc("P"), big.ib_fields_get("P"))
    with pytest.raises(IBError) as ei:
        big.ib_fields_get_noalloc("U")
    assert ei.value.status == 1 and "exceeds the no-allocation scratch" in str(ei.value)
    big.close()
    # a standalone handle and a handle held by a batch are read with ib_fields_get
    case = W.cylinder_uniform_16x16x64()
    s = IBGrid(case, precision="fp64")
    with pytest.raises(IBError):
        s.ib_fields_get_noalloc("U")
    s.close()
    d = IBGrid(case, precision="fp64", deferred=True)
    b = IBBatch([d])
    with pytest.raises(IBError):
        d.ib_fields_get_noalloc("P")
    b.close()
    # fields other than U, P and Phi are not read here
    with pytest.raises(IBError):
        d.ib_fields_get_noalloc("F_LAG")
    d.close()
