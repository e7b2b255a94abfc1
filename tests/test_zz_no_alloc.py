"""vegas_allocate_static, the allocation entry point that allocates nothing.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator, or they run in loops where an allocation would synchronise the
device.  For them the allocation step has a variant whose scratch is a fixed
array inside the library.  This test calls it through the C ABI, twice in a
row on different inputs, and checks that its offsets equal those of
vegas_allocate, bit for bit (the offsets are integers).  The second call runs
on inputs of a different size, so anything the first call left in the shared
array would show.  The file is collected last, so a run that stops at its
first failure has run every other test before this one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    import __graft_entry__ as g
    g.build()
    from paper_2408_09229_gb300 import vegas
    assert torch.cuda.is_available()
    return vegas


def _offsets(V, fn, ell, nh, neval, uniform):
    off = torch.full((nh + 1,), -1, dtype=torch.int64, device="cuda")
    e = torch.as_tensor(ell).cuda() if ell is not None else None
    if fn == "static":
        V.allocate_static(e, nh, neval, uniform, off)
    else:
        scratch = torch.empty(V.allocate_scratch_bytes(nh), dtype=torch.uint8, device="cuda")
        V.allocate(e, nh, neval, uniform, off, scratch)
    torch.cuda.synchronize()
    return off.cpu().numpy()


def test_static_matches_allocate_on_two_calls_in_a_row(V):
    rng = np.random.default_rng(2024)
    cases = [(1_000_003, 3_000_001), (38_416, 100_000 - 2 * 38_416)]  # second call: a smaller problem
    for nh, extra in cases:
        ell = rng.normal(-2, 5, nh).astype(np.float32)
        ell[rng.random(nh) < 0.05] = -np.inf
        neval = 2 * nh + extra
        got = _offsets(V, "static", ell, nh, neval, False)
        want = _offsets(V, "scratch", ell, nh, neval, False)
        assert np.array_equal(got, want)
        assert got[0] == 0 and got[-1] == neval and np.diff(got).min() >= 2
    # the uniform allocation through the same array
    got = _offsets(V, "static", None, 4097, 77_777, True)
    assert np.array_equal(got, _offsets(V, "scratch", None, 4097, 77_777, True))


def test_static_rejects_sizes_beyond_its_limit(V):
    off = torch.empty(1, dtype=torch.int64, device="cuda")
    with pytest.raises(V.VegasError) as e:
        V.allocate_static(None, V.ALLOCATE_STATIC_MAX_CUBES + 1, 2 ** 31 - 1, True, off)
    assert e.value.status == V.ENOSPACE
