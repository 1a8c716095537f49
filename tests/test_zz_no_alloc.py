"""aaag_radix_sort_static: the radix sort for callers that cannot allocate
device memory (a plug-in whose host application owns every allocation, or a
real-time loop that must not wait on the allocator).  Its scratch is a fixed
array inside the library.  Checked through the C ABI against the allocating
entry point aaag_radix_sort and a CPU stable sort on two calls in a row, and
its failure report; this file is collected last so that a stop at the first
failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_2504_12811_gb300 import aaag

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


def reference_sort(keys, vals, key_bits):
    """Output of the existing entry point (caller-provided scratch)."""
    n = keys.size
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    k2, v2 = torch.empty_like(k), torch.empty_like(v)
    sb = aaag.aaag_radix_sort_scratch_bytes(n)
    scratch = torch.zeros(sb, dtype=torch.uint8, device="cuda")
    alt = aaag.aaag_radix_sort(k.data_ptr(), v.data_ptr(), k2.data_ptr(), v2.data_ptr(), n, key_bits,
                               scratch.data_ptr(), sb, aaag.current_stream())
    rk, rv = (k2, v2) if alt else (k, v)
    return rk.cpu().numpy().view(np.uint32), rv.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("first,second", [((300_001, 32), (70_003, 20)), ((1 << 20, 32), (4097, 13))])
def test_static_scratch_sort_matches_allocating_sort(first, second):
    rng = np.random.default_rng(first[0] + second[0])
    for n, key_bits in (first, second):          # two calls in a row share the scratch
        keys = rng.integers(0, 1 << key_bits, n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 4] = keys[0]                   # equal keys: stability
        vals = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        ref_k, ref_v = reference_sort(keys, vals, key_bits)
        k = torch.from_numpy(keys.view(np.int32)).cuda()
        v = torch.from_numpy(vals.view(np.int32)).cuda()
        aaag.aaag_radix_sort_static(k.data_ptr(), v.data_ptr(), n, key_bits, aaag.current_stream())
        torch.cuda.synchronize()
        assert aaag.aaag_radix_sort_static_status() == 0
        np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), ref_k)
        np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), ref_v)
        # and against a CPU stable sort of the same keys
        order = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(ref_k, keys[order])
        np.testing.assert_array_equal(ref_v, vals[order])


def test_static_scratch_sort_rejects_oversize():
    cap = aaag.aaag_radix_sort_static_capacity()
    assert cap == 1 << 20
    k = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(aaag.AaagError) as e:
        aaag.aaag_radix_sort_static(k.data_ptr(), k.data_ptr(), cap + 1, 32, aaag.current_stream())
    assert e.value.status == 2


def test_static_scratch_sort_reports_a_wait_that_gave_up():
    """The sort's bounded look-back wait, run out on purpose against the fixed
    array's own words (a predecessor that never publishes): it returns after
    about a second, the status query reports TIMEOUT, and the next sort clears
    the flag and sorts correctly."""
    import time
    st = aaag.current_stream()
    t0 = time.time()
    aaag.aaag_selftest_wait_timeout(None, 2, st)
    torch.cuda.synchronize()
    assert 0.2 < time.time() - t0 < 30.0
    assert aaag.aaag_radix_sort_static_status() == 4
    rng = np.random.default_rng(77)
    keys = rng.integers(0, 1 << 32, 5000, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(5000, dtype=np.uint32)
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    aaag.aaag_radix_sort_static(k.data_ptr(), v.data_ptr(), keys.size, 32, st)
    torch.cuda.synchronize()
    assert aaag.aaag_radix_sort_static_status() == 0
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), vals[order])
