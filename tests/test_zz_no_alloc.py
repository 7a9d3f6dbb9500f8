"""zd_morton_sort_noalloc: the sort for callers that may not allocate device
memory on their call path (a plug-in inside a host framework that has
reserved the GPU's memory for its own pool, or a latency-critical loop that
must not wait on an allocation).  It keeps its scratch in a static device
array of the library instead of allocating.

Checked through the C ABI against the allocating zd_morton_sort on two calls
in a row -- the second call must not see the first call's leftovers in the
shared array -- and on the size limit.  Kept in a file of its own that runs
last, so a stop-at-first-failure run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_04182_gb300 import zd

    return zd


def _call_noalloc(zd, keys, key_bits, out_k, out_p):
    return zd._lib().zd_morton_sort_noalloc(C.c_void_p(keys.data_ptr()), keys.numel(), key_bits,
                                            C.c_void_p(out_k.data_ptr()), C.c_void_p(out_p.data_ptr()),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_sort_matches_allocating_sort_twice(lib):
    zd = lib
    rng = np.random.default_rng(2024)
    cases = [
        # a full-size call with 63-bit keys and many ties, then a smaller one
        # with fewer key bits: leftovers of the first must not leak into it
        (np.concatenate([rng.integers(0, 2 ** 63, size=zd.ZD_NOALLOC_MAX_KEYS - 4096, dtype=np.int64),
                         np.full(4096, 77, np.int64)]), 63),
        (rng.integers(0, 1 << 20, size=300_001, dtype=np.int64), 20),
        # then larger again with all 64 bits (eight passes): the tile counters
        # of this call sit inside the look-back words the earlier, smaller
        # calls left behind, so those must be cleared before it starts
        (rng.integers(-2 ** 63, 2 ** 63 - 1, size=zd.ZD_NOALLOC_MAX_KEYS - 777, dtype=np.int64), 64),
    ]
    for keys_np, bits in cases:
        keys = torch.from_numpy(keys_np).cuda()
        ref_k, ref_p = zd.zd_morton_sort(keys, bits)
        out_k = torch.full_like(keys, -1)
        out_p = torch.full((keys.numel(),), -1, dtype=torch.int32, device=keys.device)
        assert _call_noalloc(zd, keys, bits, out_k, out_p) == zd.ZD_OK
        assert zd.zd_check() == zd.ZD_OK
        assert torch.equal(out_k, ref_k)
        assert torch.equal(out_p, ref_p)
        # and both agree with a stable lexsort on the host
        want = np.lexsort((np.arange(len(keys_np)), keys_np.view(np.uint64)))
        assert np.array_equal(out_p.cpu().numpy(), want)


def test_noalloc_sort_rejects_oversize_and_empty(lib):
    zd = lib
    big = torch.zeros(zd.ZD_NOALLOC_MAX_KEYS + 1, dtype=torch.int64, device="cuda")
    out_k = torch.empty_like(big)
    out_p = torch.empty(big.numel(), dtype=torch.int32, device="cuda")
    assert _call_noalloc(zd, big, 64, out_k, out_p) == zd.ZD_ERR_CAPACITY
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    assert _call_noalloc(zd, empty, 64, empty, torch.empty(0, dtype=torch.int32, device="cuda")) == zd.ZD_OK
    assert zd.zd_check() == zd.ZD_OK


def test_noalloc_wrapper_with_caller_buffers(lib):
    """The Python wrapper with caller-supplied outputs allocates nothing and
    gives the allocating sort's result; mismatched outputs are refused on the
    host before anything runs."""
    zd = lib
    rng = np.random.default_rng(7)
    keys = torch.from_numpy(rng.integers(0, 1 << 40, size=65_537, dtype=np.int64)).cuda()
    ref_k, ref_p = zd.zd_morton_sort(keys, 40)
    out = (torch.empty_like(keys), torch.empty(keys.numel(), dtype=torch.int32, device="cuda"))
    got = zd.zd_morton_sort_noalloc(keys, 40, out=out)
    assert got[0] is out[0] and got[1] is out[1]
    assert torch.equal(out[0], ref_k) and torch.equal(out[1], ref_p)
    bad = [
        (out[0][:-1], out[1]),                                  # too short
        (out[0], out[1].to(torch.int64)),                       # wrong dtype
        (torch.empty(2 * keys.numel(), dtype=torch.int64, device="cuda")[::2], out[1]),  # not contiguous
        (out[0].cpu(), out[1]),                                 # wrong device
    ]
    for b in bad:
        with pytest.raises(ValueError):
            zd.zd_morton_sort_noalloc(keys, 40, out=b)
