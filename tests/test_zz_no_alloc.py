"""The allocation-free sort entry point (pgs_sort_pairs_noalloc) against the
regular one (pgs_sort_pairs), both through the C ABI.

It serves callers that cannot allocate device memory (allocator callbacks,
frameworks that own all device memory, real-time paths), so its scratch is a
fixed array in the library's device image that every call reuses.  Two calls
in a row, the second smaller than the first, check that nothing left in that
array by one call leaks into the next.  Integer output: bit-exact.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well."""
import numpy as np
import pytest
import torch

from paper_2503_23044_b300 import binding as B

pytestmark = pytest.mark.gpu


def _pairs(n, seed, hi):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 4] = keys[n // 4: 2 * (n // 4)]           # repeated keys: stability matters
    return keys, np.arange(n, dtype=np.uint32)


def test_noalloc_sort_matches_regular_sort_on_two_calls_in_a_row():
    cases = [(B.NOALLOC_MAX_N, 1, (0, 32)), (100_003, 2, (0, 17)), (4097, 3, (5, 29))]
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, seed, bits in cases:
        keys, vals = _pairs(n, seed, 1 << 32)
        k_na = torch.tensor(keys.view(np.int32), device="cuda")
        v_na = torch.tensor(vals.view(np.int32), device="cuda")
        B.sort_pairs_noalloc(k_na, v_na, *bits, err=err)
        k_ref, v_ref, e_ref = B.sort_pairs(torch.tensor(keys.view(np.int32), device="cuda"),
                                           torch.tensor(vals.view(np.int32), device="cuda"), *bits)
        torch.cuda.synchronize()
        assert int(err.item()) == 0 and int(e_ref.item()) == 0
        assert torch.equal(k_na, k_ref), (n, bits)
        assert torch.equal(v_na, v_ref), (n, bits)


def test_noalloc_sort_allocates_nothing_after_the_warm_up_call():
    """After one warm-up call on the device (which may load the library's
    device code under lazy loading), a call changes neither the device's free
    memory nor torch's allocated bytes."""
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    keys, vals = _pairs(300_000, 7, 1 << 32)
    k = torch.tensor(keys.view(np.int32), device="cuda")
    v = torch.tensor(vals.view(np.int32), device="cuda")
    B.sort_pairs_noalloc(k.clone(), v.clone(), err=err)          # warm-up
    k_ref, v_ref, _ = B.sort_pairs(k.clone(), v.clone())
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    B.sort_pairs_noalloc(k, v, err=err)
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert (free0, alloc0) == (free1, alloc1), (free0 - free1, alloc1 - alloc0)
    assert int(err.item()) == 0
    assert torch.equal(k, k_ref) and torch.equal(v, v_ref)


def test_noalloc_sort_of_nothing():
    k = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert B.sort_pairs_noalloc(k, v)[0].numel() == 0
    B.check(B.lib().pgs_sort_pairs_noalloc(None, None, 0, 0, 32, None, None))   # n = 0 with null pointers


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    n = B.NOALLOC_MAX_N + 1
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(B.PGSError) as ei:
        B.sort_pairs_noalloc(k, v)
    assert ei.value.status == B.PGS_ERR_INVALID_ARG
    assert "fixed scratch" in str(ei.value)
