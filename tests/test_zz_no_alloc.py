"""The allocation-free scan entry point (rgs_exclusive_scan_u32_static) against the allocating
one (rgs_exclusive_scan_u32), through the C ABI.

The static variant exists for callers that cannot allocate device memory at call time (a
real-time loop that must not block on the allocator, or a process whose device memory another
framework already holds). Its scratch is a fixed array inside the library shared by every call,
so the test runs it twice in a row on different inputs: a stale partial sum from the first call
would show up as a wrong second result. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_00705_gb300 import binding

pytestmark = pytest.mark.gpu


def _scan_both(ctx, lib, x):
    n = x.size
    xin = torch.from_numpy(x.view(np.int32)).cuda()
    ref = torch.empty_like(xin)
    out = torch.full_like(xin, -1)
    tot_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
    tot = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ctx.exclusive_scan_u32(xin.data_ptr(), ref.data_ptr(), n, tot_ref.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.rgs_exclusive_scan_u32_static(ctypes.c_void_p(xin.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), n,
                                           ctypes.c_void_p(tot.data_ptr()),
                                           ctypes.c_void_p(stream))
    assert st == binding.RGS_OK
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy(), int(tot_ref.item()), int(tot.item())


def test_static_scan_matches_allocating_scan_twice_in_a_row():
    lib = binding.load()
    ctx = binding.Context(0)
    rng = np.random.default_rng(123)
    # Two calls in a row, the second smaller than the first, so that any partial sum the first
    # call left in the shared scratch and the second call wrongly reused would be visible.
    for n in (3_000_017, 70_001):
        x = rng.integers(0, 1000, size=n).astype(np.uint32)
        ref, out, tot_ref, tot = _scan_both(ctx, lib, x)
        np.testing.assert_array_equal(out, ref)
        assert tot == tot_ref == int(x.astype(np.uint64).sum())
    ctx.close()


def test_static_scan_rejects_sizes_beyond_its_scratch():
    lib = binding.load()
    st = lib.rgs_exclusive_scan_u32_static(ctypes.c_void_p(16), ctypes.c_void_p(16),
                                           binding.RGS_STATIC_SCAN_MAX_N + 1, None, None)
    assert st == binding.RGS_ERR_TOO_LARGE
