"""The allocation-free scan entry point, rgs_exclusive_scan_u32_static, through the C ABI.

The static variant exists for callers that cannot allocate device memory at call time (a
real-time loop that must not block on the allocator, or a process whose device memory another
framework already holds). Its scratch is a fixed array inside the library shared by every call.
Each case is checked against numpy's cumulative sum (not against the allocating scan, which runs
the same kernels) and, where the allocating scan accepts it, against that scan too. The sizes run
in sequence on one device, so a partial sum that a call left in the shared scratch and the next
call wrongly reused would show: n = 0, 1, 65,536 (the single-cluster path, which needs no
scratch), sizes around the 4096-element block, a few million, then RGS_STATIC_SCAN_MAX_N - 1 and
RGS_STATIC_SCAN_MAX_N (every scratch slot, and the grand-total slot after them), then small again.

The file name sorts after every other test file, so a run that stops at the first failure has
run every other test before this one; nothing here depends on the order.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_00705_gb300 import binding

pytestmark = pytest.mark.gpu

MAX_N = binding.RGS_STATIC_SCAN_MAX_N


def _static_scan(lib, xin, n, stream):
    out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    tot = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = lib.rgs_exclusive_scan_u32_static(ctypes.c_void_p(xin.data_ptr() if n else 0),
                                           ctypes.c_void_p(out.data_ptr() if n else 0), n,
                                           ctypes.c_void_p(tot.data_ptr()),
                                           ctypes.c_void_p(stream))
    assert st == binding.RGS_OK
    torch.cuda.synchronize()  # the static scan is asynchronous on its stream
    return out[:n].cpu().numpy().view(np.uint32), int(tot.cpu().numpy().view(np.uint32)[0])


def test_static_scan_matches_numpy_in_sequence():
    lib = binding.load()
    ctx = binding.Context(0)
    rng = np.random.default_rng(123)
    stream = torch.cuda.current_stream().cuda_stream
    for n in (3_000_017, 70_001, 0, 1, 65_536, 4095, 4096, 4097, MAX_N - 1, MAX_N, 12_289):
        hi = 64 if n >= MAX_N - 1 else 1000  # keep the grand total below 2^32
        x = rng.integers(0, hi, size=n).astype(np.uint32)
        xin = torch.from_numpy(x.view(np.int32)).cuda() if n else torch.zeros(1, device="cuda")
        out, tot = _static_scan(lib, xin, n, stream)
        expect = np.concatenate([[0], np.cumsum(x, dtype=np.uint64)[:-1]]) if n else np.zeros(0)
        np.testing.assert_array_equal(out.astype(np.uint64), expect.astype(np.uint64), err_msg=f"n={n}")
        assert tot == int(x.astype(np.uint64).sum()), (n, tot)
        if 0 < n < (1 << 31):
            ref = torch.empty_like(xin)
            tot_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
            ctx.exclusive_scan_u32(xin.data_ptr(), ref.data_ptr(), n, tot_ref.data_ptr())
            np.testing.assert_array_equal(out, ref.cpu().numpy().view(np.uint32))
        del xin
    ctx.close()


def test_static_scan_rejects_sizes_beyond_its_scratch():
    lib = binding.load()
    st = lib.rgs_exclusive_scan_u32_static(ctypes.c_void_p(16), ctypes.c_void_p(16),
                                           MAX_N + 1, None, None)
    assert st == binding.RGS_ERR_TOO_LARGE
    st = lib.rgs_exclusive_scan_u32_static(None, None, 5, None, None)
    assert st == binding.RGS_ERR_INVALID_ARG
