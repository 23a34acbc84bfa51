"""The single-pass scan (one launch, decoupled look-back between blocks) that the forward's
compaction and pair offsets run on, through rgs_exclusive_scan_u32_single_pass:
  * exclusive prefix sums equal numpy's (u32, wrapping like the device) at sizes around the
    4096-element tile (1, one tile, one tile + 1, ragged multiples, 2^20 + 3, 5M), also in place;
  * n = 0 writes a zero total;
  * its wait is bounded: with the ticket counter started at 1 instead of 0, tile 0 is never
    published, the blocks waiting for it give up after their poll limit (about a second),
    report status bit 4 and return; the context stays usable and the next scan is right;
  * bad arguments are refused before any GPU work.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

from paper_2601_00705_gb300 import binding

pytestmark = pytest.mark.gpu


def _scan(lib, x, out, work, status, total=None):
    n = x.numel()
    return lib.rgs_exclusive_scan_u32_single_pass(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
        ctypes.c_void_p(total.data_ptr() if total is not None else None),
        ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.c_void_p(status.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _zeroed_area(lib, n):
    nbytes = int(lib.rgs_single_pass_scan_bytes(n))
    return torch.zeros(nbytes, dtype=torch.uint8, device="cuda")


def _u32(a):
    return torch.from_numpy(a.astype(np.int64).astype(np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 3 * 4096 + 5, 200 * 4096 - 1, (1 << 20) + 3,
                               5_000_000])
def test_matches_numpy(n):
    lib = binding.load()
    rng = np.random.default_rng(n)
    a = rng.integers(0, 2000, size=n).astype(np.uint32)
    x = _u32(a)
    out = torch.empty_like(x)
    total = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = _zeroed_area(lib, n)
    assert _scan(lib, x, out, work, status, total) == 0
    torch.cuda.synchronize()
    ref = np.concatenate([[0], np.cumsum(a, dtype=np.uint32)[:-1]]).astype(np.uint32)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref)
    assert int(total.cpu().numpy().view(np.uint32)[0]) == int(np.sum(a, dtype=np.uint32))
    assert int(status.item()) == 0
    # In place, with the work area zeroed again.
    work.zero_()
    assert _scan(lib, x, x, work, status) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy().view(np.uint32), ref)
    assert int(status.item()) == 0


def test_empty_input_writes_zero_total():
    lib = binding.load()
    x = torch.zeros(1, dtype=torch.int32, device="cuda")
    total = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = _zeroed_area(lib, 0)
    assert lib.rgs_exclusive_scan_u32_single_pass(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0,
        ctypes.c_void_p(total.data_ptr()), ctypes.c_void_p(work.data_ptr()), work.numel(),
        ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(0)) == 0
    torch.cuda.synchronize()
    assert int(total.item()) == 0


def test_wait_for_an_unpublished_tile_is_bounded_and_reported():
    lib = binding.load()
    n = 3 * 4096
    x = _u32(np.ones(n, np.uint32))
    out = torch.empty_like(x)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = _zeroed_area(lib, n)
    work[0] = 1  # ticket counter starts at 1: no block takes tile 0, which nothing publishes
    t0 = time.time()
    assert _scan(lib, x, out, work, status) == 0
    torch.cuda.synchronize()
    elapsed = time.time() - t0
    assert int(status.item()) & 4
    assert elapsed < 30.0, elapsed
    # The context is still usable and the next scan is right.
    work.zero_()
    status.zero_()
    assert _scan(lib, x, out, work, status) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), np.arange(n))
    assert int(status.item()) == 0


def test_bad_arguments_are_refused():
    lib = binding.load()
    x = torch.zeros(4096, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = _zeroed_area(lib, 4096)
    small = int(lib.rgs_single_pass_scan_bytes(4096)) - 8
    p = ctypes.c_void_p
    assert lib.rgs_exclusive_scan_u32_single_pass(p(x.data_ptr()), p(x.data_ptr()), 4096, None,
                                                  p(work.data_ptr()), small,
                                                  p(status.data_ptr()), None) == binding.RGS_ERR_INVALID_ARG
    assert lib.rgs_exclusive_scan_u32_single_pass(p(x.data_ptr()), p(x.data_ptr()), 4096, None,
                                                  p(work.data_ptr() + 8), work.numel(),
                                                  p(status.data_ptr()), None) == binding.RGS_ERR_INVALID_ARG
    assert lib.rgs_exclusive_scan_u32_single_pass(p(x.data_ptr()), p(x.data_ptr()), -1, None,
                                                  p(work.data_ptr()), work.numel(),
                                                  p(status.data_ptr()), None) == binding.RGS_ERR_INVALID_ARG
    assert lib.rgs_exclusive_scan_u32_single_pass(p(x.data_ptr()), p(x.data_ptr()), 4096, None,
                                                  p(work.data_ptr()), work.numel(), None,
                                                  None) == binding.RGS_ERR_INVALID_ARG
