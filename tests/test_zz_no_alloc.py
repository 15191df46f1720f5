"""stark_mul_noalloc: the 3xBF16 product for callers that cannot allocate
device memory (code that may not enter an allocator, or that has a fixed
device-memory budget).  Through the C ABI, it must match stark_mul within
the tolerance the other split tests use, on two calls in a row, allocate
nothing, and reject problems larger than its fixed scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1811_07325_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib(stark_lib):
    fn = stark_lib._lib.stark_mul_noalloc
    fn.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return stark_lib, fn


def run_noalloc(fn, n, depth, A, B, C):
    s = torch.cuda.current_stream().cuda_stream
    return fn(n, depth, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
              ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(s))


def test_noalloc_matches_stark_mul_twice(lib):
    S, fn = lib
    cases = [(1000, 1, 71), (512, 2, 72)]  # two calls in a row, different sizes and depths
    ref, outs = [], []
    for n, d, seed in cases:
        A = torch.from_numpy(synth.normal(n, seed, 0)).cuda()
        B = torch.from_numpy(synth.normal(n, seed, 1)).cuda()
        with S.Plan(n, d, S.DType.F32_SPLIT_BF16) as p:
            ref.append(p.mul(A, B))
            p.check()
        outs.append((n, d, A, B, torch.full((n, n), float("nan"), device="cuda")))
    torch.cuda.synchronize()
    for n, d, A, B, C in outs:
        assert run_noalloc(fn, n, d, A, B, C) == 0
    torch.cuda.synchronize()
    for (n, d, A, B, C), R in zip(outs, ref):
        # same kernels, only the order of the additions into C may differ:
        # the bound of the combine-mode test
        assert torch.isfinite(C).all()
        assert (C - R).abs().max().item() <= 1e-5 * R.abs().max().item()


def test_noalloc_allocates_nothing(lib):
    S, fn = lib
    n, d = 768, 1
    A = torch.from_numpy(synth.normal(n, 73, 0)).cuda()
    B = torch.from_numpy(synth.normal(n, 73, 1)).cuda()
    C = torch.empty((n, n), device="cuda")
    assert run_noalloc(fn, n, d, A, B, C) == 0  # first call on the device does the set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert run_noalloc(fn, n, d, A, B, C) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < (2 << 20)  # no device allocation (slack for driver bookkeeping)


def test_noalloc_rejects_oversize_and_bad_args(lib):
    S, fn = lib
    n = 4096  # 3xBF16 workspace at depth 1 is ~235 MB, far above the 64 MiB scratch
    A = torch.zeros((n, n), device="cuda")
    assert run_noalloc(fn, n, 1, A, A, A) == S.Status.ENOMEM
    assert run_noalloc(fn, 64, 4, A, A, A) == S.Status.EINVAL
    assert fn(64, 1, None, None, None, None) == S.Status.EINVAL
