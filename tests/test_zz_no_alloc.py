"""stark_mul_noalloc: the 3xBF16 product for callers that cannot allocate
device memory (code that may not enter an allocator, or that has a fixed
device-memory budget).  Through the C ABI, it must match stark_mul within
the tolerance the other split tests use, on two calls in a row, match the
FP64 oracle within the split bounds (including a size whose C the combine
reaches only by scalar atomics), allocate nothing, report device errors
through stark_noalloc_check, and reject problems larger than its fixed
scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1811_07325_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib(stark_lib):
    fn = stark_lib._lib.stark_mul_noalloc
    fn.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    chk = stark_lib._lib.stark_noalloc_check
    chk.argtypes = [ctypes.c_void_p]
    chk.restype = ctypes.c_int
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


@pytest.mark.parametrize("n,d", [(1001, 1), (256, 0), (512, 3), (1000, 2)])
def test_noalloc_matches_oracle(lib, n, d):
    # every element against the FP64 oracle, with the bars of the other split
    # tests: normwise max|dC| / (||A||_F ||B||_F) <= 1e-6 and the relative RMS
    # bug signal 2^-12 + 3 (L / 16) 2^-24.  n = 1001 (not a multiple of 4):
    # no staging copy of C exists here, so the combine adds by scalar atomics
    S, fn = lib
    A = synth.normal(n, 80 + n + d, 0)
    B = synth.normal(n, 80 + n + d, 1)
    want = oracle.gemm_classical(A.astype(np.float64), B.astype(np.float64))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.full((n, n), float("nan"), device="cuda")
    assert run_noalloc(fn, n, d, dA, dB, C) == 0
    assert S._lib.stark_noalloc_check(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    got = C.cpu().numpy().astype(np.float64)
    an, bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
    diff = got - want
    assert np.isfinite(got).all()
    assert np.abs(diff).max() / (an * bn) <= 1e-6
    L = (-(-n // (128 << d)) * (128 << d)) >> d
    rel = np.sqrt(np.mean(diff ** 2)) / np.sqrt(np.mean(want ** 2))
    assert rel <= 2.0 ** -12 + 3 * (L / 16) * 2.0 ** -24


def test_noalloc_check_reports_nothing_after_good_calls(lib):
    S, fn = lib
    n, d = 384, 1
    A = torch.from_numpy(synth.normal(n, 74, 0)).cuda()
    B = torch.from_numpy(synth.normal(n, 74, 1)).cuda()
    C = torch.empty((n, n), device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        assert run_noalloc(fn, n, d, A, B, C) == 0
    assert S._lib.stark_noalloc_check(s) == 0
    assert S._lib.stark_noalloc_check(s) == 0  # nothing left to report
