"""stark_error_norms: the FP64 error statistics reduced on the device, against
the same statistics computed on the host with numpy from the same data.

Maxima and componentwise ratios are exact (|g - w| and |g - w| / a are
correctly rounded FP64 operations on both sides, so they agree bit for bit);
sums of squares differ only in association, within n * 2^-52 relative."""
import numpy as np
import pytest

import oracle
from paper_1811_07325_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def host_stats(C, rows, want, absprod):
    got = C[rows].astype(np.float64)
    d = np.abs(got - want)
    comp = np.divide(d, absprod, out=np.zeros_like(d), where=absprod > 0)
    return d.max(), float(np.sum(d * d)), float(np.sum(want * want)), comp.max()


@pytest.mark.parametrize("n,d", [(1000, 2), (2048, 1), (77, 0)])
def test_error_norms_match_host_fp32(stark_lib, n, d):
    S = stark_lib
    A = synth.normal(n, 300 + n, 0)
    B = synth.normal(n, 300 + n, 1)
    rows = synth.sample_rows(n, min(n, 64), 301)
    want = oracle.gemm_rows(A, B, rows)
    absprod = oracle.gemm_rows(np.abs(A), np.abs(B), rows)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with S.Plan(n, d, S.DType.F32_SPLIT_BF16) as p:
        C = p.mul(dA, dB)
        p.check()
    rep = S.error_norms(dA, dB, C, rows, want, absprod)
    Ch = C.cpu().numpy()
    emax, e2, w2, cmax = host_stats(Ch, rows, want, absprod)
    tol = n * n * 2.0 ** -52
    assert rep["norm_a"] == pytest.approx(np.linalg.norm(A.astype(np.float64)), rel=tol)
    assert rep["norm_b"] == pytest.approx(np.linalg.norm(B.astype(np.float64)), rel=tol)
    assert rep["max_abs_err"] == emax
    assert rep["max_componentwise"] == cmax
    assert rep["sum_sq_err"] == pytest.approx(e2, rel=tol)
    assert rep["sum_sq_ref"] == pytest.approx(w2, rel=tol)
    assert rep["compared"] == rows.size * n
    assert rep["max_abs_over_normA_normB"] <= 1e-6


def test_error_norms_see_one_planted_error(stark_lib):
    # C holds the oracle's rows rounded to fp32; one entry of the reference
    # rows is moved by 3 on the CPU, and that entry is the maximum the
    # reduction reports
    S = stark_lib
    n = 512
    A = synth.normal(n, 310, 0)
    B = synth.normal(n, 310, 1)
    rows = np.arange(0, n, 8, dtype=np.int64)
    want = oracle.gemm_rows(A, B, rows)
    full = torch.zeros((n, n), device="cuda")
    full[torch.from_numpy(rows).cuda()] = torch.from_numpy(want.astype(np.float32)).cuda()
    want[5, 77] -= 3.0
    rep = S.error_norms(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), full, rows, want)
    assert rep["max_abs_err"] == pytest.approx(3.0, abs=1e-3)
    assert rep["max_componentwise"] == 0.0  # no absprod given


@pytest.mark.parametrize("dtype", ["F64", "I64"])
def test_error_norms_other_dtypes(stark_lib, dtype):
    S = stark_lib
    n = 300
    if dtype == "I64":
        A = synth.integers(n, 320, 0, -16, 16)
        B = synth.integers(n, 320, 1, -16, 16)
        want_full = oracle.gemm_classical(A, B).astype(np.float64)
    else:
        A = synth.uniform(n, 320, 0)
        B = synth.uniform(n, 320, 1)
        want_full = oracle.gemm_classical(A, B)
    rows = synth.sample_rows(n, 32, 321)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with S.Plan(n, 2, S.DType[dtype]) as p:
        C = p.mul(dA, dB)
        p.check()
    rep = S.error_norms(dA, dB, C, rows, want_full[rows])
    assert rep["norm_a"] == pytest.approx(np.linalg.norm(A.astype(np.float64)), rel=1e-12)
    assert rep["norm_b"] == pytest.approx(np.linalg.norm(B.astype(np.float64)), rel=1e-12)
    if dtype == "I64":
        assert rep["max_abs_err"] == 0.0 and rep["sum_sq_err"] == 0.0
    else:
        assert rep["max_abs_over_normA_normB"] <= 1e-12


def test_error_norms_norms_only_and_bad_args(stark_lib):
    S = stark_lib
    n = 128
    A = torch.ones((n, n), device="cuda")
    B = torch.full((n, n), 2.0, device="cuda")
    rep = S.error_norms(A, B)
    assert rep["norm_a"] == pytest.approx(n, rel=1e-15) and rep["norm_b"] == pytest.approx(2 * n, rel=1e-15)
    assert rep["compared"] == 0
    with pytest.raises(ValueError):
        S.error_norms(A, B, A, np.arange(4), None)
