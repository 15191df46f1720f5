"""GPU tests of the batched form (one grouped, graph-replayed leaf launch for
many products) and of the continuous-batching server, against the oracle and
against the same products computed alone."""
import time

import numpy as np
import pytest

import bounds
import oracle
from paper_1811_07325_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check(C, A, B, L, dtype="F32_SPLIT_BF16", rows=None):
    """Same bars as the single-product split tests (tests/bounds.py): every
    element within c S_ij of the oracle (S its error majorant; all rows
    compared, n <= 2048), 1e-6 normwise (n >= 64) and the relative-RMS model
    bound.  rows: compare those rows of C only."""
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    n = A.shape[0]
    d = bounds.infer_depth(n, L)
    if rows is None:
        want, got = oracle.gemm_classical(A64, B64), C
    else:
        want, got = oracle.gemm_rows(A64, B64, rows), C[rows]
    diff = got.astype(np.float64) - want
    if rows is None and n <= 2048:
        S = bounds.majorant(oracle, A64, B64, d, L)
        assert np.all(np.abs(diff) <= bounds.componentwise_c(dtype, L, d) * S)
    ratio = np.abs(diff).max() / (np.linalg.norm(A64) * np.linalg.norm(B64))
    rel = np.sqrt(np.mean(diff ** 2)) / np.sqrt(np.mean(want ** 2))
    if n >= 64:
        assert ratio <= 1e-6, ratio
        assert rel <= bounds.rms_bound(dtype, L, d), rel
    return want


@pytest.mark.parametrize("sizes,depth,dtype", [([512, 768, 1000, 300, 1536], -1, "F32_SPLIT_BF16"),
                                               ([1024, 2048, 512, 1536], 1, "F32_SPLIT_BF16"),
                                               ([640, 384, 1100], -1, "F32_SPLIT_TF32"),
                                               ([1000, 640, 2048, 384], 1, "F32_SPLIT_TF32")])
def test_batch_matches_oracle_and_replays(stark_lib, sizes, depth, dtype):
    S = stark_lib
    dt = S.DType[dtype]
    As = [synth.uniform(n, 300 + i, 0, dtype=np.float32) for i, n in enumerate(sizes)]
    Bs = [synth.uniform(n, 300 + i, 1, dtype=np.float32) for i, n in enumerate(sizes)]
    dA, dB = [dev(a) for a in As], [dev(b) for b in Bs]
    dC = [torch.full((n, n), float("nan"), device="cuda") for n in sizes]
    with S.Batch(sizes, depth, dt) as bt:
        depths = bt.depths()
        assert all(0 <= d <= 3 for d in depths)
        if depth >= 0:
            assert depths == [depth] * len(sizes)
        for rep in range(2):  # first call records the graph, second replays it
            bt.mul(dA, dB, dC)
            bt.check()
            for i, n in enumerate(sizes):
                L = (n + (128 << depths[i]) - 1) // (128 << depths[i]) * 128
                check(dC[i].cpu().numpy(), As[i], Bs[i], L, dtype)
            for c in dC:
                c.fill_(float("nan"))
        info = bt.info()
        assert info["graph_replays"] == 2 and info["work_items"] > 0
        # new C pointers: the graph is recorded again and stays correct
        dC2 = [torch.empty((n, n), device="cuda") for n in sizes]
        bt.mul(dA, dB, dC2)
        bt.check()
        for i, n in enumerate(sizes):
            L = (n + (128 << depths[i]) - 1) // (128 << depths[i]) * 128
            check(dC2[i].cpu().numpy(), As[i], Bs[i], L, dtype)


@pytest.mark.slow
def test_batch_of_64_members_matches_oracle(stark_lib):
    # the batched workload at its own size and in the bench's launch
    # configuration: 64 products, n drawn from {512, ..., 4096}, FP32
    # U[-1, 1], 3xBF16, depth and leaf tile autotuned, one grouped graph;
    # after a replay, 64 seeded rows of every member against the oracle
    S = stark_lib
    sizes = synth.batch_sizes(64, 2024 + 11)
    As = [synth.uniform(n, 2024 + 100 + i, 0, dtype=np.float32) for i, n in enumerate(sizes)]
    Bs = [synth.uniform(n, 2024 + 100 + i, 1, dtype=np.float32) for i, n in enumerate(sizes)]
    dA, dB = [dev(a) for a in As], [dev(b) for b in Bs]
    dC = [torch.full((n, n), float("nan"), device="cuda") for n in sizes]
    with S.Batch(sizes, -1, S.DType.F32_SPLIT_BF16) as bt:
        depths, tiles = bt.depths(), bt.tiles()
        assert all(t in (128, 256) for t in tiles)
        for _ in range(2):
            bt.mul(dA, dB, dC)
        bt.check()
        assert bt.info()["graph_replays"] >= 2
    for i, n in enumerate(sizes):
        L = (n + (128 << depths[i]) - 1) // (128 << depths[i]) * 128
        rows = synth.sample_rows(n, 64, 900 + i)
        check(dC[i].cpu().numpy(), As[i], Bs[i], L, rows=rows)


def test_batch_rejects_bad_arguments(stark_lib):
    S = stark_lib
    with pytest.raises(S.StarkError):
        S.Batch([], -1)
    with pytest.raises(S.StarkError):
        S.Batch([0, 64], -1)
    with pytest.raises(S.StarkError):
        S.Batch([64], -1, S.DType.F64)


def wait_all(srv, ids, timeout=120.0):
    pending, status = set(ids), {}
    t0 = time.time()
    while pending:
        for rid in list(pending):
            done, st = srv.poll(rid)
            if done:
                status[rid] = st
                pending.discard(rid)
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.0005)
    return status


def test_server_results_equal_solo_and_oracle(stark_lib):
    S = stark_lib
    sizes = [256, 1200, 300, 777, 2048, 513, 1024, 4096, 260, 1500]
    As = [synth.normal(n, 400 + i, 0) for i, n in enumerate(sizes)]
    Bs = [synth.normal(n, 400 + i, 1) for i, n in enumerate(sizes)]
    dA, dB = [dev(a) for a in As], [dev(b) for b in Bs]
    dC = [torch.empty((n, n), device="cuda") for n in sizes]
    torch.cuda.synchronize()
    with S.Server(16 << 30, slots=3) as srv:
        ids = [srv.submit(dA[i], dB[i], dC[i]) for i in range(len(sizes))]  # arrive while others run
        status = wait_all(srv, ids)
        assert all(st == S.Status.OK for st in status.values())
        lat = [srv.latency(r) for r in ids]
        assert all(x > 0 for x in lat)
        with pytest.raises(S.StarkError):  # reaped
            srv.poll(ids[0])
        st = srv.stats()
        assert st["owned_bytes"] <= 16 << 30 and st["queued"] == 0
    for i, n in enumerate(sizes):
        with S.Plan(n, -1, S.DType.F32_SPLIT_BF16) as p:
            solo = p.mul(dA[i], dB[i])
            p.check()
            L = p.leaf
        # the same product alone and in the mix: same kernels, only the
        # order of the combine's additions into C differs
        assert (dC[i] - solo).abs().max().item() <= 1e-5 * solo.abs().max().item(), n
        if n <= 2048:
            check(dC[i].cpu().numpy(), As[i], Bs[i], L)


def test_server_admission_under_small_budget(stark_lib):
    S = stark_lib
    # budget for about one n=1024 workspace at a time: requests queue and are
    # admitted as memory frees up; each still completes correctly
    sizes = [1024, 1000, 1024, 900, 1024, 1010]
    As = [synth.integers(n, 500 + i, 0, -16, 16) for i, n in enumerate(sizes)]
    Bs = [synth.integers(n, 500 + i, 1, -16, 16) for i, n in enumerate(sizes)]
    dA, dB = [dev(a) for a in As], [dev(b) for b in Bs]
    dC = [torch.empty((n, n), dtype=torch.int64, device="cuda") for n in sizes]
    torch.cuda.synchronize()
    budget = 60 << 20
    with S.Server(budget, slots=4) as srv:
        ids = [srv.submit(dA[i], dB[i], dC[i], S.DType.I64) for i in range(len(sizes))]
        status = wait_all(srv, ids)
        assert all(st == S.Status.OK for st in status.values())
        assert srv.stats()["owned_bytes"] <= budget
        big = torch.zeros((8192, 8192), dtype=torch.int64, device="cuda")
        with pytest.raises(S.StarkError) as e:
            srv.submit(big, big, big, S.DType.I64)
        assert e.value.status == S.Status.ENOMEM
    for i, n in enumerate(sizes):
        assert np.array_equal(dC[i].cpu().numpy(), oracle.gemm_classical(As[i], Bs[i])), n


def _dispatch_depth(S, dtype, candidates):
    """First candidate size whose automatic depth (the one the dispatcher takes:
    measured for the split dtypes and cached per process, the cost model
    otherwise) has a depth-first traversal, with that depth and leaf side."""
    for n in candidates:
        with S.Plan(n, -1, dtype) as p:
            d, L = p.depth, p.leaf
        if 1 <= d <= 3:
            return n, d, L
    pytest.skip("no candidate size with a depth the depth-first traversal serves")


@pytest.mark.parametrize("dtype,candidates", [("F32_SPLIT_BF16", (4096, 3072, 2048, 6144)),
                                              ("F64", (1024, 1536, 768)),
                                              ("I64", (1024, 1536, 768))])
def test_server_admits_depth_first_beyond_breadth_first_budget(stark_lib, dtype, candidates):
    S = stark_lib
    dt = getattr(S.DType, dtype)
    n, d, L = _dispatch_depth(S, dt, candidates)
    per = 4 if dtype == "F32_SPLIT_BF16" else 8  # hi+lo bf16, or one 8-byte value per operand element
    breadth_first = 2 * 7 ** d * L * L * per
    budget = breadth_first // 2  # the breadth-first workspace never fits; one subtree's does
    sizes = [n, n - 3, n - 64]   # one padded bucket; n - 3 is not a TMA target (staged C)
    if dtype == "F32_SPLIT_BF16":
        As = [synth.normal(m, 700 + i, 0) for i, m in enumerate(sizes)]
        Bs = [synth.normal(m, 700 + i, 1) for i, m in enumerate(sizes)]
        tdt = torch.float32
    elif dtype == "F64":
        As = [synth.uniform(m, 700 + i, 0) for i, m in enumerate(sizes)]
        Bs = [synth.uniform(m, 700 + i, 1) for i, m in enumerate(sizes)]
        tdt = torch.float64
    else:
        As = [synth.integers(m, 700 + i, 0, -(1 << 20), 1 << 20) for i, m in enumerate(sizes)]
        Bs = [synth.integers(m, 700 + i, 1, -(1 << 20), 1 << 20) for i, m in enumerate(sizes)]
        tdt = torch.int64
    dA, dB = [dev(a) for a in As], [dev(b) for b in Bs]
    dC = [torch.full((m, m), 7, dtype=tdt, device="cuda") for m in sizes]  # overwritten
    torch.cuda.synchronize()
    with S.Server(budget, slots=2) as srv:
        ids = [srv.submit(dA[i], dB[i], dC[i], dt) for i in range(len(sizes))]
        status = wait_all(srv, ids)
        assert all(st == S.Status.OK for st in status.values()), status
        st = srv.stats()
        assert 0 < st["owned_bytes"] <= budget < breadth_first
    for i, m in enumerate(sizes):
        got = dC[i].cpu().numpy()
        if dtype == "I64":
            assert np.array_equal(got, oracle.gemm_classical(As[i], Bs[i])), m
            continue
        with S.Plan(m, d, dt) as p:  # breadth first, alone
            solo = p.mul(dA[i], dB[i])
            p.check()
        # same leaf kernels; only the order of the combine's additions differs
        assert (dC[i] - solo).abs().max().item() <= 1e-5 * solo.abs().max().item(), m
        rows = np.unique(np.concatenate([np.arange(0, m, 97), [m - 1]]))
        want = oracle.gemm_rows(As[i], Bs[i], rows)
        ratio = np.abs(got[rows].astype(np.float64) - want).max() / (
            np.linalg.norm(As[i].astype(np.float64)) * np.linalg.norm(Bs[i].astype(np.float64)))
        assert ratio <= (1e-6 if dtype == "F32_SPLIT_BF16" else 1e-12), (m, ratio)


def test_server_falls_back_to_a_depth_that_fits(stark_lib):
    S = stark_lib
    # FP64, side 1024: at depth 1 one subtree's operands are 2 x 512^2 x 8 B =
    # 4 MiB (+ 1 MiB margin for the tables).  Deeper or breadth-first
    # workspaces are larger, so under this budget every request runs at depth
    # 1 depth first, one workspace at a time
    budget = (5 << 20) + (512 << 10)
    sizes = [1024, 1021, 1024]
    As = [synth.uniform(m, 800 + i, 0) for i, m in enumerate(sizes)]
    Bs = [synth.uniform(m, 800 + i, 1) for i, m in enumerate(sizes)]
    dA, dB = [dev(a) for a in As], [dev(b) for b in Bs]
    dC = [torch.empty((m, m), dtype=torch.float64, device="cuda") for m in sizes]
    torch.cuda.synchronize()
    with S.Server(budget, slots=3) as srv:
        ids = [srv.submit(dA[i], dB[i], dC[i], S.DType.F64) for i in range(len(sizes))]
        status = wait_all(srv, ids)
        assert all(st == S.Status.OK for st in status.values()), status
        st = srv.stats()
        assert st["cached_workspaces"] == 1 and 0 < st["owned_bytes"] <= budget
        with pytest.raises(S.StarkError) as e:  # below one subtree at any depth
            srv.submit(*[torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")] * 3, S.DType.F64)
        assert e.value.status == S.Status.ENOMEM
    for i, m in enumerate(sizes):
        A64, B64 = As[i], Bs[i]
        diff = dC[i].cpu().numpy() - oracle.gemm_classical(A64, B64)
        assert np.abs(diff).max() / (np.linalg.norm(A64) * np.linalg.norm(B64)) <= 1e-12, m


def test_server_unknown_id(stark_lib):
    S = stark_lib
    with S.Server(1 << 30, slots=1) as srv:
        with pytest.raises(S.StarkError) as e:
            srv.poll(12345)
        assert e.value.status == S.Status.ENOTFOUND
