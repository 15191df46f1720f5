"""Multi-device bookkeeping on CPU: world size 2 over gloo.

The real sharding code (``shard.mul_sharded``) runs with a CPU stand-in for
the plan whose ``mul_leaves`` forms the partial product of a leaf range from
the oracle's leaf operands and the library's quadrant-index table (host-only
calls).  The ranks' partial products must all-reduce to A.B exactly (int64),
and a rank that fails before the collective must make the other rank's
collective end with an error rather than hang."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1811_07325_gb300 import shard, synth  # noqa: E402


def test_leaf_range_partitions():
    for leaves in (1, 7, 49, 343, 2401):
        for world in (1, 2, 3, 8):
            spans = [shard.leaf_range(leaves, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == leaves
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.leaf_range(7, 2, 2)


class CpuLeafPlan:
    """CPU stand-in: partial product of a leaf range (oracle operands + table).

    ``set_shard`` restricts it like ``stark_plan_set_shard``: it then keeps
    the operands of the subtrees (below min(2, depth) top levels) that hold
    its leaves and refuses ranges outside its shard."""

    def __init__(self, n, depth, npad):
        from paper_1811_07325_gb300 import stark
        self.n, self.depth, self.npad = n, depth, npad
        self.leaves = 7 ** depth
        self.count, self.quad, self.sign = stark.quadrant_table(depth, 2)
        self.first, self.kept = 0, self.leaves

    def set_shard(self, begin, end):
        gs = 7 ** (self.depth - min(2, self.depth))
        self.first = begin // gs * gs
        self.kept = -(-end // gs) * gs - self.first
        self.shard = (begin, end)

    def offsets(self, q):
        r = c = 0
        for k in range(1, self.depth + 1):
            digit = (q >> (2 * (self.depth - k))) & 3
            r += (digit >> 1) * (self.npad >> k)
            c += (digit & 1) * (self.npad >> k)
        return r, c

    def mul_leaves(self, A, B, begin, end, C=None, stream=None):
        import oracle
        if not (self.first <= begin <= end <= self.first + self.kept):
            raise ValueError("leaves outside the shard")
        L = self.npad >> self.depth
        keep = slice(self.first, self.first + self.kept)  # this rank's subtrees only
        X = oracle.strassen_operands(A.numpy().astype(np.float32), self.npad, self.depth, "A")[keep].astype(np.int64)
        Y = oracle.strassen_operands(B.numpy().astype(np.float32), self.npad, self.depth, "B")[keep].astype(np.int64)
        Cp = np.zeros((self.npad, self.npad), np.int64)
        for leaf in range(begin, end):
            M = X[leaf - self.first] @ Y[leaf - self.first]
            for t in range(self.count[leaf]):
                r, c = self.offsets(int(self.quad[leaf, t]))
                Cp[r:r + L, c:c + L] += int(self.sign[leaf, t]) * M
        C.copy_(torch.from_numpy(Cp[:self.n, :self.n]))
        return C


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, depth, npad, out_path, fail_rank, rows=False):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    try:
        A = torch.from_numpy(synth.integers(n, 77, 0, -16, 16))
        B = torch.from_numpy(synth.integers(n, 77, 1, -16, 16))
        C = torch.zeros((n, n), dtype=torch.int64)
        if rank == fail_rank:
            raise SystemExit(3)  # this rank dies before the collective
        try:
            plan = CpuLeafPlan(n, depth, npad)
            plan.set_shard(*shard.leaf_range(plan.leaves, world, rank))  # as shard.shard_plan does
            if rows:
                r0, r1, blk = shard.mul_sharded_rows(plan, A, B)
                np.save(f"{out_path}.{rank}.npy", blk[:r1 - r0].numpy())
                np.save(f"{out_path}.{rank}.span.npy", np.array([r0, r1]))
            else:
                shard.mul_sharded(plan, A, B, C)
                np.save(f"{out_path}.{rank}.npy", C.numpy())
        except Exception as e:  # the collective must fail, not hang
            with open(f"{out_path}.{rank}.err", "w") as f:
                f.write(type(e).__name__)
    finally:
        if rank != fail_rank:
            dist.destroy_process_group()


@pytest.mark.parametrize("n,depth,npad", [(40, 2, 64), (33, 1, 64)])
def test_two_ranks_all_reduce_to_product(tmp_path, n, depth, npad):
    import oracle
    out = str(tmp_path / "c")
    mp.start_processes(_worker, args=(2, _free_port(), n, depth, npad, out, -1), nprocs=2, start_method="spawn")
    want = oracle.gemm_classical(synth.integers(n, 77, 0, -16, 16), synth.integers(n, 77, 1, -16, 16))
    for r in range(2):
        assert np.array_equal(np.load(f"{out}.{r}.npy"), want)


@pytest.mark.parametrize("n,depth,npad", [(40, 2, 64), (33, 1, 64)])
def test_two_ranks_reduce_scatter_rows(tmp_path, n, depth, npad):
    # each rank ends with its block of rows of the exact product; the blocks
    # tile [0, n) (n = 33: blocks of 17 and 16 rows)
    import oracle
    out = str(tmp_path / "c")
    mp.start_processes(_worker, args=(2, _free_port(), n, depth, npad, out, -1, True), nprocs=2,
                       start_method="spawn")
    want = oracle.gemm_classical(synth.integers(n, 77, 0, -16, 16), synth.integers(n, 77, 1, -16, 16))
    spans = [tuple(np.load(f"{out}.{r}.span.npy")) for r in range(2)]
    assert spans[0][0] == 0 and spans[0][1] == spans[1][0] and spans[1][1] == n
    for r, (r0, r1) in enumerate(spans):
        assert np.array_equal(np.load(f"{out}.{r}.npy"), want[r0:r1])


def test_row_block_partitions():
    for n in (0, 1, 33, 64, 1000):
        for world in (1, 2, 3, 8):
            spans = [shard.row_block(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    with pytest.raises(ValueError):
        shard.row_block(4, 2, 2)


def test_failed_rank_is_detected_not_hung(tmp_path):
    # rank 1 dies before the collective; rank 0's all-reduce must end with an
    # error within the process-group timeout (5 s), not hang
    import multiprocessing
    out = str(tmp_path / "c")
    ctx = multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 40, 2, 64, out, 1)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    assert procs[1].exitcode == 3
    assert os.path.exists(f"{out}.0.err") and not os.path.exists(f"{out}.0.npy")
