"""Host logic of the row-block sharding (paper_1901_00682_gb300/shard.py) on CPU with
world-size 2 and 3 `gloo` ranks.

The shard handle is replaced by a stand-in whose exports encode (rank, outer
iteration, side) and which checks, on every import, that it received exactly its
neighbours' exports of the same outer iteration: the routing (who sends which strip to
whom), its timing (after the rank's own iteration, before the next) and the energy
reduction (each rank's part uses the first row of the rank below, the parts add up)
are checked without a GPU.  The numerics of the sharded solve are checked on the GPU
(tests/test_gpu_shard.py: S shards reproduce the single-handle run bit for bit)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W = 24


def _code(rank, n, side):
    return torch.arange(W, dtype=torch.float32) + 1000.0 * rank + 10.0 * n + {"top": 1, "bottom": 2, "row": 3}[side]


class FakeShardSolver:
    def __init__(self, rank):
        self.rank, self.n, self.imports = rank, 0, 0

    def iterate(self, k):
        assert k == 1
        self.n += 1

    def shard_export(self, top, bottom):
        if top is not None:
            top.copy_(_code(self.rank, self.n, "top"))
        if bottom is not None:
            bottom.copy_(_code(self.rank, self.n, "bottom"))

    def shard_import(self, above, below):
        if above is not None:
            assert torch.equal(above, _code(self.rank - 1, self.n, "bottom"))
            self.imports += 1
        if below is not None:
            assert torch.equal(below, _code(self.rank + 1, self.n, "top"))
            self.imports += 1

    def shard_edge_rows(self, first, last):
        if first is not None:
            first.copy_(_code(self.rank, self.n, "row"))

    def shard_energy(self, row_below):
        if row_below is not None:
            assert torch.equal(row_below, _code(self.rank + 1, self.n, "row"))
        return 10.0 * (self.rank + 1) + self.n


class _Params:
    def __init__(self, sub_rows, width):
        self.sub_rows, self.width = sub_rows, width


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_tile_rows, steps, out):
    sys.path.insert(0, ROOT)
    from paper_1901_00682_gb300.shard import ShardedSolver, TorchDistComm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        fake = FakeShardSolver(rank)
        s = ShardedSolver(_Params(n_tile_rows, W), rank, world, TorchDistComm(dist), solver=fake,
                          new_buffer=lambda n: torch.zeros(n, dtype=torch.float32))
        s.step(steps)
        J = s.energy()
        out[rank] = (fake.n, fake.imports, J, s.sh.a0, s.sh.a1)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_tile_rows", [(2, 4), (3, 8)])
def test_sharded_exchange_routing_gloo(world, n_tile_rows):
    steps = 5
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), n_tile_rows, steps, out), nprocs=world, join=True)
    want_J = sum(10.0 * (r + 1) + steps for r in range(world))
    rows = []
    for r in range(world):
        n, imports, J, a0, a1 = out[r]
        assert n == steps
        cuts = (r > 0) + (r < world - 1)
        assert imports == steps * cuts
        assert J == want_J
        rows.append((a0, a1))
    assert rows[0][0] == 0 and rows[-1][1] == n_tile_rows
    assert all(rows[k][1] == rows[k + 1][0] for k in range(world - 1))


def test_split_rows():
    sys.path.insert(0, ROOT)
    from paper_1901_00682_gb300.shard import split_rows
    assert split_rows(32, 1) == [(0, 32)]
    assert split_rows(32, 4) == [(0, 8), (8, 16), (16, 24), (24, 32)]
    assert split_rows(8, 3) == [(0, 2), (2, 5), (5, 8)]
    with pytest.raises(ValueError):
        split_rows(2, 3)
