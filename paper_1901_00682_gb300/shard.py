"""Row-block sharding of one decomposed problem over several GPUs (one process per GPU).

Algorithm 1 couples the subdomains only through its multiplier update on the
interfaces, so each rank holds a contiguous block of tile rows (dd_tv_create_shard).
Per outer iteration a rank runs the multiplier update and the local solves of its
block (one dd_tv_iterate), then trades, with the neighbour across each cut, its copy
of p~^{n+1} on the cut side (width floats per cut); both ranks beside a cut keep equal
copies of the cut's multipliers because they update them from the same strips with the
same arithmetic.  The energy adds the ranks' parts in float64 (all-reduce) after each
rank has received the first pixel row of the rank below.

The exchange goes through a communicator object with two operations:
    exchange(shard)            after shard.send_top / send_bottom were filled, fills
                               shard.recv_above / recv_below from the neighbours
    allreduce_sum(x) -> float  float64 sum over the ranks
`TorchDistComm` implements them with torch.distributed point-to-point operations
(NCCL for CUDA tensors, gloo for CPU tensors); `LocalGroup` runs several shards in one
process (copies instead of messages).  This module only moves buffers: every
arithmetic step runs in the CUDA library.
"""
from __future__ import annotations


def split_rows(n_tile_rows: int, world: int):
    """Contiguous tile-row ranges [a0, a1) of the ranks, sizes differing by at most one."""
    if world < 1 or world > n_tile_rows:
        raise ValueError(f"{world} ranks for {n_tile_rows} tile rows: every rank needs at least one tile row")
    return [(r * n_tile_rows // world, (r + 1) * n_tile_rows // world) for r in range(world)]


class Shard:
    """One rank's block of tile rows: the shard handle (or any object with the same
    methods: iterate, shard_export, shard_import, shard_edge_rows, shard_energy) and the
    cut-side buffers.  `new_buffer(n)` makes an n-float buffer on the handle's device."""

    def __init__(self, rank: int, world: int, n_tile_rows: int, width: int, solver, new_buffer):
        self.rank, self.world = rank, world
        self.a0, self.a1 = split_rows(n_tile_rows, world)[rank]
        self.cut_top = self.a0 > 0
        self.cut_bottom = self.a1 < n_tile_rows
        self.s = solver
        buf = lambda on: new_buffer(width) if on else None
        self.send_top, self.recv_above = buf(self.cut_top), buf(self.cut_top)
        self.send_bottom, self.recv_below = buf(self.cut_bottom), buf(self.cut_bottom)
        self.first_row, self.row_below = buf(self.cut_top), buf(self.cut_bottom)

    def local_step(self):
        """The rank's part of one outer iteration and the export of its cut sides."""
        self.s.iterate(1)
        self.s.shard_export(self.send_top, self.send_bottom)

    def finish_step(self):
        self.s.shard_import(self.recv_above, self.recv_below)


class TorchDistComm:
    """Exchange over torch.distributed (one shard per rank).  stage_on_host: move the
    device buffers through host copies (for a backend without device transport, such
    as gloo; NCCL sends device memory directly)."""

    def __init__(self, dist, group=None, stage_on_host=False):
        self.dist = dist
        self.group = group
        self.stage = stage_on_host

    def exchange(self, sh: Shard, sends=None, recvs=None):
        d = self.dist
        sends = sends or ((sh.send_top, sh.rank - 1) if sh.cut_top else None,
                          (sh.send_bottom, sh.rank + 1) if sh.cut_bottom else None)
        recvs = recvs or ((sh.recv_above, sh.rank - 1) if sh.cut_top else None,
                          (sh.recv_below, sh.rank + 1) if sh.cut_bottom else None)
        ops, landing = [], []
        for t in sends:
            if t is not None:
                buf = t[0].cpu() if self.stage else t[0]
                ops.append(d.P2POp(d.isend, buf, t[1], self.group))
        for t in recvs:
            if t is not None:
                buf = t[0].new_empty(t[0].shape, device="cpu") if self.stage else t[0]
                landing.append((t[0], buf))
                ops.append(d.P2POp(d.irecv, buf, t[1], self.group))
        if ops:
            for w in d.batch_isend_irecv(ops):
                w.wait()
        if self.stage:
            for dst, buf in landing:
                dst.copy_(buf)

    def exchange_rows(self, sh: Shard):
        """Sends the first pixel row up, receives the row below (energy across a cut)."""
        self.exchange(sh, sends=((sh.first_row, sh.rank - 1) if sh.cut_top else None, None),
                      recvs=(None, (sh.row_below, sh.rank + 1) if sh.cut_bottom else None))

    def allreduce_sum(self, x: float, like=None) -> float:
        import torch
        dev = like.device if like is not None and not self.stage else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return float(t.item())


class ShardedSolver:
    """One rank of a sharded solve.  params: the whole problem (dd_tv_params of the
    full image); comm: a TorchDistComm; solver: the shard handle (created here from the
    CUDA library when None); new_buffer: buffer factory (CUDA float32 tensors when None)."""

    def __init__(self, params, rank: int, world: int, comm, solver=None, new_buffer=None, stream=None):
        if solver is None or new_buffer is None:
            import torch

            from . import _lib
            a0, a1 = split_rows(params.sub_rows, world)[rank]
            if solver is None:
                solver = _lib.Solver(params, stream, shard=(a0, a1))
            if new_buffer is None:
                new_buffer = lambda n: torch.zeros(n, dtype=torch.float32, device="cuda")
        self.params = params
        self.comm = comm
        self.sh = Shard(rank, world, params.sub_rows, params.width, solver, new_buffer)

    @property
    def solver(self):
        return self.sh.s

    def rows(self):
        """(first image row, rows) of this rank's block."""
        return self.sh.s.shard_rows()

    def load(self, f_rows, mask_rows=None):
        self.sh.s.load(f_rows, mask_rows)

    def step(self, n_outer: int = 1):
        for _ in range(n_outer):
            self.sh.local_step()
            self.comm.exchange(self.sh)
            self.sh.finish_step()

    def energy(self) -> float:
        """J(u) of the whole image (every rank gets the same value)."""
        sh = self.sh
        sh.s.shard_edge_rows(sh.first_row, None)
        self.comm.exchange_rows(sh)
        part = sh.s.shard_energy(sh.row_below)
        return self.comm.allreduce_sum(part, like=sh.send_top if sh.send_top is not None else sh.send_bottom)


class LocalGroup:
    """Several shards of one problem in one process (copies in place of messages),
    for one device: step() runs every shard's local part, then moves the cut strips."""

    def __init__(self, params, n_shards: int, stream=None, new_buffer=None, solver_factory=None):
        import torch

        from . import _lib
        if new_buffer is None:
            new_buffer = lambda n: torch.zeros(n, dtype=torch.float32, device="cuda")
        ranges = split_rows(params.sub_rows, n_shards)
        self.shards = []
        for r, (a0, a1) in enumerate(ranges):
            s = solver_factory(a0, a1) if solver_factory else _lib.Solver(params, stream, shard=(a0, a1))
            self.shards.append(Shard(r, n_shards, params.sub_rows, params.width, s, new_buffer))

    def close(self):
        for sh in self.shards:
            if hasattr(sh.s, "close"):
                sh.s.close()

    def load(self, f):
        """f: the whole image (rows x width device tensor); each shard takes its rows."""
        for sh in self.shards:
            r0, n = sh.s.shard_rows()
            sh.s.load(f[r0:r0 + n].contiguous())

    def _move(self, attr_src, attr_dst, offset):
        for k, sh in enumerate(self.shards):
            dst = getattr(sh, attr_dst)
            if dst is not None:
                dst.copy_(getattr(self.shards[k + offset], attr_src))

    def step(self, n_outer: int = 1):
        for _ in range(n_outer):
            for sh in self.shards:
                sh.local_step()
            self._move("send_bottom", "recv_above", -1)   # from the shard above
            self._move("send_top", "recv_below", +1)      # from the shard below
            for sh in self.shards:
                sh.finish_step()

    def energy(self) -> float:
        for sh in self.shards:
            sh.s.shard_edge_rows(sh.first_row, None)
        self._move("first_row", "row_below", +1)
        return sum(sh.s.shard_energy(sh.row_below) for sh in self.shards)

    def get_u(self, out):
        """Assembles u of the whole image into out (rows x width device tensor)."""
        for sh in self.shards:
            r0, n = sh.s.shard_rows()
            part = out[r0:r0 + n]
            sh.s.get_u(part)
        return out
