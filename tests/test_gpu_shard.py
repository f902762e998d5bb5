"""Row-block shards on one GPU: S shard handles of one problem, their cut strips moved
by copies between outer iterations (shard.LocalGroup), reproduce the single-handle run
bit for bit (u, and through it every later iterate), for every fused kernel that can
run a shard (4 x 4 micro-tiles, 2 x 4 micro-tiles, the cluster-barrier kernel of other
tile shapes), every fidelity and the inpainting mask; the shards' energy parts add up
to J of the whole image; and the sharded run matches the FP64 oracle at equal
iteration counts.  Several shards share the one GPU here as separate launches that do
not wait on one another (the exchange is a copy between launches)."""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_00682_gb300 import _lib as L
    L.load()
    return L


def _single_and_sharded(L, f, mask, n_outer, S, **kw):
    from paper_1901_00682_gb300.shard import LocalGroup
    H, W = f.shape
    p = L.make_params(H, W, **kw)
    fd = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    md = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).cuda()
    s = L.Solver(p)
    s.load(fd, md)
    s.iterate(n_outer)
    u1 = s.get_u(torch.empty_like(fd))
    J1 = s.current_energy()
    s.close()
    g = LocalGroup(p, S)
    if md is None:
        g.load(fd)
    else:
        for sh in g.shards:
            r0, n = sh.s.shard_rows()
            sh.s.load(fd[r0:r0 + n], md[r0:r0 + n])
    g.step(n_outer)
    uS = g.get_u(torch.empty_like(fd))
    JS = g.energy()
    g.close()
    torch.cuda.synchronize()
    return u1, J1, uS, JS


@pytest.mark.parametrize("H,W,NR,NC,S,kernel", [
    (1024, 512, 8, 4, 2, "4x4 micro-tiles"),
    (1024, 512, 8, 4, 3, "4x4 micro-tiles, uneven blocks"),
    (512, 384, 4, 3, 4, "2x4 micro-tiles (W + N_c = 387)"),
    (360, 300, 6, 3, 3, "cluster barrier, 60 x 100 tiles"),
    (300, 200, 3, 2, 3, "cluster barrier, one tile row per shard"),
])
def test_shards_reproduce_the_single_handle_run(H, W, NR, NC, S, kernel):
    L = _lib()
    f, _ = synth.rof_image(H, W, 20, 0.1, 7)
    u1, J1, uS, JS = _single_and_sharded(L, f, None, 12, S, sub_rows=NR, sub_cols=NC, fidelity="l2", alpha=8.0,
                                         inner_iters=10)
    assert torch.equal(u1, uS), kernel
    assert abs(JS - J1) <= 1e-7 * abs(J1)


@pytest.mark.parametrize("fid,mask_prob", [("l1", 0.2), ("seg", 0.0), ("l2", 0.2)])
def test_shards_every_fidelity(fid, mask_prob):
    L = _lib()
    H, W = 768, 512
    f, _ = synth.rof_image(H, W, 20, 0.1, 8)
    mask = None
    if mask_prob:
        mask = synth.bernoulli_mask((H, W), mask_prob, np.random.Generator(np.random.PCG64(3)))
        f = np.where(mask == 1, 0.0, f).astype(np.float32)
    kw = dict(sub_rows=6, sub_cols=4, fidelity=fid, alpha={"l1": 1.5, "l2": 8.0, "seg": 20.0}[fid], inner_iters=10)
    if fid == "seg":
        kw.update(c1=0.2, c2=0.8, tau=1.0)
    u1, J1, uS, JS = _single_and_sharded(L, f, mask, 9, 3, **kw)
    assert torch.equal(u1, uS)
    assert abs(JS - J1) <= 1e-7 * abs(J1)


def test_sharded_run_matches_the_oracle():
    """Two shards of a 256 x 256 image in 4 x 2 tiles of 64 x 128, 20 outer iterations,
    against the FP64 oracle's single-domain-grid run (5e-4 in u, 1e-5 in J)."""
    L = _lib()
    from paper_1901_00682_gb300.shard import LocalGroup
    f, _ = synth.rof_image(256, 256, 12, 0.05, 2)
    p = L.make_params(256, 256, 4, 2, fidelity="l2", alpha=10.0, inner_iters=10)
    g = LocalGroup(p, 2)
    fd = torch.from_numpy(f).cuda()
    g.load(fd)
    g.step(20)
    u = g.get_u(torch.empty_like(fd)).cpu().numpy().astype(np.float64)
    J = g.energy()
    g.close()
    pr = oracle.Problem(256, 256, 4, 2, fidelity="l2", alpha=10.0, inner=10)
    st = oracle.dd_run(pr, f.astype(np.float64), 20)
    assert np.abs(u - st.u).max() <= 5e-4
    Jo = oracle.energy(pr, st.u, f.astype(np.float64))
    assert abs(J - Jo) <= 1e-5 * Jo


def test_shard_refuses_whole_state_calls_and_bad_ranges():
    L = _lib()
    p = L.make_params(512, 256, 4, 2)
    s = L.Solver(p, shard=(1, 3))
    assert s.shard_rows() == (128, 256)
    with pytest.raises(L.DDTVError) as e:
        s.solve_device(torch.zeros(256, 256, device="cuda"))
    assert e.value.code == L.EUNSUPPORTED
    s.load(torch.zeros(256, 256, device="cuda"))
    with pytest.raises(L.DDTVError) as e:
        s.iterate(2)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.DDTVError) as e:
        s.shard_export(None, None)        # both sides are cut: buffers required
    assert e.value.code == L.EINVAL
    s.close()
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.dd_tv_create_shard(ctypes.byref(h), ctypes.byref(p), 2, 2) == L.EINVAL
    assert lib.dd_tv_create_shard(ctypes.byref(h), ctypes.byref(p), 0, 5) == L.EINVAL
    q = L.make_params(502, 256, 4, 2)      # tile rows of unequal height
    assert lib.dd_tv_create_shard(ctypes.byref(h), ctypes.byref(q), 0, 2) == L.EINVAL
    q = L.make_params(512, 256, 4, 2, path="plain")
    assert lib.dd_tv_create_shard(ctypes.byref(h), ctypes.byref(q), 0, 2) == L.EUNSUPPORTED


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_worker(rank, world, port, H, W, NR, NC, n_outer, out):
    """One process per shard, all on cuda:0, exchanging through gloo with host staging
    (their kernels never wait on one another: every exchange happens between launches)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import synth as sy
    from paper_1901_00682_gb300 import _lib as L
    from paper_1901_00682_gb300.shard import ShardedSolver, TorchDistComm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        p = L.make_params(H, W, NR, NC, fidelity="l2", alpha=8.0, inner_iters=10)
        ss = ShardedSolver(p, rank, world, TorchDistComm(dist, stage_on_host=True))
        f, _ = sy.rof_image(H, W, 20, 0.1, 9)
        r0, n = ss.rows()
        ss.load(torch.from_numpy(np.ascontiguousarray(f[r0:r0 + n])).cuda())
        ss.step(n_outer)
        J = ss.energy()
        u = torch.empty(n, W, device="cuda")
        ss.solver.get_u(u)
        torch.cuda.synchronize()
        out[rank] = (r0, u.cpu().numpy().tobytes(), J)
        ss.solver.close()
    finally:
        dist.destroy_process_group()


def test_sharded_solver_over_torch_distributed_ranks():
    """The distributed path end to end (ShardedSolver + TorchDistComm, one process per
    shard): three ranks reproduce the single-handle run bit for bit."""
    L = _lib()
    import torch.multiprocessing as mp
    H, W, NR, NC, world, n_outer = 768, 512, 6, 4, 3, 8
    f, _ = synth.rof_image(H, W, 20, 0.1, 9)
    p = L.make_params(H, W, NR, NC, fidelity="l2", alpha=8.0, inner_iters=10)
    fd = torch.from_numpy(f).cuda()
    with L.Solver(p) as s:
        s.load(fd)
        s.iterate(n_outer)
        u1 = s.get_u(torch.empty_like(fd)).cpu().numpy()
        J1 = s.current_energy()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_worker, args=(world, _free_port(), H, W, NR, NC, n_outer, out), nprocs=world, join=True)
    for r in range(world):
        r0, ub, J = out[r]
        u = np.frombuffer(ub, dtype=np.float32).reshape(-1, W)
        assert np.array_equal(u, u1[r0:r0 + u.shape[0]]), r
        assert abs(J - J1) <= 1e-7 * abs(J1)
