"""Adaptive inner stopping (Section 5, eq. stop_inner1) on the GPU fused path.

Where floating point decides an integer (the inner count of every local solve), the
float32 GPU trajectory and the float64 oracle may legitimately stop one subdomain at
different iterations.  So the test takes the counts the GPU reports, forces the oracle
to run exactly those counts, and checks
  * parity of the iterates at equal counts (max |du| <= 5e-4, relative energy <= 1e-5);
  * that every GPU decision is valid for the float64 trajectory: the relative change of
    p at the GPU's last iteration is below 1.5 tol (unless the cap was reached), and at
    every earlier iteration above tol / 1.5.
Tilings of exact 128 x 128 subdomains with W + N_c a multiple of 4 run the default 4 x 4
micro-tile kernel (the decision on iteration k is taken during the u-step of k + 1, which
is undone when the solve stops); every other tiling, and the other variants, run the
cluster-barrier kernel.  Both sum the residuals in a different order; the counts and the
iterates of the two kernels are compared for equality.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _run_gpu(f, NR, NC, n_outer, tol, K, fid="l2", alpha=10.0, mask=None, **kw):
    from paper_1901_00682_gb300 import _lib as L
    H, W = f.shape
    p = L.make_params(H, W, NR, NC, fidelity=fid, alpha=alpha, inner_iters=K, inner_tol=tol, **kw)
    counts = []
    with L.Solver(p) as s:
        fd = torch.from_numpy(f).cuda()
        s.load(fd, None if mask is None else torch.from_numpy(mask).cuda())
        for _ in range(n_outer):
            s.iterate(1)
            c, mx = s.inner_counts()
            assert mx == c.max()
            counts.append(c.ravel().copy())
        u = torch.empty_like(fd)
        s.get_u(u)
        torch.cuda.synchronize()
        J = s.current_energy()
        return u.cpu().numpy().astype(np.float64), np.array(counts), J


def _mask_for(shape, prob, seed=5):
    return synth.bernoulli_mask(shape, prob, np.random.Generator(np.random.PCG64(seed))) if prob else None


@pytest.mark.parametrize("shape,grid,fid,alpha,tol,mask_prob", [
    ((128, 128), (2, 2), "l2", 10.0, 1e-3, 0.0),
    ((100, 90), (3, 2), "l2", 10.0, 3e-3, 0.0),      # ragged tiles, one CTA per tile
    ((256, 256), (2, 2), "l2", 8.0, 1e-3, 0.0),      # 128 x 128 tiles, W + N_c = 258: cluster-barrier kernel
    ((96, 96), (2, 2), "seg", 20.0, 1e-3, 0.0),
    ((512, 512), (4, 4), "l2", 8.0, 1e-3, 0.0),      # 4 x 4 micro-tile kernel
    ((256, 512), (2, 4), "l1", 1.5, 3e-3, 0.2),      # ... TV-L1 inpainting
    ((256, 512), (2, 4), "seg", 20.0, 1e-3, 0.0),    # ... segmentation
])
def test_adaptive_inner_stop_parity(cuda_lib, shape, grid, fid, alpha, tol, mask_prob):
    H, W = shape
    f, _ = synth.rof_image(H, W, 8, 0.05, 21)
    mask = _mask_for(shape, mask_prob)
    if mask is not None:
        f = np.where(mask == 1, 0.0, f).astype(np.float32)
    K, N = 60, 8
    extra = dict(c1=0.2, c2=0.8) if fid == "seg" else {}
    u, counts, J = _run_gpu(f, *grid, N, tol, K, fid=fid, alpha=alpha, mask=mask, **extra)
    assert counts.min() >= 1 and counts.max() <= K
    assert counts.min() < K                                   # the rule stopped some solves
    pr = oracle.Problem(H, W, *grid, fidelity=fid, alpha=alpha, inner=K, **(dict(tau=1.0, **extra) if fid == "seg" else {}))
    st = oracle.dd_run(pr, f, N, counts=counts, record=True, mask=mask)
    assert np.abs(u - st.u).max() <= 5e-4
    Jo = oracle.energy(pr, st.u, f, mask=mask)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    res = st.inner_res
    for n in range(N):
        for t in range(counts.shape[1]):
            c = counts[n, t]
            r = res[n, t, :c]
            assert np.all(r[:-1] >= tol / 1.5), (n, t, c, r)
            if c < K:
                assert r[-1] < tol * 1.5, (n, t, c, r)


def test_fixed_count_reports_and_stats(cuda_lib):
    from paper_1901_00682_gb300 import _lib as L
    f, _ = synth.rof_image(64, 64, 6, 0.05, 3)
    fd = torch.from_numpy(f).cuda()
    with L.Solver(L.make_params(64, 64, 2, 2, inner_iters=7, outer_iters=3)) as s:
        c, mx = s.inner_counts()
        assert np.all(c == 0) and mx == 0
        _, st, _ = s.solve_device(fd)
        torch.cuda.synchronize()
        assert st.inner_max == 7 and st.pixel_iters == 64 * 64 * 7 * 3
        c, mx = s.inner_counts()
        assert np.all(c == 7) and mx == 7


def test_adaptive_stats_count_the_work(cuda_lib):
    """stats.pixel_iters of an adaptive solve = sum over outer iterations and tiles of
    tile pixels x inner count; stats.inner_max = the largest count."""
    from paper_1901_00682_gb300 import _lib as L
    H, W, N, K = 96, 80, 6, 40
    f, _ = synth.rof_image(H, W, 6, 0.05, 8)
    u, counts, _ = _run_gpu(f, 2, 2, N, 2e-3, K)
    px = np.array([(oracle.part_start(a + 1, H, 2) - oracle.part_start(a, H, 2)) *
                   (oracle.part_start(b + 1, W, 2) - oracle.part_start(b, W, 2)) for a in range(2) for b in range(2)])
    with L.Solver(L.make_params(H, W, 2, 2, inner_iters=K, inner_tol=2e-3, outer_iters=N)) as s:
        u2, st, _ = s.solve_device(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
    assert np.array_equal(u2.cpu().numpy().astype(np.float64), u)
    assert st.pixel_iters == int((counts * px).sum())
    assert st.inner_max == counts.max()


def test_adaptive_needs_fused_path(cuda_lib):
    from paper_1901_00682_gb300 import _lib as L
    for path in ("plain", "fulldim"):
        with pytest.raises(L.DDTVError) as e:
            L.Solver(L.make_params(64, 64, 2, 2, path=path, inner_tol=1e-3))
        assert e.value.code == L.EUNSUPPORTED
    with L.Solver(L.make_params(64, 64, 2, 2, inner_tol=1e-3)) as s:
        f = torch.zeros(64, 64, device="cuda")
        with pytest.raises(L.DDTVError) as e:
            s.adjoint_forward(f, None, 2, 1, torch.empty_like(f))
        assert e.value.code == L.EUNSUPPORTED


@pytest.mark.parametrize("fid,alpha,tol,mask_prob,K", [
    ("l2", 8.0, 1e-3, 0.0, 60),
    ("l2", 8.0, 1e-2, 0.0, 20),
    ("l1", 1.5, 3e-3, 0.2, 40),
    ("l2", 8.0, 3e-3, 0.2, 40),
    ("seg", 20.0, 1e-3, 0.0, 40),
])
def test_adaptive_counts_equal_across_kernels(cuda_lib, fid, alpha, tol, mask_prob, K):
    """The 4 x 4 micro-tile kernel (variant 0) and the cluster-barrier kernel (variant 3)
    compute bit-identical iterates and sum the residuals of eq. stop_inner1 in different
    orders (float32 trees in the first, float64 across warps in the second): they take
    the same decision for every local solve, so the counts and u agree exactly."""
    H, W, NR, NC, N = 512, 512, 4, 4, 10
    f, _ = synth.rof_image(H, W, 12, 0.05, 31)
    mask = _mask_for((H, W), mask_prob, 6)
    if mask is not None:
        f = np.where(mask == 1, 0.0, f).astype(np.float32)
    extra = dict(c1=0.2, c2=0.8, tau=1.0) if fid == "seg" else {}
    u0, c0, J0 = _run_gpu(f, NR, NC, N, tol, K, fid=fid, alpha=alpha, mask=mask, variant=0, **extra)
    u3, c3, J3 = _run_gpu(f, NR, NC, N, tol, K, fid=fid, alpha=alpha, mask=mask, variant=3, **extra)
    assert c0.min() < K and c0.max() > 1                      # the rule acts, and not only at k = 1
    assert np.array_equal(c0, c3)
    assert np.array_equal(u0, u3)
    assert J0 == J3


def test_adaptive_micro_tile_zero_image_stops_after_one_iteration(cuda_lib):
    """f = 0 keeps u = 0 and p = 0 exactly (sum p^2 = 0): every local solve stops after
    its first inner iteration (the decision on it is taken in the second one, whose
    u-step is undone).  (A constant image other than 0 does not: the prox of the u-step
    moves u by an ulp, and the relative change of the resulting p ~ 1e-8 stays large, so
    those solves run to the cap, in either kernel.)"""
    f = np.zeros((512, 512), dtype=np.float32)
    u, counts, J = _run_gpu(f, 4, 4, 3, 1e-3, 20)
    assert np.all(counts == 1)
    assert np.all(u == 0.0) and J == 0.0


def test_adaptive_micro_tile_matches_fixed_count_when_tol_is_tiny(cuda_lib):
    """With a tolerance no float32 iterate reaches, every solve runs to the cap and the
    adaptive kernel reproduces the fixed-count kernel bit for bit (the reduction and the
    undo machinery leave the iterates untouched)."""
    from paper_1901_00682_gb300 import _lib as L
    f, _ = synth.rof_image(512, 512, 10, 0.05, 4)
    u_a, counts, _ = _run_gpu(f, 4, 4, 5, 1e-12, 12)
    assert np.all(counts == 12)
    with L.Solver(L.make_params(512, 512, 4, 4, inner_iters=12, alpha=10.0)) as s:
        fd = torch.from_numpy(f).cuda()
        s.load(fd)
        s.iterate(5)
        u_f = s.get_u(torch.empty_like(fd)).cpu().numpy().astype(np.float64)
    assert np.array_equal(u_a, u_f)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_adaptive_micro_tile_small_caps(cuda_lib, K):
    """Caps of 1 to 3 inner iterations in the micro-tile kernel: with K = 1 no decision is
    taken (every count is 1); with K = 2, 3 the decision on iteration k is taken in
    iteration k + 1 and the counts stay in [1, K]; the iterates match the oracle run at
    the same counts."""
    H, W, N, tol = 512, 512, 6, 2e-2
    f, _ = synth.rof_image(H, W, 12, 0.05, 41)
    u, counts, J = _run_gpu(f, 4, 4, N, tol, K, alpha=8.0)
    assert counts.min() >= 1 and counts.max() <= K
    if K == 1:
        assert np.all(counts == 1)
    pr = oracle.Problem(H, W, 4, 4, fidelity="l2", alpha=8.0, inner=K)
    st = oracle.dd_run(pr, f, N, counts=counts)
    assert np.abs(u - st.u).max() <= 5e-4
    Jo = oracle.energy(pr, st.u, f)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
