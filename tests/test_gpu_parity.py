"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs, at equal iteration counts.  Bar (stated per result):
  max |u_gpu - u_oracle| <= 5e-4 on [0, 1]-range images, relative energy error <= 1e-5,
the dual field and the multipliers within their float32 error growth (p_tol, lam_tol),
and bit-exact agreement between the fused and the plain GPU paths (they share the
pointwise arithmetic).  Covers several tiles with ragged tails, every fidelity, the
inpainting mask, the 1 x 1 grid, the full-dimension comparator, state export/import
and, at the 4096^2 / 32 x 32 workload in the benchmark's launch configuration, a
few outer iterations compared element by element.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 5e-4
E_TOL = 1e-5
U32 = 2.0 ** -24  # unit roundoff of float32


def p_tol(n_steps):
    """Tolerance of the dual field after n_steps inner iterations in all.  |p| <= 1, each
    update of a dof rounds through at most 4 float32 operations, and the primal-dual
    iteration carries earlier deviations forward without amplifying them, so the
    distance to the float64 trajectory grows at most linearly: 4 u n_steps.  (Measured on
    these cases: 0.1 u to 0.5 u per inner iteration.)"""
    return 4.0 * U32 * n_steps


def lam_tol(n_outer, inner, sigma, lam_max):
    """Tolerance of the multipliers after n_outer outer iterations.  Each update adds
    sigma times the jump of 2 p~^{n+1} - p~^n across an interface (three dual values on
    each of two sides): the dual deviations contribute at most 6 sigma n_outer p_tol, and
    the update's own rounding 4 u max(1, |lambda|) per outer iteration."""
    return 6.0 * sigma * n_outer * p_tol(n_outer * inner) + 4.0 * U32 * n_outer * max(1.0, lam_max)


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_00682_gb300 import _lib
    _lib.load()
    return _lib


def _run_gpu(f, mask, n_outer, path="fused", **kw):
    L = _gpu()
    H, W = f.shape
    p = L.make_params(H, W, path=path, outer_iters=n_outer, **kw)
    s = L.Solver(p)
    fd = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    md = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).cuda()
    s.load(fd, md)
    s.iterate(n_outer)
    st = s.get_state()
    torch.cuda.synchronize()
    return s, {k: v.cpu().numpy().astype(np.float64) for k, v in st.items()}, fd, md


def _run_oracle(f, mask, n_outer, sub_rows=1, sub_cols=1, fidelity="l2", alpha=10.0, c1=0.0, c2=0.0,
                inner_iters=10, tau=None, **_):
    H, W = f.shape
    tau = tau if tau is not None else (1.0 if fidelity == "seg" else 50.0)
    pr = oracle.Problem(H, W, sub_rows, sub_cols, fidelity=fidelity, alpha=alpha, c1=c1, c2=c2, tau=tau,
                        inner=inner_iters)
    st = oracle.dd_run(pr, f.astype(np.float64), n_outer, mask=mask)
    return pr, st


def _check(f, mask, n_outer, **kw):
    s, g, fd, md = _run_gpu(f, mask, n_outer, **kw)
    pr, o = _run_oracle(f, mask, n_outer, **kw)
    du = np.abs(g["u"] - o.u).max()
    assert du <= U_TOL, f"max|du| = {du}"
    Jg = oracle.energy(pr, g["u"], f.astype(np.float64), mask)
    Jo = oracle.energy(pr, o.u, f.astype(np.float64), mask)
    assert abs(Jg - Jo) <= E_TOL * abs(Jo), (Jg, Jo)
    # the dual field and the multipliers follow the same trajectory, within the float32
    # error growth of p_tol / lam_tol
    K = kw.get("inner_iters", 10)
    tau = kw.get("tau") or (1.0 if kw.get("fidelity") == "seg" else 50.0)
    sigma = kw.get("sigma") or 0.5 / tau
    tp = p_tol(n_outer * K)
    assert np.abs(g["P1"] - o.P1).max() <= tp and np.abs(g["P2"] - o.P2).max() <= tp
    for k in ("lamh", "lamv"):
        ref = getattr(o, k)
        if ref.size:
            assert np.abs(g[k] - ref).max() <= lam_tol(n_outer, K, sigma, np.abs(ref).max()), k
    return s, g, o, du


def test_rof128_parity():
    """ROF 128x128, 2x2 subdomains of 64x64, 200 outer x 10 inner."""
    f, _ = synth.rof_image(128, 128, 12, 0.05, 0)
    _check(f, None, 200, sub_rows=2, sub_cols=2, fidelity="l2", alpha=10.0, inner_iters=10)


@pytest.mark.parametrize("H,W,NR,NC", [(67, 45, 3, 2), (96, 200, 2, 3), (33, 31, 1, 1), (130, 130, 2, 2),
                                       (40, 64, 5, 1), (16, 256, 1, 2)])
def test_ragged_tiles_parity(H, W, NR, NC):
    f, _ = synth.rof_image(H, W, 6, 0.05, 1)
    _check(f, None, 30, sub_rows=NR, sub_cols=NC, fidelity="l2", alpha=10.0, inner_iters=7)


@pytest.mark.parametrize("H,W,NR,NC", [(1, 1, 1, 1), (1, 2, 1, 2), (2, 1, 2, 1), (8, 8, 8, 8), (5, 7, 5, 7),
                                       (1, 64, 1, 4), (64, 1, 4, 1)])
def test_degenerate_geometries_parity(H, W, NR, NC):
    """The method's degenerate cases: a single pixel (no dual dofs at all), single rows
    and columns, and one-pixel subdomains (every dof of a subdomain is an interface
    dof; the 1 x 2 image split into two pixels is the smallest decomposition).  Fused
    and plain paths against the oracle, and against each other bit for bit."""
    f = np.random.Generator(np.random.PCG64(1000 * H + W)).random((H, W)).astype(np.float32)
    kw = dict(sub_rows=NR, sub_cols=NC, fidelity="l2", alpha=10.0, inner_iters=5)
    n = 40
    _, g, _, _ = _run_gpu(f, None, n, **kw)
    _, gp, _, _ = _run_gpu(f, None, n, path="plain", **kw)
    pr, o = _run_oracle(f, None, n, **kw)
    assert np.abs(g["u"] - o.u).max() <= U_TOL
    Jg = oracle.energy(pr, g["u"], f.astype(np.float64), None)
    Jo = oracle.energy(pr, o.u, f.astype(np.float64), None)
    assert abs(Jg - Jo) <= E_TOL * max(abs(Jo), 1.0), (Jg, Jo)   # J* = 0 for a single pixel
    for k in ("u", "P1", "P2", "lamh", "lamv"):
        assert np.array_equal(g[k], gp[k]), k


def test_tvl1_inpainting_parity():
    f, mask, _ = synth.tvl1_inpaint_image(160, 96, 10, 0.1, 0.2, 2)
    _check(f, mask, 60, sub_rows=3, sub_cols=2, fidelity="l1", alpha=1.5, inner_iters=10)


def test_l2_inpainting_parity():
    f, _ = synth.rof_image(96, 96, 8, 0.05, 3)
    mask = synth.bernoulli_mask(f.shape, 0.2, np.random.Generator(np.random.PCG64(5)))
    f = f.copy()
    f[mask == 1] = 0.0
    _check(f, mask, 60, sub_rows=2, sub_cols=2, fidelity="l2", alpha=10.0, inner_iters=10)


def test_segmentation_parity():
    f, _ = synth.seg_image(128, 64, 10, 0.05, 4)
    _check(f, None, 80, sub_rows=2, sub_cols=1, fidelity="seg", alpha=20.0, c1=0.2, c2=0.8, inner_iters=10)


def test_tile_128_parity_with_interfaces():
    # the 128x128-tile configuration (cluster of CTAs per subdomain) with all four sides active
    f, _ = synth.rof_image(384, 384, 30, 0.1, 6)
    _check(f, None, 12, sub_rows=3, sub_cols=3, fidelity="l2", alpha=8.0, inner_iters=10)


def test_fused_equals_plain_bitwise():
    f, mask, _ = synth.tvl1_inpaint_image(96, 80, 8, 0.1, 0.2, 7)
    kw = dict(sub_rows=3, sub_cols=2, fidelity="l1", alpha=1.5, inner_iters=9)
    _, a, _, _ = _run_gpu(f, mask, 17, path="fused", **kw)
    _, b, _, _ = _run_gpu(f, mask, 17, path="plain", **kw)
    for k in ("u", "P1", "P2", "lamh", "lamv"):
        assert np.array_equal(a[k], b[k]), k


def test_fulldim_parity():
    f, _ = synth.rof_image(64, 96, 8, 0.05, 8)
    s, g, _, _ = _run_gpu(f, None, 30, path="fulldim", fidelity="l2", alpha=10.0, inner_iters=10)
    pr = oracle.Problem(64, 96, fidelity="l2", alpha=10.0)
    cp = oracle.cp_run(pr, f.astype(np.float64), 300)
    assert np.abs(g["u"] - cp.u).max() <= U_TOL
    assert np.abs(g["P1"] - cp.p1).max() <= p_tol(300)


def test_energy_and_gap_kernels():
    L = _gpu()
    f, _ = synth.rof_image(257, 131, 10, 0.05, 9)
    rng = np.random.default_rng(0)
    u = (f + 0.01 * rng.standard_normal(f.shape)).astype(np.float32)
    mask = (rng.uniform(size=f.shape) < 0.2).astype(np.uint8)
    for fid, m in (("l2", None), ("l2", mask), ("l1", mask), ("seg", None)):
        p = L.make_params(257, 131, 3, 2, fidelity=fid, alpha=7.0, c1=0.2, c2=0.8)
        s = L.Solver(p)
        ud = torch.from_numpy(np.clip(u, 0, 1) if fid == "seg" else u).cuda()
        J = s.energy(ud, torch.from_numpy(f).cuda(), None if m is None else torch.from_numpy(m).cuda())
        pr = oracle.Problem(257, 131, 3, 2, fidelity=fid, alpha=7.0, c1=0.2, c2=0.8)
        Jo = oracle.energy(pr, ud.cpu().numpy().astype(np.float64), f.astype(np.float64), m)
        assert abs(J - Jo) <= 1e-6 * abs(Jo), (fid, J, Jo)
    # duality gap of a DD iterate: same J and dual value as the oracle on the same state
    s, g, _, _ = _run_gpu(f, None, 40, sub_rows=3, sub_cols=3, fidelity="l2", alpha=7.0)
    J, D = s.gap()
    pr = oracle.Problem(257, 131, 3, 3, alpha=7.0)
    p1, p2 = oracle.torn_to_global(pr, g["P1"], g["P2"])
    Do = oracle.dual_value(pr, p1, p2, f.astype(np.float64))
    Jo = oracle.energy(pr, g["u"], f.astype(np.float64))
    assert abs(J - Jo) <= 1e-6 * Jo and abs(D - Do) <= 1e-6 * abs(Do)
    assert D <= J


def test_state_roundtrip_resume_is_bit_identical():
    L = _gpu()
    f, _ = synth.rof_image(96, 64, 8, 0.05, 10)
    kw = dict(sub_rows=3, sub_cols=2, fidelity="l2", alpha=10.0)
    s, a, _, _ = _run_gpu(f, None, 23, **kw)
    s2, b, fd, _ = _run_gpu(f, None, 11, **kw)
    st = s2.get_state()
    s3 = L.Solver(L.make_params(96, 64, **kw))
    s3.load(fd)
    s3.set_state(st, 11)
    s3.iterate(12)
    c = {k: v.cpu().numpy().astype(np.float64) for k, v in s3.get_state().items()}
    for k in ("u", "P1", "P2", "lamh", "lamv"):
        assert np.array_equal(a[k], c[k]), k


def test_host_solve_matches_device_path():
    L = _gpu()
    f, _ = synth.rof_image(128, 128, 12, 0.05, 0)
    p = L.make_params(128, 128, 2, 2, outer_iters=37)
    s = L.Solver(p)
    u_host, stats, rc = s.solve_host(f)
    assert rc == L.OK and stats.outer_done == 37 and stats.pixel_iters == 128 * 128 * 10 * 37
    _, g, _, _ = _run_gpu(f, None, 37, sub_rows=2, sub_cols=2)
    assert np.array_equal(u_host.astype(np.float64), g["u"])


def test_outer_tolerance_stops():
    L = _gpu()
    f, _ = synth.rof_image(64, 64, 6, 0.05, 11)
    pr = oracle.Problem(64, 64, alpha=10.0)
    Jstar = oracle.energy(pr, oracle.cp_run(pr, f.astype(np.float64), 20000).u, f.astype(np.float64))
    p = L.make_params(64, 64, 2, 2, outer_iters=2000, outer_tol=1e-4, energy_ref=Jstar, energy_every=5)
    s = L.Solver(p)
    u, stats, rc = s.solve_host(f)
    assert rc == L.OK and stats.converged == 1
    assert stats.rel_err <= 1e-4 and stats.outer_done % 5 == 0 and stats.outer_done < 2000
    # one check earlier had not converged
    p2 = L.make_params(64, 64, 2, 2, outer_iters=stats.outer_done - 5)
    u2, _, _ = L.Solver(p2).solve_host(f)
    J2 = oracle.energy(pr, u2.astype(np.float64), f.astype(np.float64))
    assert (J2 - Jstar) / Jstar > 1e-4


def test_errors_are_reported_not_raised_on_device():
    L = _gpu()
    s = L.Solver(L.make_params(32, 32, 2, 2))
    with pytest.raises(L.DDTVError) as e:
        s.iterate(1)   # nothing loaded
    assert e.value.code == L.EINVAL
    with pytest.raises(L.DDTVError):
        L.Solver(L.make_params(32, 32, 2, 2, fidelity="seg")).load(torch.zeros(32, 32, device="cuda"),
                                                                  torch.zeros(32, 32, dtype=torch.uint8,
                                                                              device="cuda"))
    # tiles larger than the fused kernel supports are refused up front
    with pytest.raises(L.DDTVError) as e:
        L.Solver(L.make_params(512, 512, 1, 1))
    assert e.value.code == L.EUNSUPPORTED


@pytest.mark.slow
def test_full_size_4096_sampled_parity():
    """4096^2, 32x32 subdomains of 128^2, inner 10, the benchmark's launch
    configuration: 2 outer iterations, every pixel compared with the oracle."""
    f, _ = synth.rof_image(4096, 4096, 400, 0.1, 0)
    kw = dict(sub_rows=32, sub_cols=32, fidelity="l2", alpha=8.0, inner_iters=10)
    _, g, _, _ = _run_gpu(f, None, 2, **kw)
    _, o = _run_oracle(f, None, 2, **kw)
    assert np.abs(g["u"] - o.u).max() <= U_TOL
    assert np.abs(g["P1"] - o.P1).max() <= p_tol(20) and np.abs(g["P2"] - o.P2).max() <= p_tol(20)
    assert np.abs(g["lamh"] - o.lamh).max() <= lam_tol(2, 10, 0.01, np.abs(o.lamh).max())


@pytest.mark.slow
@pytest.mark.parametrize("side", [46080, 46336])
def test_maximum_size_sampled_subdomains(side):
    """The largest square images the interface accepts with 128 x 128 subdomains (about
    2^31 pixels).  At 46080^2 (360 x 360 subdomains, W + N_c a multiple of 4) the
    default tensor-copy kernel runs; at 46336^2 the 2 x 4 micro-tile kernel runs and the
    torn arrays P1, P2 hold more than 2^31 values.  After 2 outer iterations, sampled
    subdomains (the four corners and an interior one) are compared element by element
    with the oracle run on the subdomain and the two rings of subdomains around it: after
    n outer iterations a subdomain depends on the subdomains fewer than n steps away, and
    their local problems on which of their own neighbours exist, so a radius-n block of
    subdomains reproduces its trajectory exactly."""
    L = _gpu()
    base = torch.from_numpy(synth.rof_image(4096, 4096, 400, 0.1, 0)[0]).cuda()
    reps = -(-side // 4096)
    big = base.repeat(reps, reps)
    fd = big[:side, :side].contiguous()
    del big, base
    NT, n_outer = side // 128, 2
    kw = dict(fidelity="l2", alpha=8.0, inner_iters=10)
    with L.Solver(L.make_params(side, side, NT, NT, outer_iters=n_outer, **kw)) as s:
        s.load(fd, None)
        s.iterate(n_outer)
        st = s.get_state()
        torch.cuda.synchronize()
    for a, b in [(0, 0), (0, NT - 1), (NT - 1, 0), (NT - 1, NT - 1), (NT // 2, NT // 3)]:
        r0, r1, c0, c1 = max(0, a - n_outer), min(NT, a + n_outer + 1), max(0, b - n_outer), min(NT, b + n_outer + 1)
        fs = fd[r0 * 128:r1 * 128, c0 * 128:c1 * 128].cpu().numpy()
        _, o = _run_oracle(fs, None, n_outer, sub_rows=r1 - r0, sub_cols=c1 - c0, **kw)
        ug = st["u"][a * 128:(a + 1) * 128, b * 128:(b + 1) * 128].cpu().numpy().astype(np.float64)
        uo = o.u[(a - r0) * 128:(a - r0 + 1) * 128, (b - c0) * 128:(b - c0 + 1) * 128]
        assert np.abs(ug - uo).max() <= U_TOL, (a, b)
        # the subdomain's p1 dofs: rows a*129 .. a*129 + 128 of the torn layout
        pg = st["P1"][a * 129:(a + 1) * 129, b * 128:(b + 1) * 128].cpu().numpy().astype(np.float64)
        po = o.P1[(a - r0) * 129:(a - r0 + 1) * 129, (b - c0) * 128:(b - c0 + 1) * 128]
        assert np.abs(pg - po).max() <= p_tol(n_outer * 10), (a, b)
    del st, fd
    torch.cuda.empty_cache()


N_VARIANTS = 4  # hardware mappings of a 128 x 128 subdomain (dd_tv_params.variant)


def test_variant_count():
    L = _gpu()
    with L.Solver(L.make_params(256, 256, 2, 2, variant=N_VARIANTS - 1)):
        pass
    with pytest.raises(L.DDTVError) as e:
        L.Solver(L.make_params(256, 256, 2, 2, variant=N_VARIANTS))
    assert e.value.code == L.EINVAL


@pytest.mark.parametrize("fid,mask_prob,K", [("l2", 0.2, 10), ("l1", 0.2, 10), ("seg", 0.0, 10), ("l2", 0.0, 70)])
def test_persistent_variants_bitwise_all_fidelities(fid, mask_prob, K):
    """The default 4 x 4 micro-tile mapping (tensor copies) against the cp.async 4 x 4
    (1), 2 x 4 micro-tile (2) and cluster-barrier (3) mappings for every fidelity, with
    and without the inpainting mask, and with more inner iterations than the 4 x 4
    kernel keeps coefficient sets in shared memory (K = 70 > 64: variants 0 and 1 then
    run the 2 x 4 kernel, which reads the sets past 64 from global memory)."""
    L = _gpu()
    H, W = 384, 512  # 3 x 4 tiles: W + N_c = 516 keeps the p2 rows 16-byte aligned (variants 0, 1)
    f, _ = synth.rof_image(H, W, 12, 0.1, 5)
    mask = None
    if mask_prob:
        mask = synth.bernoulli_mask((H, W), mask_prob, np.random.Generator(np.random.PCG64(9)))
        f = np.where(mask == 1, 0.0, f).astype(np.float32)
    kw = dict(sub_rows=3, sub_cols=4, fidelity=fid, alpha={"l2": 8.0, "l1": 1.5, "seg": 20.0}[fid],
              inner_iters=K)
    if fid == "seg":
        kw.update(c1=0.2, c2=0.8, tau=1.0)
    outs = [_run_gpu(f, mask, 5, variant=v, **kw)[1] for v in range(N_VARIANTS)]
    for o in outs[1:]:
        for k in ("u", "P1", "P2", "lamh", "lamv"):
            assert np.array_equal(outs[0][k], o[k]), k


@pytest.mark.parametrize("H,W,NR,NC", [(384, 384, 3, 3), (250, 260, 2, 3), (128, 128, 1, 1), (1024, 1280, 8, 10),
                                        (512, 512, 4, 4), (1024, 1024, 8, 8)])
def test_fused_variants_bitwise_identical(H, W, NR, NC):
    """Every hardware mapping of a 128x128-class subdomain runs the same arithmetic.
    W + N_c a multiple of 4 (512 / 4 x 4, 1024 / 8 x 8) runs the mappings that copy p2
    rows in 16-byte chunks; the other exact grids run the 2 x 4 mapping in their place,
    and ragged grids the cluster-barrier kernel."""
    L = _gpu()
    f, _ = synth.rof_image(H, W, 12, 0.1, 12)
    outs = []
    for v in range(N_VARIANTS):
        _, g, _, _ = _run_gpu(f, None, 7, sub_rows=NR, sub_cols=NC, alpha=8.0, variant=v)
        outs.append(g)
    for g in outs[1:]:
        for k in ("u", "P1", "P2", "lamh", "lamv"):
            assert np.array_equal(g[k], outs[0][k]), k


@pytest.mark.slow
def test_full_size_tvl1_inpainting_2048():
    """TV-L1 inpainting + impulse denoising at 2048^2, 16x16 subdomains of 128^2
    (mask on 20 % of the pixels, 10 % salt and pepper, alpha 1.5): 3 outer
    iterations in the benchmark's launch configuration, every pixel compared."""
    f, mask, _ = synth.tvl1_inpaint_image(2048, 2048, 100, 0.1, 0.2, 0)
    kw = dict(sub_rows=16, sub_cols=16, fidelity="l1", alpha=1.5, inner_iters=10)
    _, g, _, _ = _run_gpu(f, mask, 3, **kw)
    pr, o = _run_oracle(f, mask, 3, **kw)
    assert np.abs(g["u"] - o.u).max() <= U_TOL
    Jg = oracle.energy(pr, g["u"], f.astype(np.float64), mask)
    Jo = oracle.energy(pr, o.u, f.astype(np.float64), mask)
    assert abs(Jg - Jo) <= E_TOL * Jo
