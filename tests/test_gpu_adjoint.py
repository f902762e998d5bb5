"""Reverse pass of the unrolled outer iterations (dd_tv_adjoint_*) on the GPU.

The derivative of u_N with respect to f and alpha is compared with
  * autograd through the FP64 PyTorch restatement of the unrolled Algorithm 1
    (oracle/unrolled_torch.py, itself pinned to the C oracle and to central
    differences by tests/test_oracle_unrolled.py), field by field;
  * central differences of the FP64 C oracle at the differentiation workload
    (8 ROF images 1024 x 1024, 8 x 8 subdomains, 100 outer iterations,
    checkpoints every 10), along unit-norm random directions with h = 1e-3.
The loss is L = 1/2 ||u_N - g||^2 against the clean image g throughout.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import unrolled_torch as UT

pytestmark = pytest.mark.gpu

ALPHA = {"l2": 10.0, "l1": 1.5, "seg": 20.0}


def _case(H, W, fid, mask_prob, seed):
    f, clean = synth.rof_image(H, W, 6, 0.08, seed)
    mask = None
    if mask_prob:
        mask = synth.bernoulli_mask((H, W), mask_prob, np.random.Generator(np.random.PCG64(seed + 7)))
        f = f.copy()
        f[mask == 1] = 0.0
    return f, clean, mask


def _extra(fid):
    return dict(c1=0.2, c2=0.8) if fid == "seg" else {}


def _gpu(f, g, mask, NR, NC, N, fid, every=5, path="fused", alpha=None, K=10):
    from paper_1901_00682_gb300 import _lib as L
    H, W = f.shape
    a = ALPHA[fid] if alpha is None else alpha
    p = L.make_params(H, W, NR, NC, fidelity=fid, alpha=a, path=path, inner_iters=K, **_extra(fid))
    fd = torch.from_numpy(f).cuda()
    md = None if mask is None else torch.from_numpy(mask).cuda()
    with L.Solver(p) as s:
        u = torch.empty_like(fd)
        s.adjoint_forward(fd, md, N, every, u)
        gu = u - torch.from_numpy(g).cuda()
        gf = torch.empty_like(fd)
        ga = s.adjoint_backward(gu, gf)
        torch.cuda.synchronize()
        return u.cpu().numpy().astype(np.float64), gf.cpu().numpy().astype(np.float64), ga


def _ref(f, g, mask, NR, NC, N, fid, alpha=None, K=10):
    a = ALPHA[fid] if alpha is None else alpha
    ft = torch.tensor(f.astype(np.float64), requires_grad=True)
    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    mt = None if mask is None else torch.tensor(mask == 1)
    u = UT.unrolled(ft, at, NR, NC, N, fidelity=fid, mask=mt, K=K, **_extra(fid))
    (0.5 * ((u - torch.tensor(g.astype(np.float64))) ** 2).sum()).backward()
    return u.detach().numpy(), ft.grad.numpy(), at.grad.item()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("fid,mask_prob,shape,tiles,alpha,K,path", [
    ("l2", 0.0, (48, 40), (3, 2), None, 10, "fused"),
    ("l2", 0.0, (50, 37), (3, 2), None, 10, "fused"),      # ragged tiles
    ("l2", 0.2, (48, 40), (3, 2), None, 10, "fused"),      # inpainting domain
    # segmentation with alpha 20 saturates every pixel at 0 or 1 within a few outer
    # iterations (zero derivative); alpha 1 keeps about 12% of the pixels inside (0, 1)
    ("seg", 0.0, (48, 40), (2, 2), 1.0, 10, "fused"),
    ("l2", 0.0, (100, 90), (2, 2), None, 6, "fused"),      # 50 x 45 tiles: the 64-column mapping
    ("l2", 0.0, (256, 256), (2, 2), None, 4, "fused"),     # 128 x 128 tiles: clusters of 8 CTAs
    ("l2", 0.0, (128, 128), (2, 2), None, 16, "fused"),
    # 80 x 150 tiles are wider than the tile-fused reverse kernel: the tape is recorded
    # in global memory by the plain path's kernels and reversed by the per-step kernels
    ("l2", 0.0, (160, 150), (2, 1), None, 6, "plain"),
    ("l2", 0.2, (160, 150), (2, 1), None, 6, "plain"),
])
def test_adjoint_matches_fp64_autograd(cuda_lib, fid, mask_prob, shape, tiles, alpha, K, path):
    H, W = shape
    f, g, mask = _case(H, W, fid, mask_prob, seed=0 if fid == "seg" else 3)
    N = 12 if H * W < 10000 else 4
    u, gf, ga = _gpu(f, g, mask, *tiles, N, fid, alpha=alpha, K=K, path=path)
    ur, gfr, gar = _ref(f, g, mask, *tiles, N, fid, alpha=alpha, K=K)
    assert np.abs(u - ur).max() <= 5e-4
    assert gar != 0.0 and np.abs(gfr).max() > 0.0
    rf, ra = _rel(gf, gfr), abs(ga - gar) / abs(gar)
    print(f"{fid} mask={mask_prob} {shape}: rel|dL/df| {rf:.2e}  rel dL/dalpha {ra:.2e}")
    assert rf <= 1e-3, rf
    assert ra <= 1e-3, ra
    if mask is not None:
        assert np.all(gf[mask == 1] == 0.0)


def test_adjoint_l1_matches_fp64_autograd(cuda_lib):
    """TV-L1 inpainting: the unrolled map has kinks almost everywhere (the shrink
    decision flips for pixels whose residual sits at the threshold), so a handful of
    decisions taken differently in float32 and float64 perturb the derivative locally.
    The bulk must agree: the directional derivative along the loss gradient's own
    direction and the alpha derivative to 1e-2, the field to 5e-2."""
    f, g, mask = _case(48, 40, "l1", 0.2, seed=3)
    u, gf, ga = _gpu(f, g, mask, 3, 2, 12, "l1")
    ur, gfr, gar = _ref(f, g, mask, 3, 2, 12, "l1")
    assert np.abs(u - ur).max() <= 5e-4
    rf = _rel(gf, gfr)
    rd = abs(float((gf * gfr).sum()) - float((gfr * gfr).sum())) / float((gfr * gfr).sum())
    ra = abs(ga - gar) / abs(gar)
    print(f"l1: rel field {rf:.2e} directional {rd:.2e} alpha {ra:.2e}")
    assert rf <= 5e-2 and rd <= 1e-2 and ra <= 1e-2


def test_adjoint_checkpoint_spacing_and_path_do_not_change_bits(cuda_lib):
    """Recomputation is deterministic and the fused and plain paths run the same
    arithmetic, so the gradient does not depend on the checkpoint spacing or path: u
    and dL/df bit for bit; dL/dalpha bit for bit across checkpoint spacings, and to 1e-6
    relative between the paths (the fused reverse kernels sum each thread's share in
    compensated float32, the plain path every pixel's term in float64)."""
    f, g, mask = _case(64, 48, "l2", 0.0, seed=5)
    N = 9
    base = _gpu(f, g, None, 2, 3, N, "l2", every=1)
    for every, path in [(2, "fused"), (4, "fused"), (9, "fused"), (50, "fused"), (3, "plain")]:
        u, gf, ga = _gpu(f, g, None, 2, 3, N, "l2", every=every, path=path)
        assert np.array_equal(u, base[0]), (every, path)
        assert np.array_equal(gf, base[1]), (every, path)
        if path == "fused":
            assert ga == base[2], (every, path)
        else:
            assert abs(ga - base[2]) <= 1e-6 * abs(base[2]), (every, path, ga, base[2])


def test_full_tile_reverse_kernel_against_plain_path(cuda_lib):
    """With 128 x 128 subdomains the fused path runs the full-tile reverse kernel, which
    sums its share of dL/dalpha in compensated float32 per thread (float64 across
    threads); the plain path sums in float64 per pixel.  dL/df is bit-identical, dL/dalpha
    agrees to 1e-6 relative."""
    f, g, _ = _case(256, 256, "l2", 0.0, seed=7)
    N = 6
    u1, gf1, ga1 = _gpu(f, g, None, 2, 2, N, "l2", every=3, path="fused")
    u2, gf2, ga2 = _gpu(f, g, None, 2, 2, N, "l2", every=3, path="plain")
    assert np.array_equal(u1, u2)
    assert np.array_equal(gf1, gf2)
    assert ga2 != 0.0 and abs(ga1 - ga2) <= 1e-6 * abs(ga2), (ga1, ga2)


def test_adjoint_backward_repeats_and_profiling_mode(cuda_lib):
    """A second backward on the same checkpoints (graph replay) and a backward with the
    measurement hooks on (direct launches) give the bits of the first one."""
    from paper_1901_00682_gb300 import _lib as L
    f, g, _ = _case(64, 48, "l2", 0.0, seed=6)
    with L.Solver(L.make_params(64, 48, 2, 3)) as s:
        fd = torch.from_numpy(f).cuda()
        u = torch.empty_like(fd)
        s.adjoint_forward(fd, None, 7, 3, u)
        gu = u - torch.from_numpy(g).cuda()
        outs = []
        for prof in (False, False, True):
            s.set_profiling(prof)
            gf = torch.empty_like(fd)
            ga = s.adjoint_backward(gu, gf)
            outs.append((gf.cpu().numpy(), ga))
        s.set_profiling(False)
        s.profile_read()
    for gf, ga in outs[1:]:
        assert np.array_equal(gf, outs[0][0]) and ga == outs[0][1]


def test_adjoint_zero_outer_iterations(cuda_lib):
    """N = 0: u_0 = f, so dL/df = u_0 - g and dL/dalpha = 0."""
    f, g, _ = _case(32, 32, "l2", 0.0, seed=1)
    u, gf, ga = _gpu(f, g, None, 2, 2, 0, "l2")
    assert np.array_equal(u, f.astype(np.float64))
    np.testing.assert_allclose(gf, (f - g).astype(np.float64), rtol=0, atol=1e-7)
    assert ga == 0.0


def test_adjoint_errors(cuda_lib):
    from paper_1901_00682_gb300 import _lib as L
    f = torch.zeros(32, 32, device="cuda")
    u = torch.empty_like(f)
    with L.Solver(L.make_params(32, 32, 2, 2)) as s:
        with pytest.raises(L.DDTVError) as e:
            s.adjoint_backward(f, u)            # no forward yet
        assert e.value.code == L.EINVAL
        with pytest.raises(L.DDTVError):
            s.adjoint_forward(f, None, 4, 0, u)  # checkpoint_every < 1
        s.adjoint_forward(f, None, 4, 2, u)
        s.load(f)                                # a load invalidates the checkpoints
        with pytest.raises(L.DDTVError):
            s.adjoint_backward(f, u)
        with pytest.raises(L.DDTVError):
            s.set_alpha(-1.0)
        s.adjoint_forward(f, None, 4, 2, u)
        s.set_alpha(7.0)                         # a new alpha invalidates the checkpoints
        with pytest.raises(L.DDTVError) as e:
            s.adjoint_backward(f, u)
        assert e.value.code == L.EINVAL
        s.adjoint_forward(f, None, 4, 2, u)      # the same alpha again keeps them valid
        s.set_alpha(7.0)
        s.adjoint_backward(f, torch.empty_like(f))
    with L.Solver(L.make_params(32, 32, path="fulldim")) as s:
        with pytest.raises(L.DDTVError) as e:
            s.adjoint_forward(f, None, 4, 2, u)
        assert e.value.code == L.EUNSUPPORTED


def test_autograd_function_batch_and_alpha(cuda_lib):
    """torch.autograd through UnrolledDDTV: a batch with per-image handles and streams
    gives each image's gradient of the single-image call, and dL/dalpha summed over
    the batch (shared alpha) or per image ((B,) alpha)."""
    from paper_1901_00682_gb300.autograd import UnrolledDDTV
    B, H, W, N = 3, 48, 40, 6
    fs, gs = zip(*[_case(H, W, "l2", 0.0, seed=10 + b)[:2] for b in range(B)])
    f = torch.from_numpy(np.stack(fs)).cuda().requires_grad_(True)
    g = torch.from_numpy(np.stack(gs)).cuda()
    alpha = torch.tensor(10.0, dtype=torch.float64, device="cuda", requires_grad=True)
    mod = UnrolledDDTV(H, W, 3, 2, N, checkpoint_every=4)
    u = mod(f, alpha)
    (0.5 * ((u - g) ** 2).sum()).backward()
    singles = [_gpu(fs[b], gs[b], None, 3, 2, N, "l2", every=4) for b in range(B)]
    for b in range(B):
        assert np.array_equal(u[b].detach().cpu().numpy().astype(np.float64), singles[b][0])
        assert np.array_equal(f.grad[b].cpu().numpy().astype(np.float64), singles[b][1])
    assert abs(alpha.grad.item() - sum(s[2] for s in singles)) <= 1e-12 * abs(alpha.grad.item())
    # per-image alpha, changed between calls (dd_tv_set_alpha)
    f.grad = None
    alphas = torch.tensor([8.0, 10.0, 12.0], dtype=torch.float64, device="cuda", requires_grad=True)
    u = mod(f, alphas)
    (0.5 * ((u - g) ** 2).sum()).backward()
    for b in range(B):
        s = _gpu(fs[b], gs[b], None, 3, 2, N, "l2", every=4, alpha=float(alphas[b].detach()))
        assert np.array_equal(f.grad[b].cpu().numpy().astype(np.float64), s[1])
        assert alphas.grad[b].item() == s[2]
    mod.close()


def test_autograd_two_forwards_before_their_backwards(cuda_lib):
    """Two calls of the module before either backward (each forward keeps its own
    checkpoints): each backward, in either order, gives the single-call gradients."""
    from paper_1901_00682_gb300.autograd import UnrolledDDTV
    B, H, W, N = 2, 48, 40, 6
    cases = [[_case(H, W, "l2", 0.0, seed=30 + 10 * k + b)[:2] for b in range(B)] for k in range(2)]
    mod = UnrolledDDTV(H, W, 3, 2, N, checkpoint_every=4)
    fs, losses, alphas = [], [], []
    for k in range(2):
        f = torch.from_numpy(np.stack([c[0] for c in cases[k]])).cuda().requires_grad_(True)
        g = torch.from_numpy(np.stack([c[1] for c in cases[k]])).cuda()
        a = torch.tensor(10.0 + k, dtype=torch.float64, device="cuda", requires_grad=True)
        u = mod(f, a)
        fs.append(f)
        alphas.append(a)
        losses.append(0.5 * ((u - g) ** 2).sum())
    losses[1].backward()
    losses[0].backward()
    for k in range(2):
        for b in range(B):
            s = _gpu(cases[k][b][0], cases[k][b][1], None, 3, 2, N, "l2", every=4, alpha=10.0 + k)
            assert np.array_equal(fs[k].grad[b].cpu().numpy().astype(np.float64), s[1]), (k, b)
        want = sum(_gpu(cases[k][b][0], cases[k][b][1], None, 3, 2, N, "l2", every=4, alpha=10.0 + k)[2]
                   for b in range(B))
        assert abs(alphas[k].grad.item() - want) <= 1e-12 * abs(want)
    mod.close()


def _oracle_loss(f64, g64, alpha, N):
    pr = oracle.Problem(f64.shape[0], f64.shape[1], 8, 8, alpha=alpha)
    st = oracle.dd_run(pr, f64, N)
    return 0.5 * float(((st.u - g64) ** 2).sum())


def test_adjoint_fd_differentiation_workload(cuda_lib):
    """8 ROF images 1024 x 1024 (sigma 0.08, alpha 10), 8 x 8 subdomains, K = 100
    outer iterations of 10 inner ones, checkpoints every 10, through the autograd
    Function, against FP64 central differences of the C oracle.

    Along unit-norm random directions v, a step h = 1e-3 moves each pixel by ~1e-6,
    which still crosses a few kinks of the 1000 unrolled projections: the central
    difference then carries an error of a few 1e-7 in absolute terms, which exceeds
    1e-3 relative where the directional derivative is small by cancellation.  So:
      * against h = 1e-5 (kink-free; the derivative itself): 1e-3 relative;
      * against h = 1e-3: 1e-3 relative to max(|fd|, ||dL/df||_2 / sqrt(H W)), the
        root-mean-square directional derivative over unit random directions;
      * along the gradient's own direction and for alpha, h = 1e-3: 1e-3 relative."""
    from paper_1901_00682_gb300.autograd import UnrolledDDTV
    B, S, N = 8, 1024, 100
    fs, gs = [], []
    for b in range(B):
        f, clean = synth.rof_image(S, S, 400 // 16, 0.08, 500 + b)
        fs.append(f)
        gs.append(clean)
    f = torch.from_numpy(np.stack(fs)).cuda().requires_grad_(True)
    g = torch.from_numpy(np.stack(gs)).cuda()
    alpha = torch.tensor([10.0] * B, dtype=torch.float64, device="cuda", requires_grad=True)
    mod = UnrolledDDTV(S, S, 8, 8, N, checkpoint_every=10)
    u = mod(f, alpha)
    (0.5 * ((u - g) ** 2).sum()).backward()
    gf = f.grad.cpu().numpy().astype(np.float64)
    ga = alpha.grad.cpu().numpy()
    mod.close()

    def fd(b, v, h):
        f64, g64 = fs[b].astype(np.float64), gs[b].astype(np.float64)
        return (_oracle_loss(f64 + h * v, g64, 10.0, N) - _oracle_loss(f64 - h * v, g64, 10.0, N)) / (2 * h)

    rng = np.random.Generator(np.random.PCG64(77))
    for b in (0, 5):
        v = rng.standard_normal((S, S))
        v /= np.linalg.norm(v)
        ad = float((gf[b] * v).sum())
        fd3, fd5 = fd(b, v, 1e-3), fd(b, v, 1e-5)
        scale = max(abs(fd3), float(np.linalg.norm(gf[b])) / S)
        print(f"image {b}: adjoint {ad:.8e}  fd(1e-5) {fd5:.8e} rel {abs(fd5 - ad) / abs(fd5):.2e}  "
              f"fd(1e-3) {fd3:.8e} rel-to-scale {abs(fd3 - ad) / scale:.2e}")
        assert abs(fd5 - ad) <= 1e-3 * abs(fd5)
        assert abs(fd3 - ad) <= 1e-3 * scale
    b = 0
    v = gf[b] / np.linalg.norm(gf[b])
    ad, fd3 = float((gf[b] * v).sum()), fd(b, v, 1e-3)
    print(f"image {b} along its gradient: adjoint {ad:.8e} fd(1e-3) {fd3:.8e} rel {abs(fd3 - ad) / abs(fd3):.2e}")
    assert abs(fd3 - ad) <= 1e-3 * abs(fd3)
    b, h = 2, 1e-3
    f64, g64 = fs[b].astype(np.float64), gs[b].astype(np.float64)
    fda = (_oracle_loss(f64, g64, 10.0 + h, N) - _oracle_loss(f64, g64, 10.0 - h, N)) / (2 * h)
    print(f"image {b}: alpha fd {fda:.8e} adjoint {ga[b]:.8e} rel {abs(fda - ga[b]) / abs(fda):.2e}")
    assert abs(fda - ga[b]) <= 1e-3 * abs(fda)
