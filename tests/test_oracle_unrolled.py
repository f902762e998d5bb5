"""Pins of the FP64 PyTorch restatement of the unrolled Algorithm 1 (the autograd
reference of the reverse pass): its forward values against the C oracle, and its
autograd derivatives against central differences of the C oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import unrolled_torch as UT

ALPHA = {"l2": 10.0, "l1": 1.5, "seg": 20.0}


def _case(fid, mask_prob, H=48, W=40, seed=0):
    f, clean = synth.rof_image(H, W, 6, 0.08, seed)
    f = f.astype(np.float64)
    mask = None
    if mask_prob:
        mask = synth.bernoulli_mask((H, W), mask_prob, np.random.Generator(np.random.PCG64(seed + 7)))
        f[mask == 1] = 0.0
    return f, clean.astype(np.float64), mask


def _problem(fid, H, W, NR, NC, alpha):
    kw = dict(c1=0.2, c2=0.8, tau=1.0) if fid == "seg" else {}
    return oracle.Problem(H, W, NR, NC, fidelity=fid, alpha=alpha, **kw)


def _torch_kw(fid):
    return dict(c1=0.2, c2=0.8) if fid == "seg" else {}


@pytest.mark.parametrize("fid,mask_prob", [("l2", 0.0), ("l2", 0.2), ("l1", 0.2), ("seg", 0.0)])
def test_forward_matches_c_oracle(fid, mask_prob):
    f, _, mask = _case(fid, mask_prob, H=37, W=29)
    pr = _problem(fid, 37, 29, 3, 2, ALPHA[fid])
    st = oracle.dd_run(pr, f, 7, mask=mask)
    mt = None if mask is None else torch.tensor(mask == 1)
    u = UT.unrolled(torch.tensor(f), torch.tensor(ALPHA[fid], dtype=torch.float64), 3, 2, 7, fidelity=fid,
                    mask=mt, **_torch_kw(fid))
    assert np.abs(u.numpy() - st.u).max() <= 1e-12


@pytest.mark.parametrize("fid,mask_prob", [("l2", 0.0), ("l2", 0.2), ("seg", 0.0)])
def test_autograd_matches_central_differences(fid, mask_prob):
    """FP64 central differences of the C oracle.  The unrolled map is piecewise
    affine in f (L2, and SEG whose g is affine in f): between kinks of the projections
    a central difference is exact up to rounding, so along unit-norm random directions
    with h = 1e-5 (each pixel moves by ~2e-7 and no kink is crossed) autograd must
    agree to 1e-6.  alpha enters nonlinearly (h = 1e-3, 1e-5)."""
    H, W, N = 48, 40, 12
    f, g, mask = _case(fid, mask_prob, H, W)
    a = ALPHA[fid]
    ft = torch.tensor(f, requires_grad=True)
    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    mt = None if mask is None else torch.tensor(mask == 1)
    u = UT.unrolled(ft, at, 3, 2, N, fidelity=fid, mask=mt, **_torch_kw(fid))
    (0.5 * ((u - torch.tensor(g)) ** 2).sum()).backward()
    gf, ga = ft.grad.numpy(), at.grad.item()

    def loss(ff, aa):
        st = oracle.dd_run(_problem(fid, H, W, 3, 2, aa), ff, N, mask=mask)
        return 0.5 * float(((st.u - g) ** 2).sum())

    h = 1e-5
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(3):
        v = rng.standard_normal((H, W))
        if mask is not None:
            v[mask == 1] = 0.0
        v /= np.linalg.norm(v)
        fd = (loss(f + h * v, a) - loss(f - h * v, a)) / (2 * h)
        ad = float((gf * v).sum())
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
    h = 1e-3
    fd = (loss(f, a + h) - loss(f, a - h)) / (2 * h)
    assert abs(fd - ga) <= 1e-5 * abs(fd), (fd, ga)
    if mask is not None:
        assert np.all(gf[mask == 1] == 0.0)

