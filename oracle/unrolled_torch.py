"""FP64 PyTorch restatement of the unrolled Algorithm 1, for autograd (TEST INFRASTRUCTURE).

Algorithm 1 (Section 4) with the accelerated local solver of Section 5, written with
plain PyTorch CPU tensor operations in float64 on the torn layout of the C oracle
(P1 (H+NR) x W, P2 H x (W+NC), lamh (NR-1) x W, lamv (NC-1) x H), so that
torch.autograd differentiates the unrolled map (f, alpha) -> u_N.  The paper never
differentiates its method; the derivative at the kinks of the pointwise maps is a
reading, and every kink is written with an explicit torch.where that fixes it:

  * projection onto [-1, 1] (dual constraint set C): passes iff -1 <= t <= 1;
  * L1 prox f + shr(v, s) with v = ubar - f: passes ubar iff |v| > s, else f;
  * segmentation prox clamp(ubar - s g, 0, 1): passes iff 0 <= x <= 1.

Only the tests import this module; it shares no code with the CUDA library.  Its
forward values are pinned against the C oracle, and its derivatives against central
differences of the C oracle, by the tests.
"""
from __future__ import annotations

import math

import torch


def part(a, n, k):
    return (a * n) // k


def _clamp_box(t, lo, hi):
    """clamp with derivative 1 iff lo <= t <= hi."""
    return torch.where(t > hi, torch.full_like(t, hi), torch.where(t < lo, torch.full_like(t, lo), t))


def _prox(fid, ubar, f, s, in_d, c1, c2):
    """prox_{s F} at ubar (Section 3 proximity maps); s = sigma_k alpha (a tensor)."""
    if fid == "seg":
        g = (f - c1) ** 2 - (f - c2) ** 2
        return _clamp_box(ubar - s * g, 0.0, 1.0)
    if fid == "l2":
        out = (ubar + s * f) / (1.0 + s)
    else:
        v = ubar - f
        out = torch.where(v.abs() > s, ubar - s * torch.sign(v), f)
    if in_d is not None:
        out = torch.where(in_d, ubar, out)
    return out


def _local_solve(u, p1, p2, h1, h2, f, in_d, alpha, act, pr, K):
    """Accelerated local iteration on one tile (Section 5), restarted schedule."""
    top, bot, lft, rgt = act
    mr, mc = u.shape
    m1 = torch.ones(mr + 1, mc, dtype=u.dtype)
    m2 = torch.ones(mr, mc + 1, dtype=u.dtype)
    if not top:
        m1[0] = 0
    if not bot:
        m1[-1] = 0
    if not lft:
        m2[:, 0] = 0
    if not rgt:
        m2[:, -1] = 0
    tau, gamma = pr["tau"], pr["gamma"]
    q1, q2 = p1, p2
    tk, sk = pr["tau0"], pr["sigma0"]
    zrow = torch.zeros(1, mc, dtype=u.dtype)
    zcol = torch.zeros(mr, 1, dtype=u.dtype)
    for _ in range(K):
        d = (q1[1:] - q1[:-1]) + (q2[:, 1:] - q2[:, :-1])
        u = _prox(pr["fid"], u + sk * d, f, sk * alpha, in_d, pr["c1"], pr["c2"])
        up = torch.cat([zrow, u, zrow], 0)
        g1 = up[1:] - up[:-1]
        uq = torch.cat([zcol, u, zcol], 1)
        g2 = uq[:, 1:] - uq[:, :-1]
        th = 1.0 / math.sqrt(1.0 + 2.0 * gamma * tk)
        n1 = _clamp_box((tau * (p1 + tk * g1) + tk * h1) / (tau + tk), -1.0, 1.0) * m1
        n2 = _clamp_box((tau * (p2 + tk * g2) + tk * h2) / (tau + tk), -1.0, 1.0) * m2
        q1 = n1 + th * (n1 - p1)
        q2 = n2 + th * (n2 - p2)
        p1, p2 = n1, n2
        tk, sk = th * tk, sk / th
    return u, p1, p2


def unrolled(f, alpha, NR, NC, n_outer, fidelity="l2", mask=None, c1=0.0, c2=0.0, K=10, tau=None,
             sigma=None, tau0=10.0, sigma0=None, gamma=None):
    """u_N of Algorithm 1 from u^0 = f (0 on D; 1/2 for segmentation), p = 0,
    lambda = 0; differentiable in f (H x W float64 tensor) and alpha (0-d float64
    tensor).  mask: bool H x W tensor of the inpainting domain D, or None."""
    tau = (1.0 if fidelity == "seg" else 50.0) if tau is None else tau
    pr = dict(fid=fidelity, tau=tau, tau0=tau0, c1=c1, c2=c2,
              sigma0=0.125 / tau0 if sigma0 is None else sigma0,
              gamma=1.0 / (8.0 * tau) if gamma is None else gamma)
    sigma = 0.5 / tau if sigma is None else sigma
    H, W = f.shape
    dt = f.dtype
    if fidelity == "seg":
        u = torch.full((H, W), 0.5, dtype=dt)
    elif mask is not None:
        u = torch.where(mask, torch.zeros_like(f), f)
    else:
        u = f
    P1 = torch.zeros(H + NR, W, dtype=dt)
    P2 = torch.zeros(H, W + NC, dtype=dt)
    P1p, P2p = P1, P2
    lamh = torch.zeros(NR - 1, W, dtype=dt)
    lamv = torch.zeros(NC - 1, H, dtype=dt)
    rows = [(part(a, H, NR), part(a + 1, H, NR)) for a in range(NR)]
    cols = [(part(b, W, NC), part(b + 1, W, NC)) for b in range(NC)]
    for _ in range(n_outer):
        # multipliers: lambda += sigma B (2 p~^n - p~^{n-1}), (B p)_e = p_s - p_t
        if NR > 1:
            rs = [part(a + 1, H, NR) + a for a in range(NR - 1)]
            jn = torch.stack([P1[r] - P1[r + 1] for r in rs])
            jp = torch.stack([P1p[r] - P1p[r + 1] for r in rs])
            lamh = lamh + sigma * (2.0 * jn - jp)
        if NC > 1:
            cs = [part(b + 1, W, NC) + b for b in range(NC - 1)]
            jn = torch.stack([P2[:, c] - P2[:, c + 1] for c in cs])
            jp = torch.stack([P2p[:, c] - P2p[:, c + 1] for c in cs])
            lamv = lamv + sigma * (2.0 * jn - jp)
        # proximal centre phat = p~^n - tau B^* lambda^{n+1}
        Ph1, Ph2 = P1.clone(), P2.clone()
        for a in range(NR - 1):
            r = part(a + 1, H, NR) + a
            Ph1[r] = P1[r] - tau * lamh[a]
            Ph1[r + 1] = P1[r + 1] + tau * lamh[a]
        for b in range(NC - 1):
            c = part(b + 1, W, NC) + b
            Ph2[:, c] = P2[:, c] - tau * lamv[b]
            Ph2[:, c + 1] = P2[:, c + 1] + tau * lamv[b]
        P1p, P2p = P1, P2
        ru, r1, r2 = [], [], []
        for a, (i0, i1) in enumerate(rows):
            bu, b1, b2 = [], [], []
            for b, (j0, j1) in enumerate(cols):
                act = (a > 0, a + 1 < NR, b > 0, b + 1 < NC)
                lu, l1, l2 = _local_solve(u[i0:i1, j0:j1], P1[i0 + a:i1 + a + 1, j0:j1],
                                          P2[i0:i1, j0 + b:j1 + b + 1], Ph1[i0 + a:i1 + a + 1, j0:j1],
                                          Ph2[i0:i1, j0 + b:j1 + b + 1], f[i0:i1, j0:j1],
                                          None if mask is None else mask[i0:i1, j0:j1], alpha, act, pr, K)
                bu.append(lu)
                b1.append(l1)
                b2.append(l2)
            ru.append(torch.cat(bu, 1))
            r1.append(torch.cat(b1, 1))
            r2.append(torch.cat(b2, 1))
        u, P1, P2 = torch.cat(ru, 0), torch.cat(r1, 0), torch.cat(r2, 0)
    return u
