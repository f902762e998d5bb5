"""Pins of the oracle's proximity operators (Section 3, Section 5) against a brute-force
minimisation of each prox objective  s F(v) + 1/2 (v - vbar)^2  (definition of
prox in the assumption on simple proximity operators), pixel by pixel, and of the
prox of G_s^* in the local solver against a brute-force 1-D minimisation of
  chi_[-1,1](p) + 1/(2 tau) (p - phat)^2 + 1/(2 tau0) (p - pbar)^2.
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle


def _argmin_1d(obj, lo, hi):
    xs = np.linspace(lo, hi, 20001)
    vals = np.array([obj(x) for x in xs])
    k = int(np.argmin(vals))
    a, b = xs[max(k - 1, 0)], xs[min(k + 1, len(xs) - 1)]
    r = minimize_scalar(obj, bounds=(a, b), method="bounded", options={"xatol": 1e-13})
    return r.x if r.fun <= vals[k] else xs[k]


@pytest.mark.parametrize("fid", ["l2", "l1", "seg"])
def test_prox_matches_bruteforce(fid):
    rng = np.random.default_rng(11)
    n = 40
    vbar = rng.uniform(-1.0, 2.0, n)
    f = rng.uniform(0.0, 1.0, n)
    mask = (rng.uniform(size=n) < 0.3).astype(np.uint8) if fid != "seg" else None
    s, c1, c2 = 0.37, 0.2, 0.8
    got = oracle.prox(fid, vbar, f, s, mask=mask, c1=c1, c2=c2)
    for k in range(n):
        in_d = mask is not None and mask[k]
        if fid == "l2":
            F = (lambda v: 0.0) if in_d else (lambda v: 0.5 * (v - f[k]) ** 2)
            lo, hi = -3, 3
        elif fid == "l1":
            F = (lambda v: 0.0) if in_d else (lambda v: abs(v - f[k]))
            lo, hi = -3, 3
        else:
            g = (f[k] - c1) ** 2 - (f[k] - c2) ** 2
            F = lambda v: v * g
            lo, hi = 0.0, 1.0
        want = _argmin_1d(lambda v: s * F(v) + 0.5 * (v - vbar[k]) ** 2, lo, hi)
        assert abs(got[k] - want) < 1e-7, (k, got[k], want)


def test_shrink_zero_convention_and_kink():
    f = np.zeros(3)
    v = np.array([0.0, 0.5, -0.5])
    out = oracle.prox("l1", v, f, 0.5)
    assert np.array_equal(out, np.zeros(3))   # |v| = s gives 0, and 0/|0| = 0


def test_local_step_prox_of_G_star():
    """One inner iteration on a tile equals: u-step by the (pinned) prox, then for
    every active dof the brute-force minimiser of the G_s^* prox objective."""
    rng = np.random.default_rng(5)
    mr, mc = 3, 4
    pr = oracle.Problem(mr, mc, fidelity="l2", alpha=4.0, tau=2.0, tau0=0.7, sigma0=0.1)
    f = rng.uniform(0, 1, (mr, mc))
    u0 = rng.uniform(0, 1, (mr, mc))
    p1 = rng.uniform(-1, 1, (mr + 1, mc)); p2 = rng.uniform(-1, 1, (mr, mc + 1))
    ph1 = rng.uniform(-2, 2, p1.shape); ph2 = rng.uniform(-2, 2, p2.shape)
    sides = (1, 1, 1, 1)
    u, q1, q2 = u0.copy(), p1.copy(), p2.copy()
    oracle.local_solve(pr, f, u, q1, q2, ph1, ph2, 1, sides)
    # u-step with pbar = p at the start of a local solve
    want_u = oracle.prox("l2", u0 + 0.1 * oracle.tile_div(p1, p2), f, 0.1 * 4.0)
    assert np.allclose(u, want_u, atol=1e-14)
    g1, g2 = oracle.tile_grad(want_u, *sides)
    for p, g, ph, got in ((p1, g1, ph1, q1), (p2, g2, ph2, q2)):
        for idx in np.ndindex(p.shape):
            pbar = p[idx] + 0.7 * g[idx]
            obj = lambda x: (x - ph[idx]) ** 2 / (2 * 2.0) + (x - pbar) ** 2 / (2 * 0.7)
            want = _argmin_1d(obj, -1.0, 1.0)
            assert abs(got[idx] - want) < 1e-7
