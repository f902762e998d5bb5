"""Pins of the oracle's dual values (the duality-gap certificates) against brute-force
LPs/QPs of 8 x 8 problems written from the definitions.

Weak duality (d(p) <= J(u) for every feasible pair) and strong duality (max_p d(p) =
min_u J(u) for these finite-dimensional convex problems) fix the dual value exactly:
its sign, the scaling that keeps |div p| <= alpha for the L1 fidelity, and the conjugate
of the L2 fidelity (the form alpha F^*(div p / alpha) of the reading of the conjugate
scaling)."""
import numpy as np
import pytest
from scipy.optimize import linprog

import oracle
from bruteforce import fd_matrix, rof, tvl1


def _global_field(q, H, W):
    """q on the interior edges (vertical neighbours first, then horizontal) into the
    global Y layout; fd_matrix's D is -div^T on those edges, so p = q."""
    nv = (H - 1) * W
    p1 = np.zeros((H + 1, W))
    p1[1:H] = q[:nv].reshape(H - 1, W)
    p2 = np.zeros((H, W + 1))
    p2[:, 1:W] = q[nv:].reshape(H, W - 1)
    return p1, p2


def _tvl1_dual_lp(f, alpha):
    """max_{|q| <= 1, |D^T q| <= alpha} <D f, q>: the dual of min_u alpha ||u - f||_1 +
    ||D u||_1 (min over u of alpha |u - f| - u w is -f w when |w| <= alpha, -inf
    otherwise, with w = div p = -D^T q)."""
    H, W = f.shape
    D = fd_matrix(H, W)
    m = D.shape[0]
    A = np.vstack([D.T, -D.T])
    r = linprog(-(D @ f.ravel()), A_ub=A, b_ub=np.full(2 * H * W, alpha), bounds=[(-1, 1)] * m, method="highs",
                options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert r.status == 0
    return _global_field(r.x, H, W), -r.fun


@pytest.mark.parametrize("seed,alpha", [(0, 1.5), (1, 0.7), (2, 3.0)])
def test_l1_dual_value_strong_duality(seed, alpha):
    """At the dual LP's optimum the oracle's L1 dual value equals the primal optimum J*
    of the brute-force LP, and J(u*) = J*."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(0, 1, (8, 8))
    f[rng.uniform(size=f.shape) < 0.15] = 1.0
    pr = oracle.Problem(8, 8, fidelity="l1", alpha=alpha)
    u, J = tvl1(f, alpha)
    (p1, p2), Jd = _tvl1_dual_lp(f, alpha)
    assert abs(Jd - J) <= 1e-9 * max(1.0, abs(J))
    assert abs(oracle.dual_value(pr, p1, p2, f) - J) <= 1e-8 * max(1.0, abs(J))
    assert abs(oracle.energy(pr, u, f) - J) <= 1e-8 * max(1.0, abs(J))


@pytest.mark.parametrize("fid", ["l1", "l2", "seg"])
def test_dual_value_is_a_lower_bound(fid):
    """Weak duality for random fields p in C, including fields with |div p| far above
    alpha (the L1 value must scale them back into its domain) and random images u."""
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, (8, 8))
    alpha = {"l1": 0.6, "l2": 2.0, "seg": 5.0}[fid]
    pr = oracle.Problem(8, 8, fidelity=fid, alpha=alpha, c1=0.2, c2=0.8)
    if fid == "l1":
        _, J = tvl1(f, alpha)
    elif fid == "l2":
        J = oracle.energy(pr, rof(f, alpha), f)
    else:
        from bruteforce import seg
        _, J = seg(f, alpha, 0.2, 0.8)
    for _ in range(200):
        p1, p2 = np.zeros((9, 8)), np.zeros((8, 9))
        p1[1:8] = rng.uniform(-1, 1, (7, 8))
        p2[:, 1:8] = rng.uniform(-1, 1, (8, 7))
        if rng.uniform() < 0.5:   # saturated fields: |div p| up to 4
            p1[1:8] = np.sign(p1[1:8])
            p2[:, 1:8] = np.sign(p2[:, 1:8])
        d = oracle.dual_value(pr, p1, p2, f)
        assert d <= J + 1e-12 * abs(J)
        if fid != "seg":
            u = rng.uniform(-0.5, 1.5, (8, 8))
            assert d <= oracle.energy(pr, u, f) + 1e-12


@pytest.mark.parametrize("seed,alpha", [(4, 3.0), (5, 0.8)])
def test_l2_dual_value_strong_duality(seed, alpha):
    """The ROF dual value at a dual solution equals the primal optimum.  The dual
    solution is recovered from the brute-force minimiser u* by the optimality
    conditions alone (an LP feasibility problem): |p| <= 1, div p = alpha (u* - f)
    (u* = f + div p / alpha), and p_e = sign((D u*)_e) wherever (D u*)_e != 0."""
    f = np.random.default_rng(seed).uniform(0, 1, (8, 8))
    pr = oracle.Problem(8, 8, fidelity="l2", alpha=alpha)
    u = rof(f, alpha)
    D = fd_matrix(8, 8)
    g = D @ u.ravel()
    m = D.shape[0]
    bounds = [(np.sign(v), np.sign(v)) if abs(v) > 1e-9 else (-1, 1) for v in g]
    r = linprog(np.zeros(m), A_eq=-D.T, b_eq=alpha * (u.ravel() - f.ravel()), bounds=bounds, method="highs",
                options={"primal_feasibility_tolerance": 1e-10})
    assert r.status == 0
    p1, p2 = _global_field(r.x, 8, 8)
    J = oracle.energy(pr, u, f)
    assert abs(oracle.dual_value(pr, p1, p2, f) - J) <= 1e-9 * J
