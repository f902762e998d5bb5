"""Pins of the oracle's solvers (Algorithm 1 and the full-dimension primal-dual
comparator) against results fixed outside the oracle:

* brute-force QP/LP minimisers of 8x8 instances (tests/bruteforce.py) for ROF,
  TV-L1, L1 inpainting, L2 inpainting and convex Chan-Vese segmentation
  (Theorem on the convergence of u^(n) and its corollary on J(u^(n)) -> J(u*));
* the closed-form ROF solution of a one-step image (rows decouple under the
  anisotropic TV; each side moves by 1/(alpha * width) toward the other);
* constant f = c converges to u = c with multipliers lambda = -c;
* DD with a 1x1 grid and DD with many subdomains reach the single-domain solution,
  with the jump B p~ -> 0 (Proposition on the equivalence of the torn saddle problem);
* the primal-dual gap of the averaged dual field goes to 0 (weak duality).
"""
import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth


def _img(H, W, seed, shapes=3, sigma=0.1):
    f, _ = synth.rof_image(H, W, shapes, sigma, seed)
    return f.astype(np.float64)


@pytest.mark.parametrize("grid", [(1, 1), (2, 2), (3, 3), (1, 2), (4, 1), (8, 8)])
@pytest.mark.parametrize("seed", [0, 1])
def test_rof_bruteforce_8x8(grid, seed):
    f = _img(8, 8, seed)
    ub = bf.rof(f, 10.0)
    pr = oracle.Problem(8, 8, *grid, fidelity="l2", alpha=10.0, inner=10)
    st = oracle.dd_run(pr, f, 3000)
    assert np.abs(st.u - ub).max() < 1e-9
    jh, jv = oracle.jump(pr, st.P1, st.P2)
    assert (np.abs(jh).max(initial=0) < 1e-8) and (np.abs(jv).max(initial=0) < 1e-8)


def test_rof_bruteforce_8x8_single_domain_cp():
    f = _img(8, 8, 2)
    ub = bf.rof(f, 10.0)
    cp = oracle.cp_run(oracle.Problem(8, 8, alpha=10.0), f, 20000)
    assert np.abs(cp.u - ub).max() < 1e-9


@pytest.mark.parametrize("grid", [(1, 1), (2, 2), (3, 2)])
def test_tvl1_bruteforce_8x8(grid):
    f = _img(8, 8, 3)
    _, Jstar = bf.tvl1(f, 1.5)
    pr = oracle.Problem(8, 8, *grid, fidelity="l1", alpha=1.5)
    st = oracle.dd_run(pr, f, 4000)
    assert abs(oracle.energy(pr, st.u, f) - Jstar) <= 1e-8 * Jstar


def test_l1_inpainting_bruteforce_8x8():
    f, mask, _ = synth.tvl1_inpaint_image(8, 8, 3, 0.1, 0.2, 4)
    f = f.astype(np.float64)
    assert mask.any()
    _, Jstar = bf.tvl1(f, 1.5, mask)
    pr = oracle.Problem(8, 8, 2, 2, fidelity="l1", alpha=1.5)
    st = oracle.dd_run(pr, f, 4000, mask=mask)
    assert abs(oracle.energy(pr, st.u, f, mask) - Jstar) <= 1e-8 * Jstar


def test_l2_inpainting_bruteforce_8x8():
    rng = np.random.default_rng(9)
    f = _img(8, 8, 5)
    mask = (rng.uniform(size=(8, 8)) < 0.25).astype(np.uint8)
    f[mask == 1] = 0.0
    _, Jstar = bf.l2_inpaint(f, 10.0, mask)
    pr = oracle.Problem(8, 8, 2, 2, fidelity="l2", alpha=10.0)
    st = oracle.dd_run(pr, f, 4000, mask=mask)
    J = oracle.energy(pr, st.u, f, mask)
    # SLSQP is accurate to ~1e-9 here; the oracle must not be worse than it
    assert J <= Jstar + 1e-8 * Jstar
    assert abs(J - Jstar) <= 1e-7 * Jstar


@pytest.mark.parametrize("grid", [(1, 1), (2, 2)])
def test_segmentation_bruteforce_8x8(grid):
    f = _img(8, 8, 6, sigma=0.05)
    _, Jstar = bf.seg(f, 20.0, 0.2, 0.8)
    pr = oracle.Problem(8, 8, *grid, fidelity="seg", alpha=20.0, c1=0.2, c2=0.8, tau=1.0)
    st = oracle.dd_run(pr, f, 4000)
    assert abs(oracle.energy(pr, st.u, f) - Jstar) <= 1e-8 * abs(Jstar)
    assert st.u.min() >= 0.0 and st.u.max() <= 1.0


def _step_solution(H, W, c, a, b, alpha):
    left = a + np.sign(b - a) / (alpha * c)
    right = b - np.sign(b - a) / (alpha * (W - c))
    if (right - left) * (b - a) < 0:       # the two sides meet: both at the weighted mean
        left = right = (c * a + (W - c) * b) / W
    u = np.empty((H, W))
    u[:, :c] = left
    u[:, c:] = right
    return u


@pytest.mark.parametrize("H,W,c,grid", [
    (8, 16, 8, (2, 2)),    # step on the vertical interface
    (8, 16, 5, (2, 2)),    # step inside a subdomain
    (6, 12, 4, (3, 3)),    # step on an interface of a 3x3 grid
    (5, 9, 3, (2, 3)),     # ragged tiles
    (1, 2, 1, (1, 2)),     # smallest DD case: two one-pixel subdomains
])
def test_step_image_closed_form(H, W, c, grid):
    a, b, alpha = 0.2, 0.9, 4.0
    f = np.where(np.arange(W)[None, :] < c, a, b) * np.ones((H, 1))
    want = _step_solution(H, W, c, a, b, alpha)
    pr = oracle.Problem(H, W, *grid, fidelity="l2", alpha=alpha)
    st = oracle.dd_run(pr, f, 3000)
    assert np.abs(st.u - want).max() < 1e-9


def test_step_image_merged_sides():
    # small alpha: the two sides merge into the weighted mean
    H, W, c, a, b, alpha = 4, 8, 3, 0.4, 0.6, 0.5
    f = np.where(np.arange(W)[None, :] < c, a, b) * np.ones((H, 1))
    want = _step_solution(H, W, c, a, b, alpha)
    assert np.ptp(want) == 0.0
    pr = oracle.Problem(H, W, 2, 2, fidelity="l2", alpha=alpha)
    st = oracle.dd_run(pr, f, 3000)
    assert np.abs(st.u - want).max() < 1e-9


@pytest.mark.parametrize("fid", ["l2", "l1"])
def test_constant_image_limit(fid):
    """Constant f = c: u* = c and every divergence-free p in C is a dual solution.
    Optimality of the torn Lagrangian in p~ then needs B^* lambda = D_s c on the
    interface dofs (D_s c = -c on a bottom/right side, +c on a top/left side), i.e.
    lambda* = -c on every interface edge; this fixes the signs of B and of the
    multiplier update.  (It is not a fixed point from step 0: the first p-step sees
    D_s u = +-u on the interface dofs.)"""
    c = 0.37
    f = np.full((12, 10), c)
    pr = oracle.Problem(12, 10, 3, 2, fidelity=fid, alpha=5.0)
    st = oracle.dd_run(pr, f, 3000)
    assert np.abs(st.u - c).max() < 1e-12
    assert np.abs(st.lamh + c).max() < 1e-12 and np.abs(st.lamv + c).max() < 1e-12
    jh, jv = oracle.jump(pr, st.P1, st.P2)
    assert max(np.abs(jh).max(), np.abs(jv).max()) < 1e-12
    p1, p2 = oracle.torn_to_global(pr, st.P1, st.P2)
    assert np.abs(oracle.div(p1, p2)).max() < 1e-12
    assert np.abs(st.P1).max() <= 1.0 and np.abs(st.P2).max() <= 1.0


def test_dd_matches_single_domain_and_gap_vanishes():
    f = _img(32, 32, 7, shapes=5, sigma=0.05)
    pr1 = oracle.Problem(32, 32, alpha=10.0)
    cp = oracle.cp_run(pr1, f, 20000)
    J1, d1 = oracle.energy(pr1, cp.u, f), oracle.dual_value(pr1, cp.p1, cp.p2, f)
    assert 0 <= J1 - d1 < 1e-10 * J1
    pr = oracle.Problem(32, 32, 4, 4, alpha=10.0)
    st = oracle.dd_run(pr, f, 1500)
    J, d = oracle.dd_gap(pr, st, f)
    assert J - d >= -1e-12 * J          # weak duality
    assert J - d < 1e-7 * J
    assert np.abs(st.u - cp.u).max() < 1e-6
    jh, jv = oracle.jump(pr, st.P1, st.P2)
    assert max(np.abs(jh).max(), np.abs(jv).max()) < 1e-6


def test_energy_tends_to_minimum():
    f = _img(16, 16, 8, shapes=4)
    pr = oracle.Problem(16, 16, 2, 2, alpha=10.0)
    st = oracle.dd_run(pr, f, 400, trace=True)
    cp = oracle.cp_run(oracle.Problem(16, 16, alpha=10.0), f, 20000)
    Jstar = oracle.energy(pr, cp.u, f)
    e = np.array(st.energies)
    rel = (e - Jstar) / Jstar
    assert rel.min() >= -1e-12
    assert rel[-1] < 1e-9
    assert rel[-1] < 1e-3 * rel[0]


def test_resume_is_bit_identical():
    f = _img(16, 12, 9)
    pr = oracle.Problem(16, 12, 2, 3, alpha=10.0)
    a = oracle.dd_run(pr, f, 30)
    b = oracle.dd_run(pr, f, 10)
    b = oracle.dd_run(pr, f, 20, state=b)
    for x, y in ((a.u, b.u), (a.P1, b.P1), (a.P2, b.P2), (a.lamh, b.lamh), (a.lamv, b.lamv)):
        assert np.array_equal(x, y)


def test_seg_gap_certificate():
    f = _img(16, 16, 10, sigma=0.05)
    pr = oracle.Problem(16, 16, 2, 2, fidelity="seg", alpha=20.0, c1=0.2, c2=0.8, tau=1.0)
    st = oracle.dd_run(pr, f, 2000)
    J, d = oracle.dd_gap(pr, st, f)
    assert J - d >= -1e-10 * abs(J)
    assert J - d < 1e-6 * abs(J)


# ---- adaptive inner stopping (Section 5, eq. stop_inner1)

def test_inner_stop_rule_matches_its_definition():
    """The oracle's adaptive count for one tile equals the first k with
    ||p^k - p^{k-1}||_2 < tol ||p^k||_2, recomputed here with numpy from k-iteration
    local solves started from the same state (the schedule restarts at every call)."""
    H = W = 24
    f, _ = synth.rof_image(H, W, 4, 0.05, 2)
    pr = oracle.Problem(H, W, 2, 2, alpha=10.0, inner=60)
    st = oracle.dd_run(pr, f, 3)                       # a warm state with nonzero interfaces
    st2 = oracle.dd_run(pr, f, 1, state=st.copy(), inner_tol=2e-3, record=True)
    # tile (0, 0): rows 0..11, cols 0..11; its proximal centre from the state's multipliers
    lamh = st.lamh + pr.c().sigma * (2 * oracle.jump(pr, st.P1, st.P2)[0] - oracle.jump(pr, st.P1prev, st.P2prev)[0])
    lamv = st.lamv + pr.c().sigma * (2 * oracle.jump(pr, st.P1, st.P2)[1] - oracle.jump(pr, st.P1prev, st.P2prev)[1])
    B1, B2 = oracle.jump_adjoint(pr, lamh, lamv)
    Ph1, Ph2 = st.P1 - pr.tau * B1, st.P2 - pr.tau * B2
    u0 = np.ascontiguousarray(st.u[:12, :12])
    p10, p20 = np.ascontiguousarray(st.P1[0:13, :12]), np.ascontiguousarray(st.P2[:12, 0:13])
    h1, h2 = np.ascontiguousarray(Ph1[0:13, :12]), np.ascontiguousarray(Ph2[:12, 0:13])
    fl = np.ascontiguousarray(f[:12, :12], dtype=np.float64)
    prev = (p10, p20)
    first = None
    for k in range(1, 61):
        u, q1, q2 = u0.copy(), p10.copy(), p20.copy()
        oracle.local_solve(pr, fl, u, q1, q2, h1, h2, k, sides=(0, 1, 0, 1))
        num = np.sqrt(((q1 - prev[0]) ** 2).sum() + ((q2 - prev[1]) ** 2).sum())
        den = np.sqrt((q1 ** 2).sum() + (q2 ** 2).sum())
        if num < 2e-3 * den:
            first = k
            break
        prev = (q1, q2)
    assert first is not None and 1 < first < 60
    assert st2.inner_counts[0, 0] == first
    assert np.all(st2.inner_counts <= 60) and np.all(st2.inner_counts >= 1)


def test_inner_stop_constant_image_single_domain():
    """One subdomain, constant f: D u = 0 and p stays 0, which the rule counts as
    converged after one iteration."""
    pr = oracle.Problem(16, 16, 1, 1, alpha=10.0, inner=40)
    st = oracle.dd_run(pr, np.full((16, 16), 0.3), 4, inner_tol=1e-6, record=True)
    assert np.all(st.inner_counts == 1)
    np.testing.assert_array_equal(st.u, np.full((16, 16), 0.3))


def test_forced_counts_reproduce_fixed_and_adaptive_runs():
    """Forcing every count to K gives the fixed-K run bit for bit; forcing the counts an
    adaptive run recorded gives that run bit for bit."""
    f, _ = synth.rof_image(40, 36, 5, 0.05, 4)
    pr = oracle.Problem(40, 36, 3, 2, alpha=10.0, inner=30)
    a = oracle.dd_run(pr, f, 5)
    b = oracle.dd_run(pr, f, 5, counts=np.full((5, 6), 30))
    assert np.array_equal(a.u, b.u) and np.array_equal(a.P1, b.P1) and np.array_equal(a.lamh, b.lamh)
    c = oracle.dd_run(pr, f, 5, inner_tol=1e-3, record=True)
    d = oracle.dd_run(pr, f, 5, counts=c.inner_counts, record=True)
    assert np.array_equal(c.u, d.u) and np.array_equal(c.inner_counts, d.inner_counts)
    assert c.inner_counts.min() < 30  # the rule did stop some solves early


@pytest.mark.parametrize("n_outer", [1, 2, 3])
def test_locality_of_the_outer_iteration(n_outer):
    """Algorithm 1 starts from p~ = 0, lambda = 0, so the first local solves see only their
    own f, and each further outer iteration couples a subdomain to its side neighbours
    through lambda alone.  After n outer iterations a subdomain therefore depends on the
    subdomains fewer than n steps away, whose local problems depend on which of their own
    neighbours exist: the block of subdomains within n steps (clipped at the image border)
    reproduces the subdomain's u and p exactly.  (This is what makes sampled comparisons
    at sizes beyond the oracle's reach exact.)  The bound is sufficient, not always
    necessary: inside one local solve information moves about a pixel per inner
    iteration, so a smaller block can agree too.  The subdomain alone never does: its
    sides turn from interface dofs into pinned image-border edges."""
    T, m = 9, 8   # 9 x 9 subdomains of 8 x 8
    f, _ = synth.rof_image(T * m, T * m, 30, 0.1, 11)
    f = f.astype(np.float64)
    kw = dict(fidelity="l2", alpha=6.0, tau=50.0, inner=5)
    full = oracle.dd_run(oracle.Problem(T * m, T * m, T, T, **kw), f, n_outer)

    def block(a, b, rad):
        r0, r1, c0, c1 = max(0, a - rad), min(T, a + rad + 1), max(0, b - rad), min(T, b + rad + 1)
        st = oracle.dd_run(oracle.Problem((r1 - r0) * m, (c1 - c0) * m, r1 - r0, c1 - c0, **kw),
                           f[r0 * m:r1 * m, c0 * m:c1 * m], n_outer)
        u = st.u[(a - r0) * m:(a - r0 + 1) * m, (b - c0) * m:(b - c0 + 1) * m]
        p1 = st.P1[(a - r0) * (m + 1):(a - r0 + 1) * (m + 1), (b - c0) * m:(b - c0 + 1) * m]
        return u, p1

    for a, b in [(4, 4), (0, 0), (0, 4), (8, 3)]:
        u_ref = full.u[a * m:(a + 1) * m, b * m:(b + 1) * m]
        p_ref = full.P1[a * (m + 1):(a + 1) * (m + 1), b * m:(b + 1) * m]
        u, p1 = block(a, b, n_outer)
        assert np.array_equal(u, u_ref) and np.array_equal(p1, p_ref), (a, b)
        u_alone, _ = block(a, b, 0)
        assert np.abs(u_alone - u_ref).max() > 1e-3
