"""Pins of the oracle's discrete operators (Section 2.3 and 2.4) against facts the
paper and the mathematics fix, independently of the oracle's own formulas:

* div is the outflow of the Raviart-Thomas normal components (dof orientation:
  down for horizontal edges, right for vertical edges), checked on unit vectors;
* D = -div^* (exact adjoint identity, global and on torn tiles);
* TV is the anisotropic finite-difference TV (Proposition on the FE/FD equivalence),
  checked on inputs with closed-form TV and through max_{p in C} <u, div p>;
* the jump operator B has B B^T = 2 I exactly, so ||B||^2 = 2 (Proposition on the
  norm of B), B^* is its transpose, and ker B is the image of the global space Y.
"""
import itertools

import numpy as np
import pytest

import oracle


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_div_unit_vectors_are_outflow():
    H, W = 4, 5
    # horizontal edge k (between rows k-1 and k), oriented downward
    for k in range(1, H):
        for j in range(W):
            p1 = np.zeros((H + 1, W)); p2 = np.zeros((H, W + 1))
            p1[k, j] = 1.0
            d = oracle.div(p1, p2)
            expect = np.zeros((H, W))
            expect[k - 1, j] = 1.0   # leaves pixel (k-1, j) through its bottom edge
            expect[k, j] = -1.0      # enters pixel (k, j) through its top edge
            assert np.array_equal(d, expect)
    # vertical edge l (between columns l-1 and l), oriented rightward
    for i in range(H):
        for l in range(1, W):
            p1 = np.zeros((H + 1, W)); p2 = np.zeros((H, W + 1))
            p2[i, l] = 1.0
            d = oracle.div(p1, p2)
            expect = np.zeros((H, W))
            expect[i, l - 1] = 1.0
            expect[i, l] = -1.0
            assert np.array_equal(d, expect)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 7), (5, 3), (8, 8)])
def test_global_adjoint_identity(H, W):
    u = _rand((H, W), 1)
    p1 = _rand((H + 1, W), 2); p2 = _rand((H, W + 1), 3)
    p1[0] = p1[-1] = 0.0; p2[:, 0] = p2[:, -1] = 0.0   # H_0(div): no boundary dofs
    g1, g2 = oracle.grad(u)
    lhs = np.sum(u * oracle.div(p1, p2))
    rhs = -(np.sum(g1 * p1) + np.sum(g2 * p2))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))
    # boundary entries of D u are not dofs
    assert not g1[0].any() and not g1[-1].any() and not g2[:, 0].any() and not g2[:, -1].any()


@pytest.mark.parametrize("sides", list(itertools.product([0, 1], repeat=4)))
def test_tile_adjoint_identity(sides):
    mr, mc = 4, 6
    top, bottom, left, right = sides
    u = _rand((mr, mc), 4)
    p1 = _rand((mr + 1, mc), 5); p2 = _rand((mr, mc + 1), 6)
    if not top: p1[0] = 0
    if not bottom: p1[-1] = 0
    if not left: p2[:, 0] = 0
    if not right: p2[:, -1] = 0
    g1, g2 = oracle.tile_grad(u, *sides)
    lhs = np.sum(u * oracle.tile_div(p1, p2))
    rhs = -(np.sum(g1 * p1) + np.sum(g2 * p2))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))
    # an active interface side sees only the inside pixel: D_s u = +u on top/left, -u on bottom/right
    if top: assert np.array_equal(g1[0], u[0])
    if bottom: assert np.array_equal(g1[-1], -u[-1])
    if left: assert np.array_equal(g2[:, 0], u[:, 0])
    if right: assert np.array_equal(g2[:, -1], -u[:, -1])


def test_tv_closed_forms():
    H, W = 6, 9
    ramp = np.repeat(np.arange(H, dtype=float)[:, None], W, axis=1)
    assert oracle.tv(ramp) == (H - 1) * W
    checker = (-1.0) ** np.add.outer(np.arange(H), np.arange(W))
    assert oracle.tv(checker) == 2 * ((H - 1) * W + H * (W - 1))
    assert oracle.tv(np.full((H, W), 0.3)) == 0.0


def test_tv_is_max_over_box_of_u_div_p():
    # TV(u) = max_{p in C} <u, div p> = max -<D u, p>, attained at p = -sign(D u)
    u = _rand((7, 5), 7)
    g1, g2 = oracle.grad(u)
    val = np.sum(u * oracle.div(-np.sign(g1), -np.sign(g2)))
    assert abs(val - oracle.tv(u)) <= 1e-12 * oracle.tv(u)
    # and no other point of C does better
    rng = np.random.default_rng(0)
    for _ in range(20):
        q1 = rng.uniform(-1, 1, g1.shape); q2 = rng.uniform(-1, 1, g2.shape)
        q1[0] = q1[-1] = 0; q2[:, 0] = q2[:, -1] = 0
        assert np.sum(u * oracle.div(q1, q2)) <= oracle.tv(u) + 1e-12


def _torn_sizes(pr):
    return (pr.H + pr.NR) * pr.W, pr.H * (pr.W + pr.NC)


def _assemble_B(pr):
    n1, n2 = _torn_sizes(pr)
    cols = []
    for k in range(n1 + n2):
        P1 = np.zeros(n1); P2 = np.zeros(n2)
        if k < n1: P1[k] = 1.0
        else: P2[k - n1] = 1.0
        jh, jv = oracle.jump(pr, P1.reshape(pr.H + pr.NR, pr.W), P2.reshape(pr.H, pr.W + pr.NC))
        cols.append(np.concatenate([jh.ravel(), jv.ravel()]))
    return np.array(cols).T


@pytest.mark.parametrize("H,W,NR,NC", [(4, 6, 2, 3), (5, 7, 2, 2), (3, 3, 3, 3), (1, 2, 1, 2), (6, 4, 3, 1)])
def test_jump_operator(H, W, NR, NC):
    pr = oracle.Problem(H, W, NR, NC)
    B = _assemble_B(pr)
    n_gamma = (NR - 1) * W + (NC - 1) * H
    assert B.shape[0] == n_gamma
    # every row has one +1 (s side) and one -1 (t side): B B^T = 2 I exactly
    assert np.array_equal(B @ B.T, 2.0 * np.eye(n_gamma))
    if n_gamma:
        assert abs(np.linalg.norm(B, 2) ** 2 - 2.0) < 1e-12
    # B^* is the transpose
    rng = np.random.default_rng(1)
    lamh = rng.standard_normal((NR - 1, W)); lamv = rng.standard_normal((NC - 1, H))
    P1, P2 = oracle.jump_adjoint(pr, lamh, lamv)
    lam = np.concatenate([lamh.ravel(), lamv.ravel()])
    assert np.allclose(np.concatenate([P1.ravel(), P2.ravel()]), B.T @ lam, atol=0, rtol=0)
    # a global field of Y, torn by duplication, has no jump (Y ~ ker B)
    p1 = rng.standard_normal((H + 1, W)); p2 = rng.standard_normal((H, W + 1))
    p1[0] = p1[-1] = 0; p2[:, 0] = p2[:, -1] = 0
    T1, T2 = oracle.global_to_torn(pr, p1, p2)
    jh, jv = oracle.jump(pr, T1, T2)
    assert not jh.any() and not jv.any()
    g1, g2 = oracle.torn_to_global(pr, T1, T2)
    assert np.array_equal(g1, p1) and np.array_equal(g2, p2)


def test_torn_divergence_matches_global_on_ker_B():
    # for p~ in ker B, the tile-wise divergence equals the global one (div~ p~ = div p)
    pr = oracle.Problem(6, 8, 2, 2)
    rng = np.random.default_rng(3)
    p1 = rng.standard_normal((7, 8)); p2 = rng.standard_normal((6, 9))
    p1[0] = p1[-1] = 0; p2[:, 0] = p2[:, -1] = 0
    T1, T2 = oracle.global_to_torn(pr, p1, p2)
    d = oracle.div(p1, p2)
    for a in range(2):
        for b in range(2):
            r0, c0 = 3 * a, 4 * b
            loc1 = T1[r0 + a:r0 + a + 4, c0:c0 + 4]
            loc2 = T2[r0:r0 + 3, c0 + b:c0 + b + 5]
            assert np.allclose(oracle.tile_div(loc1, loc2), d[r0:r0 + 3, c0:c0 + 4], atol=1e-15)
