"""Pins of the oracle's trajectory, not only of its fixed point.

The fixed-point pins (brute-force minimisers, closed forms, DD = single domain) would
also pass an oracle whose step sizes, extrapolations or multiplier update were wrong
but still convergent.  These tests check the iterates themselves against convergence
results whose statements depend on the exact schedule of the two nested iterations:

* Local solver (Section 5: the accelerated primal-dual algorithm of Chambolle and Pock,
  2011, Algorithm 2, with the dual field p as the uniformly convex variable: K = div_s,
  G(p) = chi_C(p) + 1/(2 tau) ||p - phat||^2, F^* = alpha F).  The proof of their
  Theorem 2 bounds, for every N, with tau_0 sigma_0 ||div_s||^2 <= 1 and gamma at most
  the convexity modulus 1/tau of G,
      ||p_N - p*||^2 <= tau_N^2 (||p* - p_0||^2 / tau_0^2 + ||u* - u_0||^2 / (tau_0 sigma_0)),
  tau_N the step after N accelerated updates, and it does so through a Lyapunov function
      Psi_n = ||p* - p_n||^2 / tau_n^2 + ||u* - u_n||^2 / (tau_0 sigma_0)
              + ||p_n - p_{n-1}||^2 / tau_{n-1}^2 + (2 / tau_{n-1}) <div (p_n - p_{n-1}), u_n - u*>
  that never increases.
* Outer iteration (Algorithm 1 is the primal-dual algorithm with theta = 1 applied to
  the torn saddle problem eq. DD: x = p~, y = lambda, K = B, ||B||^2 = 2, tau sigma =
  1/2).  The ergodic bound of the paper's theorem on Algorithm 1, in the sharper form of
  Chambolle and Pock (2011), Theorem 1:
      L(p~_n, lambda) - L(p~, lambda_n) <= (||p~ - p~^0||^2 / (2 tau) + ||lambda - lambda^0||^2 / (2 sigma)) / n
  for every (p~, lambda), with the averages p~_n, lambda_n of the iterates 1..n; and the
  Lyapunov function of the same proof at a saddle point,
      Psi_n = ||p~* - p~^n||^2 / tau + ||lambda* - lambda^n||^2 / sigma
              + ||p~^n - p~^{n-1}||^2 / tau + 2 <B (p~^n - p~^{n-1}), lambda^n - lambda*>,
  never increases.
The saddle points come from brute-force QPs written here from the definitions
(tests/bruteforce.py), never from the oracle.  The last tests plant mistakes in copies
of the oracle and check that each one breaks at least one of these pins.
"""
import numpy as np
import pytest

import oracle
from bruteforce import box_qp, rof_dual, tile_div_matrix

TAU0, SIGMA0 = 10.0, 1.0 / 80.0


# ------------------------------------------------------------ local solver (Section 5)

class LocalInstance:
    """One interior ROF tile (every side on the interface) with a fixed proximal
    centre: the local saddle problem eq. local, its exact solution by brute force, and
    the oracle's iterates from (u_0, p_0)."""

    def __init__(self, m, alpha, tau, gamma, seed, p0_scale=0.0, u0_random=False):
        rng = np.random.default_rng(seed)
        self.m, self.alpha, self.tau, self.gamma = m, alpha, tau, gamma
        self.n1 = (m + 1) * m
        self.f = rng.uniform(0.0, 1.0, (m, m))
        n = 2 * self.n1
        self.ph = rng.uniform(-1.5, 1.5, n)
        self.p0 = rng.uniform(-1.0, 1.0, n) * p0_scale
        self.u0 = rng.uniform(-1.0, 2.0, (m, m)) if u0_random else self.f.copy()
        self.D, act = tile_div_matrix(m, m)
        assert act.all()
        # local dual: min_{|p| <= 1} (alpha F)^*(div p) + 1/(2 tau) ||p - phat||^2 with
        # (alpha F)^*(w) = <f, w> + ||w||^2 / (2 alpha) for F = 1/2 ||u - f||^2
        fv = self.f.ravel()
        Q = self.D.T @ self.D / alpha + np.eye(n) / tau
        b = self.D.T @ fv - self.ph / tau
        self.p_star, _, kkt = box_qp(Q, b)
        assert kkt < 1e-12
        # primal part of the saddle point: u* = argmin alpha F(u) - <u, div p*>
        self.u_star = fv + self.D @ self.p_star / alpha
        self.L2 = np.linalg.norm(self.D, 2) ** 2

    def problem(self, gamma=None):
        g = self.gamma if gamma is None else gamma
        return oracle.Problem(self.m, self.m, fidelity="l2", alpha=self.alpha, tau=self.tau, tau0=TAU0,
                              sigma0=SIGMA0, gamma=g)

    def iterate(self, N, gamma=None):
        """(p_N, u_N) of the oracle's local solve run for N inner iterations."""
        m, n1 = self.m, self.n1
        u = self.u0.copy()
        p1 = self.p0[:n1].reshape(m + 1, m).copy()
        p2 = self.p0[n1:].reshape(m, m + 1).copy()
        oracle.local_solve(self.problem(gamma), self.f, u, p1, p2, self.ph[:n1].reshape(m + 1, m),
                           self.ph[n1:].reshape(m, m + 1), N)
        return np.concatenate([p1.ravel(), p2.ravel()]), u.ravel()

    def taus(self, N):
        """tau_0 .. tau_N of the accelerated schedule (Chambolle-Pock Algorithm 2)."""
        t = [TAU0]
        for _ in range(N):
            t.append(t[-1] / np.sqrt(1.0 + 2.0 * self.gamma * t[-1]))
        return np.array(t)

    def delta0(self):
        return (np.sum((self.p_star - self.p0) ** 2) / TAU0 ** 2 +
                np.sum((self.u_star - self.u0.ravel()) ** 2) / (TAU0 * SIGMA0))


def _rate_ratios(inst, Ns, gamma_oracle=None):
    """||p_N - p*||^2 / (tau_N^2 Delta_0) for each N."""
    taus = inst.taus(max(Ns))
    d0 = inst.delta0()
    out = []
    for N in Ns:
        p, _ = inst.iterate(N, gamma_oracle)
        out.append(np.sum((p - inst.p_star) ** 2) / (taus[N] ** 2 * d0))
    return np.array(out)


def _lyapunov(inst, K):
    """Psi_0 .. Psi_K along the oracle's iterates."""
    taus = inst.taus(K)
    P = [inst.p0]
    U = [inst.u0.ravel()]
    for N in range(1, K + 1):
        p, u = inst.iterate(N)
        P.append(p)
        U.append(u)
    psi = []
    for n in range(K + 1):
        v = np.sum((inst.p_star - P[n]) ** 2) / taus[n] ** 2 + np.sum((inst.u_star - U[n]) ** 2) / (TAU0 * SIGMA0)
        if n >= 1:
            dp = P[n] - P[n - 1]
            v += dp @ dp / taus[n - 1] ** 2 + 2.0 / taus[n - 1] * (inst.D @ dp) @ (U[n] - inst.u_star)
        psi.append(v)
    return np.array(psi)


RATE_NS = list(range(1, 41)) + list(range(50, 2001, 50))

# strong: gamma = 1/tau, the largest modulus the local problem allows, so the bound is
# tight enough to need the acceleration; paper: Section 5's tau = 50, gamma = 1/(8 tau)
STRONG = dict(m=8, alpha=0.05, tau=1.0, gamma=1.0, seed=3)
PAPER = dict(m=8, alpha=10.0, tau=50.0, gamma=1.0 / 400.0, seed=3)
# a start away from the solution, weak fidelity: the instance on which the Lyapunov
# function separates the extrapolation of p from its absence
LYAP = dict(m=6, alpha=0.0104, tau=1.4, gamma=1.0 / 1.4, seed=17, p0_scale=1.0, u0_random=True)


@pytest.mark.parametrize("prm", [STRONG, PAPER], ids=["gamma=1/tau", "paper"])
def test_local_solver_meets_the_accelerated_rate(prm):
    """The oracle's local iterates satisfy the O(1/N^2) bound of Chambolle-Pock's
    Algorithm 2 for N = 1..2000 (tau_0 sigma_0 ||div_s||^2 <= 1 holds: ||div_s||^2 < 8)."""
    inst = LocalInstance(**prm)
    assert TAU0 * SIGMA0 * inst.L2 <= 1.0
    r = _rate_ratios(inst, RATE_NS)
    assert r.max() <= 1.0, (r.max(), RATE_NS[int(r.argmax())])


def test_unaccelerated_local_iteration_misses_the_rate():
    """With gamma = 0 the same code runs theta = 1 and constant steps (the plain
    primal-dual iteration); on the gamma = 1/tau instance it breaks the accelerated
    bound within a few iterations, so the bound does tell the schedules apart."""
    inst = LocalInstance(**STRONG)
    r = _rate_ratios(inst, list(range(1, 21)), gamma_oracle=0.0)
    assert r.max() > 10.0


@pytest.mark.parametrize("prm", [STRONG, LYAP], ids=["gamma=1/tau", "far-start"])
def test_local_solver_lyapunov_function_decreases(prm):
    inst = LocalInstance(**prm)
    psi = _lyapunov(inst, 120)
    inc = (psi[1:] - psi[:-1]) / np.abs(psi[:-1])
    assert inc.max() <= 1e-12, (inc.max(), int(inc.argmax()))
    assert psi[-1] < 0.1 * psi[0]


# ------------------------------------------------------------ outer iteration (Algorithm 1)

OUTER = dict(H=12, W=12, NR=2, NC=2, alpha=2.0, seed=1, inner=3000)


def _outer_problem(H, W, NR, NC, alpha, seed, inner):
    f = np.random.default_rng(seed).uniform(0.0, 1.0, (H, W))
    return oracle.Problem(H, W, NR, NC, fidelity="l2", alpha=alpha, inner=inner), f


def _tiles(pr):
    for a in range(pr.NR):
        for b in range(pr.NC):
            r0, r1 = oracle.part_start(a, pr.H, pr.NR), oracle.part_start(a + 1, pr.H, pr.NR)
            c0, c1 = oracle.part_start(b, pr.W, pr.NC), oracle.part_start(b + 1, pr.W, pr.NC)
            yield a, b, r0, r1, c0, c1


def _tile_dofs(P1, P2, a, b, r0, r1, c0, c1):
    """One tile's dofs from the torn arrays, ordered as tile_div_matrix's columns."""
    return np.concatenate([P1[r0 + a:r1 + a + 1, c0:c1].ravel(), P2[r0:r1, c0 + b:c1 + b + 1].ravel()])


def _sup_gap(pr, f, P1, P2, lamh, lamv, n):
    """sup over (p~ in C~, lambda) of  L(p~_n, lambda) - L(p~, lambda_n)
    - (||p~||^2 / (2 tau) + ||lambda||^2 / (2 sigma)) / n  for averages (P1, P2, lamh,
    lamv) = (p~_n, lambda_n) and p~^0 = 0, lambda^0 = 0, where
    L(p~, lambda) = sum_s [(alpha F_s)^*(div p~_s) + chi_C(p~_s)] + <B p~, lambda>.
    The lambda part is (n sigma / 2) ||B p~_n||^2; the p~ part splits into one box QP
    per tile."""
    sigma = pr.c().sigma
    jh, jv = oracle.jump(pr, P1, P2)
    val = 0.5 * n * sigma * (np.sum(jh ** 2) + np.sum(jv ** 2))
    Bl1, Bl2 = oracle.jump_adjoint(pr, lamh, lamv)
    for a, b, r0, r1, c0, c1 in _tiles(pr):
        D, act = tile_div_matrix(r1 - r0, c1 - c0, a > 0, a + 1 < pr.NR, b > 0, b + 1 < pr.NC)
        fv = f[r0:r1, c0:c1].ravel()
        d = D @ _tile_dofs(P1, P2, a, b, r0, r1, c0, c1)[act]
        val += d @ d / (2 * pr.alpha) + fv @ d                 # (alpha F)^*(div p~_n) on the tile
        c = _tile_dofs(Bl1, Bl2, a, b, r0, r1, c0, c1)[act]    # B^* lambda_n on the tile
        Q = D.T @ D / pr.alpha + np.eye(D.shape[1]) / (n * pr.tau)
        _, m, kkt = box_qp(Q, D.T @ fv + c)
        assert kkt < 1e-10
        val -= m
    return val


def _outer_ergodic_gaps(pr, f, N, check):
    st = oracle.dd_init(pr, f)
    S = [np.zeros_like(st.P1), np.zeros_like(st.P2), np.zeros_like(st.lamh), np.zeros_like(st.lamv)]
    out = []
    for n in range(1, N + 1):
        oracle.dd_run(pr, f, 1, state=st)
        for s, v in zip(S, (st.P1, st.P2, st.lamh, st.lamv)):
            s += v
        if n in check:
            out.append(_sup_gap(pr, f, *(s / n for s in S), n))
    return np.array(out)


def _saddle_point(pr, f):
    """A saddle point of eq. DD: p~* the torn copy of a brute-force ROF dual solution
    (the proposition on the equivalence of eq. DD with the dual model problem), and
    lambda*_e = -(u*_s + u*_t) / 2 from the two pixels beside edge e (the optimality
    condition of the torn Lagrangian in p~: -u* where u* is continuous across e, and
    inside [-u*_t, -u*_s] where |p*_e| = 1)."""
    p1, p2, u, kkt = rof_dual(f, pr.alpha)
    assert kkt < 1e-10
    P1, P2 = oracle.global_to_torn(pr, p1, p2)
    lamh = np.zeros((pr.NR - 1, pr.W))
    lamv = np.zeros((pr.NC - 1, pr.H))
    for a in range(pr.NR - 1):
        r = oracle.part_start(a + 1, pr.H, pr.NR)
        lamh[a] = -0.5 * (u[r - 1] + u[r])
    for b in range(pr.NC - 1):
        c = oracle.part_start(b + 1, pr.W, pr.NC)
        lamv[b] = -0.5 * (u[:, c - 1] + u[:, c])
    return P1, P2, lamh, lamv


def _outer_lyapunov(pr, f, N):
    P1s, P2s, lhs, lvs = _saddle_point(pr, f)
    tau, sigma = pr.tau, pr.c().sigma
    xs = np.concatenate([P1s.ravel(), P2s.ravel()])
    ys = np.concatenate([lhs.ravel(), lvs.ravel()])
    st = oracle.dd_init(pr, f)
    x_old = np.concatenate([st.P1.ravel(), st.P2.ravel()])
    y = np.concatenate([st.lamh.ravel(), st.lamv.ravel()])
    psi = [np.sum((xs - x_old) ** 2) / tau + np.sum((ys - y) ** 2) / sigma]
    n1 = st.P1.size
    for _ in range(N):
        oracle.dd_run(pr, f, 1, state=st)
        x = np.concatenate([st.P1.ravel(), st.P2.ravel()])
        y = np.concatenate([st.lamh.ravel(), st.lamv.ravel()])
        dx = x - x_old
        jh, jv = oracle.jump(pr, dx[:n1].reshape(st.P1.shape), dx[n1:].reshape(st.P2.shape))
        Bdx = np.concatenate([jh.ravel(), jv.ravel()])
        psi.append(np.sum((xs - x) ** 2) / tau + np.sum((ys - y) ** 2) / sigma + dx @ dx / tau +
                   2.0 * Bdx @ (y - ys))
        x_old = x
    return np.array(psi)


ERGODIC_NS = {1, 2, 3, 4, 5, 6, 8, 10, 15, 20, 30, 40}


def test_saddle_point_is_a_fixed_point_of_algorithm_1():
    """The brute-force (p~*, lambda*) used below: B p~* = 0 and one outer iteration of
    the oracle started there leaves it in place (exact local solves)."""
    pr, f = _outer_problem(**OUTER)
    P1, P2, lamh, lamv = _saddle_point(pr, f)
    jh, jv = oracle.jump(pr, P1, P2)
    assert np.abs(jh).max() < 1e-12 and np.abs(jv).max() < 1e-12
    st = oracle.dd_init(pr, f)
    st.P1[:], st.P2[:], st.P1prev[:], st.P2prev[:] = P1, P2, P1, P2
    st.lamh[:], st.lamv[:] = lamh, lamv
    st.u[:] = f + oracle.div(*rof_dual(f, pr.alpha)[:2]) / pr.alpha
    oracle.dd_run(pr, f, 1, state=st)
    assert np.abs(st.P1 - P1).max() < 1e-9 and np.abs(st.P2 - P2).max() < 1e-9
    assert np.abs(st.lamh - lamh).max() < 1e-12 and np.abs(st.lamv - lamv).max() < 1e-12


def test_outer_iteration_meets_the_ergodic_bound():
    pr, f = _outer_problem(**OUTER)
    g = _outer_ergodic_gaps(pr, f, 40, ERGODIC_NS)
    assert g.max() <= 0.0, g


def test_outer_lyapunov_function_decreases():
    pr, f = _outer_problem(**OUTER)
    psi = _outer_lyapunov(pr, f, 40)
    inc = (psi[1:] - psi[:-1]) / psi[:-1]
    assert inc.max() <= 1e-12, (inc.max(), int(inc.argmax()))


# ------------------------------------------------------------ planted mistakes

# (name, [(text in dd_tv_oracle.c, replacement)], which pins)
LOCAL_MUTANTS = [
    ("theta without the factor 2", [("sqrt(1.0 + 2.0 * pr->gamma * tk)", "sqrt(1.0 + pr->gamma * tk)")]),
    ("sigma_k multiplied by theta", [("    sk = sk / theta;\n    done", "    sk = sk * theta;\n    done")]),
    ("tau_k divided by theta", [("    tk = theta * tk;\n    sk = sk / theta;\n    done",
                                 "    tk = tk / theta;\n    sk = sk / theta;\n    done")]),
    ("no extrapolation of p", [("pb1[e] = pn + theta * (pn - p1[e]);", "pb1[e] = pn;"),
                               ("pb2[e] = pn + theta * (pn - p2[e]);", "pb2[e] = pn;")]),
    ("no extrapolation of p1", [("pb1[e] = pn + theta * (pn - p1[e]);", "pb1[e] = pn;")]),
    ("extrapolation with the wrong sign", [("pb1[e] = pn + theta * (pn - p1[e]);", "pb1[e] = pn - theta * (pn - p1[e]);"),
                                           ("pb2[e] = pn + theta * (pn - p2[e]);", "pb2[e] = pn - theta * (pn - p2[e]);")]),
]

OUTER_MUTANTS = [
    ("no extrapolation in the multiplier update",
     [("lamh[e] += pr->sigma * (2.0 * jh[e] - jh_prev[e]);", "lamh[e] += pr->sigma * jh[e];"),
      ("lamv[e] += pr->sigma * (2.0 * jv[e] - jv_prev[e]);", "lamv[e] += pr->sigma * jv[e];")]),
    ("previous iterate never updated",
     [("    memcpy(P1prev, P1, sizeof(double) * n1);\n    memcpy(P2prev, P2, sizeof(double) * n2);\n", "")]),
    ("proximal centre with the wrong sign",
     [("Ph1[e] = P1[e] - pr->tau * Ph1[e];", "Ph1[e] = P1[e] + pr->tau * Ph1[e];"),
      ("Ph2[e] = P2[e] - pr->tau * Ph2[e];", "Ph2[e] = P2[e] + pr->tau * Ph2[e];")]),
    ("sigma doubled", [("lamh[e] += pr->sigma * (2.0", "lamh[e] += 2.0 * pr->sigma * (2.0"),
                       ("lamv[e] += pr->sigma * (2.0", "lamv[e] += 2.0 * pr->sigma * (2.0")]),
    ("jump with s and t exchanged", [("jh[a * W + j] = P1[rs * W + j] - P1[rt * W + j];",
                                      "jh[a * W + j] = P1[rt * W + j] - P1[rs * W + j];")]),
]


def _mutant(tmp_path, edits):
    src = oracle.source()
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    return oracle.build_variant(src, str(tmp_path))


def _local_pins_hold():
    try:
        inst = LocalInstance(**STRONG)
        if _rate_ratios(inst, RATE_NS[::3]).max() > 1.0:
            return False
        for prm in (STRONG, LYAP):
            psi = _lyapunov(LocalInstance(**prm), 120)
            if not np.all(np.isfinite(psi)) or ((psi[1:] - psi[:-1]) / np.abs(psi[:-1])).max() > 1e-12:
                return False
    except (FloatingPointError, AssertionError):
        return False
    return True


def _outer_pins_hold():
    pr, f = _outer_problem(**OUTER)
    if _outer_ergodic_gaps(pr, f, 40, ERGODIC_NS).max() > 0.0:
        return False
    psi = _outer_lyapunov(pr, f, 40)
    return ((psi[1:] - psi[:-1]) / psi[:-1]).max() <= 1e-12


@pytest.mark.parametrize("name,edits", LOCAL_MUTANTS, ids=[m[0] for m in LOCAL_MUTANTS])
def test_planted_local_schedule_mistake_is_caught(tmp_path, name, edits):
    with oracle.using_library(_mutant(tmp_path, edits)):
        with np.errstate(all="ignore"):
            assert not _local_pins_hold(), name


@pytest.mark.parametrize("name,edits", OUTER_MUTANTS, ids=[m[0] for m in OUTER_MUTANTS])
def test_planted_outer_iteration_mistake_is_caught(tmp_path, name, edits):
    with oracle.using_library(_mutant(tmp_path, edits)):
        assert not _outer_pins_hold(), name


def test_unmodified_copy_passes_every_pin(tmp_path):
    """The mutation harness itself: a copy of the unchanged source passes."""
    with oracle.using_library(_mutant(tmp_path, [])):
        assert _local_pins_hold() and _outer_pins_hold()
