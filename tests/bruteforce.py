"""Brute-force solvers of tiny instances of the model problem (eq. model, Section 3),
independent of the oracle: the finite-difference operator is assembled here as a
dense matrix from the definition (eq. FFD), and generic SciPy QP/LP solvers do the
minimisation.  Used only to pin the oracle.
"""
import numpy as np
from scipy.optimize import linprog, minimize


def fd_matrix(H, W):
    """Dense forward-difference operator D (eq. FFD), one row per interior edge:
    vertical neighbours first (u[i+1,j] - u[i,j]), then horizontal (u[i,j+1] - u[i,j])."""
    rows = []
    for i in range(H - 1):
        for j in range(W):
            r = np.zeros(H * W); r[(i + 1) * W + j] = 1.0; r[i * W + j] = -1.0; rows.append(r)
    for i in range(H):
        for j in range(W - 1):
            r = np.zeros(H * W); r[i * W + j + 1] = 1.0; r[i * W + j] = -1.0; rows.append(r)
    return np.array(rows).reshape(-1, H * W)


def rof(f, alpha):
    """min_u alpha/2 ||u - f||^2 + ||D u||_1 through its dual box QP
       min_{|q| <= 1} 1/(2 alpha) ||alpha f - D^T q||^2,  u = f - D^T q / alpha,
    solved by L-BFGS-B and polished on the free set by least squares."""
    H, W = f.shape
    D = fd_matrix(H, W)
    fv = f.ravel().astype(np.float64)
    n = D.shape[0]

    def obj(q):
        r = alpha * fv - D.T @ q
        return 0.5 / alpha * r @ r, -(D @ r) / alpha

    res = minimize(obj, np.zeros(n), jac=True, method="L-BFGS-B", bounds=[(-1, 1)] * n,
                   options={"maxiter": 100000, "ftol": 1e-16, "gtol": 1e-13, "maxcor": 50})
    q = res.x
    # Polish: with the bound-active set A fixed (q = +-1 there), the optimal D^T q is
    # the projection of alpha f - D_A^T q_A onto range(D_F^T); it is unique even where
    # q_F is not, and so is u.  The projected gradient of the L-BFGS-B point must be
    # small for A to be the right active set.
    grad = obj(q)[1]
    assert np.abs(q - np.clip(q - grad, -1, 1)).max() < 1e-6
    act = np.abs(q) > 1 - 1e-7
    qa = np.sign(q[act])
    rhs = alpha * fv - D[act].T @ qa
    free = ~act
    if free.any():
        sol, *_ = np.linalg.lstsq(D[free].T, rhs, rcond=None)
        dtq = D[act].T @ qa + D[free].T @ sol
    else:
        dtq = D[act].T @ qa
    u = fv - dtq / alpha
    return u.reshape(H, W)


def _lp_solve(c, A_ub, b_ub, bounds):
    r = linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs",
                options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert r.status == 0, r.message
    return r


def tvl1(f, alpha, mask=None):
    """min_u alpha sum_{T not in D} |u - f| + ||D u||_1 as an LP.  Returns (u, J*)."""
    H, W = f.shape
    D = fd_matrix(H, W)
    n, m = H * W, D.shape[0]
    fv = f.ravel().astype(np.float64)
    w = np.ones(n) if mask is None else (np.asarray(mask).ravel() == 0).astype(float)
    # variables [u (n), t (n), s (m)]
    c = np.concatenate([np.zeros(n), alpha * w, np.ones(m)])
    I, Z = np.eye(n), np.zeros((n, m))
    A = np.block([[I, -I, Z], [-I, -I, Z],
                  [D, np.zeros((m, n)), -np.eye(m)], [-D, np.zeros((m, n)), -np.eye(m)]])
    b = np.concatenate([fv, -fv, np.zeros(2 * m)])
    r = _lp_solve(c, A, b, [(None, None)] * n + [(0, None)] * (n + m))
    return r.x[:n].reshape(H, W), r.fun


def seg(f, alpha, c1, c2):
    """min_{0 <= u <= 1} alpha <u, g> + ||D u||_1, g = (f-c1)^2 - (f-c2)^2, as an LP."""
    H, W = f.shape
    D = fd_matrix(H, W)
    n, m = H * W, D.shape[0]
    fv = f.ravel().astype(np.float64)
    g = (fv - c1) ** 2 - (fv - c2) ** 2
    c = np.concatenate([alpha * g, np.ones(m)])
    A = np.block([[D, -np.eye(m)], [-D, -np.eye(m)]])
    r = _lp_solve(c, A, np.zeros(2 * m), [(0, 1)] * n + [(0, None)] * m)
    return r.x[:n].reshape(H, W), r.fun


def l2_inpaint(f, alpha, mask):
    """min_u alpha/2 sum_{T not in D} (u - f)^2 + ||D u||_1 by SLSQP on the smooth
    reformulation with s >= |D u|.  Returns (u, J*)."""
    H, W = f.shape
    D = fd_matrix(H, W)
    n, m = H * W, D.shape[0]
    fv = f.ravel().astype(np.float64)
    w = (np.asarray(mask).ravel() == 0).astype(float)

    def obj(x):
        u, s = x[:n], x[n:]
        r = w * (u - fv)
        return 0.5 * alpha * r @ r + s.sum(), np.concatenate([alpha * w * r, np.ones(m)])

    A = np.block([[-D, np.eye(m)], [D, np.eye(m)]])   # s - Du >= 0, s + Du >= 0
    cons = {"type": "ineq", "fun": lambda x: A @ x, "jac": lambda x: A}
    x0 = np.concatenate([fv, np.abs(D @ fv)])
    r = minimize(obj, x0, jac=True, constraints=[cons], method="SLSQP",
                 options={"maxiter": 2000, "ftol": 1e-15})
    u = r.x[:n]
    J = 0.5 * alpha * np.sum((w * (u - fv)) ** 2) + np.abs(D @ u).sum()
    return u.reshape(H, W), J
