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


def tile_div_matrix(mr, mc, top=True, bottom=True, left=True, right=True):
    """Dense div_s of one mr x mc tile (outflow: bottom - top + right - left, Section
    2.3) on its dual dofs, written from the definition: columns are p1 ((mr+1) x mc,
    edge k above row k) then p2 (mr x (mc+1), edge l left of column l), row-major.
    Returns (D, active): D keeps only the columns of active dofs (a side on the image
    boundary is not a dof); active is the boolean mask over all dofs."""
    n1, n2 = (mr + 1) * mc, mr * (mc + 1)
    D = np.zeros((mr * mc, n1 + n2))
    for i in range(mr):
        for j in range(mc):
            q = i * mc + j
            D[q, (i + 1) * mc + j] += 1.0
            D[q, i * mc + j] -= 1.0
            D[q, n1 + i * (mc + 1) + j + 1] += 1.0
            D[q, n1 + i * (mc + 1) + j] -= 1.0
    act = np.ones(n1 + n2, dtype=bool)
    act[:mc] = top
    act[mr * mc:n1] = bottom
    act[n1::mc + 1] = left
    act[n1 + mc::mc + 1] = right
    return D[:, act], act


def box_qp(Q, b, x0=None):
    """argmin_{|x_i| <= 1} 1/2 x^T Q x + b^T x for a positive semidefinite Q: L-BFGS-B,
    then the free variables solved exactly with the active set fixed.  Returns
    (x, value, kkt) where kkt is the largest violation of the projected-gradient
    optimality condition x = proj(x - grad)."""
    n = len(b)
    obj = lambda x: (0.5 * x @ Q @ x + b @ x, Q @ x + b)
    kkt_of = lambda x: float(np.abs(x - np.clip(x - (Q @ x + b), -1, 1)).max())
    x = np.zeros(n) if x0 is None else np.clip(x0, -1, 1)
    best = (np.inf, x)
    for _ in range(5):   # L-BFGS-B, then an exact solve on the free set; restart if needed
        r = minimize(obj, x, jac=True, method="L-BFGS-B", bounds=[(-1, 1)] * n,
                     options={"maxiter": 100000, "ftol": 1e-16, "gtol": 1e-14, "maxcor": 50})
        x = r.x
        for _ in range(10):
            g = Q @ x + b
            act = ((x <= -1 + 1e-9) & (g > 0)) | ((x >= 1 - 1e-9) & (g < 0))
            y = np.where(act, np.sign(x), x)
            fr = ~act
            if fr.any():
                sol, *_ = np.linalg.lstsq(Q[np.ix_(fr, fr)], -(b[fr] + Q[np.ix_(fr, act)] @ y[act]), rcond=None)
                y[fr] = sol
            x = np.clip(y, -1, 1)
        k = kkt_of(x)
        if k < best[0]:
            best = (k, x)
        if k < 1e-12:
            break
    k, x = best
    return x, float(obj(x)[0]), k


def rof_dual(f, alpha):
    """A solution p of the ROF dual  min_{|p| <= 1} 1/(2 alpha) ||div p + alpha f||^2
    (global field: p1 (H+1) x W, p2 H x (W+1), zero on the image boundary) and the
    primal solution u = f + div p / alpha.  Returns (p1, p2, u, kkt)."""
    H, W = f.shape
    D = fd_matrix(H, W)          # D = -div^T on the interior edges
    fv = f.ravel().astype(np.float64)
    q, _, kkt = box_qp(D @ D.T / alpha, -(D @ fv))
    u = fv - D.T @ q / alpha
    nv = (H - 1) * W
    p1 = np.zeros((H + 1, W))
    p1[1:H] = q[:nv].reshape(H - 1, W)
    p2 = np.zeros((H, W + 1))
    p2[:, 1:W] = q[nv:].reshape(H, W - 1)
    return p1, p2, u.reshape(H, W), kkt
