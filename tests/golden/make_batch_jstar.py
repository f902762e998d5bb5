"""Writes certified reference minima J* of the 64 images of the batched workload
(synth.batch_workload(64, 0)), using only the FP64 oracle.

ROF images: the oracle's accelerated full-dimension iteration (u strongly convex) runs
until the duality gap J(u) - d(p) <= rtol J(u).  Segmentation images (convex
Chan-Vese, Section 5.3): the oracle's plain full-dimension primal-dual iteration, with
the segmentation dual value d(p) = sum_T min(0, alpha g - div p), until the gap is
below rtol_seg |J(u)| (or the iteration cap, the gap reached being stored).  Weak
duality brackets d(p) <= J* <= J(u) for every image; the file stores both bounds, and
the relative energy error of a batch iterate, (J(u^n) - J*)/|J*| (eq. stop_outer), is
measured against the upper bound, exact to within the stored gap.

Usage: OMP_NUM_THREADS=6 python tests/golden/make_batch_jstar.py
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def certify_rof(f, alpha, rtol, check_every=250, max_iters=100000):
    H, W = f.shape
    pr = oracle.Problem(H, W, alpha=alpha)
    st = oracle.rof_accel_init(pr, f)
    st.steps[:] = [0.05, 1.0 / (8 * 0.05)]   # t0 s0 ||D||^2 <= 1
    best_J, best_D = np.inf, -np.inf
    while st.n < max_iters:
        oracle.rof_accel_run(pr, f, check_every, state=st)
        best_J = min(best_J, oracle.energy(pr, st.u, f))
        best_D = max(best_D, oracle.dual_value(pr, st.p1, st.p2, f))
        if best_J - best_D <= rtol * abs(best_J):
            break
    return best_J, best_D, st.n, "oracle.rof_accel_run (accelerated full-dimension primal-dual)"


def certify_seg(f, alpha, c1, c2, rtol, check_every=500, max_iters=60000):
    H, W = f.shape
    pr = oracle.Problem(H, W, fidelity="seg", alpha=alpha, c1=c1, c2=c2)
    st = oracle.cp_init(pr, f)
    best_J, best_D = np.inf, -np.inf
    while st.n < max_iters:
        oracle.cp_run(pr, f, check_every, state=st)
        best_J = min(best_J, oracle.energy(pr, st.u, f))
        best_D = max(best_D, oracle.dual_value(pr, st.p1, st.p2, f))
        if best_J - best_D <= rtol * abs(best_J):
            break
    return best_J, best_D, st.n, "oracle.cp_run (full-dimension primal-dual) with the segmentation dual value"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--rtol-seg", type=float, default=1e-5)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = a.out or os.path.join(HERE, f"jstar_batch{a.n}_seed{a.seed}.json")
    recs = []
    t0 = time.time()
    for i, m in enumerate(synth.batch_workload(a.n, a.seed)):
        f = m["f"].astype(np.float64)
        if m["fidelity"] == "l2":
            J, D, it, solver = certify_rof(f, m["alpha"], a.rtol)
        else:
            J, D, it, solver = certify_seg(f, m["alpha"], m["c1"], m["c2"], a.rtol_seg)
        recs.append(dict(index=i, height=m["height"], width=m["width"], fidelity=m["fidelity"], alpha=m["alpha"],
                         c1=m["c1"], c2=m["c2"], f_sha256=synth.array_digest(m["f"]), J_upper=J, D_lower=D,
                         J_star=J, rel_gap=(J - D) / abs(J), iterations=it, solver=solver))
        print(f"image {i} {m['height']}x{m['width']} {m['fidelity']}: J={J:.10g} gap/J={(J - D) / abs(J):.2e} "
              f"after {it} iterations ({time.time() - t0:.0f} s)", flush=True)
        with open(out, "w") as fh:
            json.dump(dict(workload=f"synth.batch_workload({a.n}, {a.seed})", images=recs), fh, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
