"""Writes certified reference minima J* of the ROF benchmark images, using only the
FP64 oracle.

J* is the minimum of J(u) = alpha/2 ||u - f||^2 + TV(u) (eq. model with the L2
fidelity).  The oracle's accelerated full-dimension iteration (u strongly convex)
runs until the duality gap J(u) - d(p) <= rtol * J(u); weak duality then brackets
d(p) <= J* <= J(u), and the file stores both bounds.  The relative energy error of
an iterate, (J(u^n) - J*)/J* (eq. stop_outer), is measured against J(u) of the
certificate, so it is exact to within the stored relative gap.

Usage: python tests/golden/make_jstar.py [--size 4096] [--rtol 1e-6]
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


def certify(H, W, shapes, sigma, alpha, seed, rtol, check_every=250, max_iters=200000, log=print):
    f32, _ = synth.rof_image(H, W, shapes, sigma, seed)
    f = f32.astype(np.float64)
    pr = oracle.Problem(H, W, alpha=alpha)
    st = oracle.rof_accel_init(pr, f)
    st.steps[:] = [0.05, 1.0 / (8 * 0.05)]   # t0 s0 ||D||^2 <= 1
    t0 = time.time()
    best = None
    while st.n < max_iters:
        oracle.rof_accel_run(pr, f, check_every, state=st)
        J = oracle.energy(pr, st.u, f)
        D = oracle.dual_value(pr, st.p1, st.p2, f)
        gap = (J - D) / J
        if best is None or J < best[0]:
            best = (J, D)
        log(f"{H}x{W} iter {st.n}: J={J:.10f} d={D:.10f} gap/J={gap:.3e} ({time.time() - t0:.0f}s)")
        if gap <= rtol:
            break
    return dict(height=H, width=W, n_shapes=shapes, noise_sigma=sigma, alpha=alpha, seed=seed,
                f_sha256=synth.array_digest(f32), J_upper=J, D_lower=D, J_star=J, rel_gap=(J - D) / J,
                iterations=st.n, solver="oracle.rof_accel_run (accelerated full-dimension primal-dual)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--shapes", type=int, default=400)
    ap.add_argument("--sigma", type=float, default=0.1)
    ap.add_argument("--alpha", type=float, default=8.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    rec = certify(a.size, a.size, a.shapes, a.sigma, a.alpha, a.seed, a.rtol,
                  log=lambda s: print(s, flush=True))
    out = a.out or os.path.join(HERE, f"jstar_rof{a.size}_seed{a.seed}.json")
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
