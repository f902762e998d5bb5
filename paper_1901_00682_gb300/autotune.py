"""Autotuner for the subdomain size and the inner-iteration count.

Both choices change the iterates of Algorithm 1 (more subdomains mean more interface
constraints to reconcile; more inner iterations solve each local problem more
exactly but cost more per outer iteration), so the tuner optimises what a user waits
for: the wall time until the relative energy error (J(u^n) - J*)/|J*| falls below a
tolerance (the outer stopping rule of Section 5), measured on the device for each
candidate (tile side, K, hardware variant).  J* is either given (a certified value)
or estimated as the lowest energy of a long run of the most accurate candidate.

Every candidate runs the same kernels as a normal solve, so the choice never changes
correctness, only speed; a tuned configuration is still checked against the oracle
by the parity tests at equal (tile, K).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

from . import _lib as L


@dataclass
class Trial:
    tile: int
    inner: int
    variant: int
    ms: float            # wall time of the solve to tolerance (ms), inf if not reached
    outer: int           # outer iterations run
    rel_err: float       # relative energy error at exit
    reached: bool


@dataclass
class TuneResult:
    best: Trial
    trials: list = field(default_factory=list)
    j_ref: float = math.nan
    tol: float = 0.0

    def table(self):
        return [dict(tile=t.tile, inner=t.inner, variant=t.variant, ms=t.ms, outer=t.outer, rel_err=t.rel_err,
                     reached=t.reached) for t in self.trials]


def candidates(height, width, tiles=(64, 128), inners=(5, 10, 20), variants=(0,)):
    """(tile, K, variant) triples whose tiles divide the image."""
    out = []
    for t in tiles:
        if height % t or width % t:
            continue
        for k in inners:
            for v in variants:
                out.append((t, k, v))
    return out


def pick_best(trials):
    """The reached trial with the least time; ties go to fewer outer iterations."""
    ok = [t for t in trials if t.reached and math.isfinite(t.ms)]
    if not ok:
        return min(trials, key=lambda t: (t.rel_err, t.ms)) if trials else None
    return min(ok, key=lambda t: (t.ms, t.outer))


def _params(height, width, tile, inner, variant, problem, **kw):
    return L.make_params(height, width, height // tile, width // tile, inner_iters=inner, variant=variant,
                         **problem, **kw)


def estimate_reference(f, problem, tile=128, inner=20, outer=2000, stream=None):
    """Lowest energy over a long run of one candidate (an upper bound of J*)."""
    H, W = f.shape
    s = L.Solver(_params(H, W, tile, inner, 0, problem), stream)
    s.load(f)
    best = math.inf
    step = max(outer // 20, 1)
    for _ in range(0, outer, step):
        s.iterate(step)
        best = min(best, s.current_energy())
    s.close()
    return best


def tune(f, problem, tol=1e-4, j_ref=None, tiles=(64, 128), inners=(5, 10, 20), variants=(0,),
         max_outer=3000, energy_every=5, stream=None, solve_fn=None):
    """Measures every candidate's time to tolerance on image f (a device tensor) and
    returns the fastest.  problem: dict of make_params keywords (fidelity, alpha, c1,
    c2, tau ...).  solve_fn(tile, inner, variant, j_ref) -> Trial replaces the GPU
    measurement (used by the host-side tests)."""
    H, W = f.shape
    if j_ref is None:
        j_ref = estimate_reference(f, problem, stream=stream)
    trials = []
    for tile, inner, variant in candidates(H, W, tiles, inners, variants):
        if solve_fn is not None:
            trials.append(solve_fn(tile, inner, variant, j_ref))
            continue
        p = _params(H, W, tile, inner, variant, problem, outer_iters=max_outer, outer_tol=tol, energy_ref=j_ref,
                    energy_every=energy_every)
        try:
            s = L.Solver(p, stream)
        except L.DDTVError:
            continue   # tile shape not supported by the fused path
        u = f.new_empty(f.shape)
        s.solve_device(f, None, u)            # warm-up: graph capture, caches
        t0 = time.perf_counter()
        _, st, rc = s.solve_device(f, None, u)
        ms = (time.perf_counter() - t0) * 1e3
        s.close()
        reached = bool(st.converged)
        trials.append(Trial(tile, inner, variant, ms if reached else math.inf, st.outer_done, st.rel_err, reached))
    best = pick_best(trials)
    return TuneResult(best, trials, j_ref, tol)


def batch_reference_energies(images, fs, inner=20, outer=2000, stream=None):
    """Lowest energy of every image of a batch over a long batched run (upper bounds
    of the images' J*, for batches without a certified reference).  images: dicts as for
    _lib.Batch; fs: device tensors."""
    b = L.Batch(images, inner_iters=inner, stream=stream)
    b.load(fs)
    best = [math.inf] * len(images)
    step = max(outer // 20, 1)
    for _ in range(0, outer, step):
        b.iterate(step)
        for i in range(len(images)):
            best[i] = min(best[i], b.energy(i))
    b.close()
    return best


def _batch_trial(images, fs, tile, inner, j_ref, tol, max_outer, check_every, stream):
    """Device time (CUDA events around the outer iterations only) until every image's
    relative energy error (J - J*)/|J*| is <= tol, checked every check_every outer
    iterations; the batch advances all images together."""
    import torch
    if any(im["height"] % tile or im["width"] % tile for im in images):
        return Trial(tile, inner, 0, math.inf, 0, math.inf, False)
    b = L.Batch(images, inner_iters=inner, stream=stream, tile=tile)
    st = torch.cuda.current_stream() if stream is None else stream
    b.load(fs)
    b.iterate(4)                      # warm-up: graph capture
    b.load(fs)
    done, ms, worst = 0, 0.0, math.inf
    while done < max_outer:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.iterate(check_every)
        e1.record(st)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        done += check_every
        worst = max((b.energy(i) - j_ref[i]) / abs(j_ref[i]) for i in range(len(images)))
        if worst <= tol:
            break
    b.close()
    reached = worst <= tol
    return Trial(tile, inner, 0, ms if reached else math.inf, done, worst, reached)


def tune_batch(images, fs, tol=1e-4, j_ref=None, inners=(5, 10, 20), tiles=(64, 128), max_outer=3000,
               check_every=10, stream=None, solve_fn=None):
    """Chooses the subdomain side and the inner-iteration count K of a batched solve by
    the measured device time until every image of the batch reaches relative energy
    error tol.  j_ref: per-image J* (certified values, or estimated by
    batch_reference_energies when None).  solve_fn(tile, inner, j_ref) -> Trial
    replaces the GPU measurement (host-side tests)."""
    if j_ref is None and solve_fn is None:
        j_ref = batch_reference_energies(images, fs, stream=stream)
    trials = []
    for tile in tiles:
        for inner in inners:
            if solve_fn is not None:
                trials.append(solve_fn(tile, inner, j_ref))
            else:
                trials.append(_batch_trial(images, fs, tile, inner, j_ref, tol, max_outer, check_every, stream))
    return TuneResult(pick_best(trials), trials, j_ref, tol)


def time_variants(f, problem, sub_rows, sub_cols, variants, inner=10, outer=100, warmup=8, stream=None):
    """Average device time of one outer iteration (CUDA-graph replay, CUDA events on
    the solver's stream) for each hardware mapping; f is a device tensor."""
    import torch
    H, W = f.shape
    out = {}
    for v in variants:
        p = L.make_params(H, W, sub_rows, sub_cols, inner_iters=inner, variant=v, **problem)
        s = L.Solver(p, stream)
        st = torch.cuda.current_stream() if stream is None else stream
        s.load(f)
        s.iterate(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.iterate(outer)
        e1.record(st)
        e1.synchronize()
        out[v] = e0.elapsed_time(e1) / outer
        s.close()
    return out


if __name__ == "__main__":
    # Times the fused hardware mappings on the 4096^2 ROF workload (32 x 32 subdomains
    # of 128^2, alpha 8, K = 10): python -m paper_1901_00682_gb300.autotune [v,v,...]
    import sys

    import torch

    import synth
    vs = [int(x) for x in sys.argv[1].split(",")] if len(sys.argv) > 1 else list(range(L.N_VARIANTS))
    img, _ = synth.rof_image(4096, 4096, 400, 0.1, 0)
    ms = time_variants(torch.from_numpy(img).cuda(), dict(fidelity="l2", alpha=8.0), 32, 32, vs)
    for v, t in ms.items():
        print(f"variant {v}: {t:.4f} ms per outer iteration ({4096 * 4096 * 10 / t / 1e3:.0f} Mpixel*iter/s)")
