"""Host logic of the autotuner (candidate set, choice by time to tolerance) without a
GPU, and on the GPU a tuning run whose chosen configuration reaches the tolerance."""
import math

import numpy as np
import pytest

from paper_1901_00682_gb300 import autotune as at


def test_candidates_respect_divisibility():
    c = at.candidates(384, 256, tiles=(64, 128), inners=(5, 10), variants=(0, 1))
    assert (128, 5, 0) in c and (64, 10, 1) in c
    c2 = at.candidates(192, 256, tiles=(64, 128), inners=(10,))
    assert all(t == 64 for t, _, _ in c2)
    assert len(at.candidates(384, 256, tiles=(64, 128), inners=(5, 10), variants=(0, 1))) == 8


def test_pick_best_prefers_reached_then_fastest():
    T = at.Trial
    trials = [T(128, 5, 0, math.inf, 3000, 2e-4, False), T(128, 10, 0, 50.0, 200, 9e-5, True),
              T(64, 10, 0, 40.0, 300, 9.9e-5, True), T(64, 20, 0, 40.0, 250, 9e-5, True)]
    best = at.pick_best(trials)
    assert (best.tile, best.inner) == (64, 20)       # equal time: fewer outer iterations
    assert at.pick_best([T(128, 5, 0, math.inf, 3000, 2e-4, False),
                         T(128, 10, 0, math.inf, 3000, 1e-4, False)]).inner == 10   # none reached: least error


def test_tune_with_injected_measurement():
    class F:
        shape = (256, 256)

    def fake(tile, inner, variant, j_ref):
        ms = 100.0 / inner + (10.0 if tile == 64 else 0.0)
        return at.Trial(tile, inner, variant, ms, 1000 // inner, 5e-5, True)

    r = at.tune(F(), dict(fidelity="l2", alpha=10.0), j_ref=1.0, tiles=(64, 128), inners=(5, 10, 20),
                solve_fn=fake)
    assert (r.best.tile, r.best.inner) == (128, 20)
    assert len(r.trials) == 6 and r.j_ref == 1.0


@pytest.mark.gpu
def test_tuned_configuration_reaches_tolerance():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import synth
    from paper_1901_00682_gb300 import _lib as L
    f, _ = synth.rof_image(256, 256, 12, 0.05, 31)
    pr = oracle.Problem(256, 256, alpha=10.0)
    st = oracle.cp_run(pr, f.astype(np.float64), 20000)
    jstar = oracle.energy(pr, st.u, f.astype(np.float64))
    fd = torch.from_numpy(f).cuda()
    r = at.tune(fd, dict(fidelity="l2", alpha=10.0), tol=1e-4, j_ref=jstar, tiles=(64, 128), inners=(5, 10, 20),
                max_outer=2000)
    assert r.best.reached
    b = r.best
    p = L.make_params(256, 256, 256 // b.tile, 256 // b.tile, alpha=10.0, inner_iters=b.inner,
                      outer_iters=b.outer)
    u, _, _ = L.Solver(p).solve_host(f)
    assert (oracle.energy(pr, u.astype(np.float64), f.astype(np.float64)) - jstar) / jstar <= 1.01e-4


def test_tune_batch_with_injected_measurement():
    """The batch autotuner searches subdomain side x K and keeps the fastest trial that
    reached the tolerance."""
    def fake(tile, inner, j_ref):
        ms = {5: 30.0, 10: 25.0, 20: 32.0}[inner] + (5.0 if tile == 64 else 0.0)
        return at.Trial(tile, inner, 0, ms, 600 // inner, 8e-5, True)

    r = at.tune_batch([dict(height=128, width=128)], None, j_ref=[1.0], inners=(5, 10, 20), tiles=(64, 128),
                      solve_fn=fake)
    assert (r.best.tile, r.best.inner) == (128, 10)
    assert len(r.trials) == 6 and {t.tile for t in r.trials} == {64, 128}


@pytest.mark.gpu
def test_tuned_batch_reaches_tolerance():
    """A small mixed batch: the tuned K reaches the tolerance on every image, against
    J* estimated by a long batched run."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import synth
    ims = []
    for k, (h, w, fid) in enumerate([(256, 256, "l2"), (128, 256, "seg"), (256, 128, "l2")]):
        f, _ = synth.rof_image(h, w, 8, 0.05, 40 + k)
        ims.append(dict(height=h, width=w, fidelity=fid, alpha=10.0 if fid == "l2" else 20.0,
                        c1=0.2 if fid == "seg" else 0.0, c2=0.8 if fid == "seg" else 0.0, f=f))
    fs = [torch.from_numpy(m["f"]).cuda() for m in ims]
    jr = at.batch_reference_energies(ims, fs, inner=20, outer=1500)
    r = at.tune_batch(ims, fs, tol=1e-3, j_ref=jr, inners=(5, 10), tiles=(64, 128), max_outer=1500)
    assert r.best.reached and r.best.rel_err <= 1e-3
    assert {t.tile for t in r.trials} == {64, 128} and all(t.reached for t in r.trials)
