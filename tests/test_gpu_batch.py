"""Batched solve (many images, mixed sizes and fidelities, one launch per phase):
every image's iterate equals, bit for bit, the iterate of a solve of that image alone
with the same parameters, and matches the FP64 oracle within the parity tolerances."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_00682_gb300 import _lib as L
    L.load()
    return L


def _images():
    specs = [(256, 256, "l2", 10.0, 0.0, 0.0), (128, 384, "seg", 20.0, 0.2, 0.8), (384, 128, "l1", 1.5, 0.0, 0.0),
             (128, 128, "l2", 8.0, 0.0, 0.0), (512, 256, "seg", 20.0, 0.2, 0.8)]
    out = []
    for k, (h, w, fid, alpha, c1, c2) in enumerate(specs):
        f, _ = synth.rof_image(h, w, 10, 0.05, 100 + k)
        out.append(dict(height=h, width=w, fidelity=fid, alpha=alpha, c1=c1, c2=c2, f=f))
    return out


@pytest.mark.parametrize("tile,variant,K", [(128, 0, 10), (128, 2, 10), (64, 0, 10), (128, 0, 70)])
def test_batch_equals_single_image_solves_bitwise(tile, variant, K):
    """The batch kernels (128: persistent clusters over the work list, 4 x 4 micro-tiles
    (variant 0) or 2 x 4 (variant 2); 64: one CTA per subdomain) give each image the
    bits of its own solve.  Every image here has W + N_c not a multiple of 4, so the
    4 x 4 kernel copies their p2 rows 4 bytes at a time (the full-workload test below
    covers the 16-byte copies).  K = 70 exceeds the 4 x 4 kernel's coefficient table:
    variant 0 then runs the 2 x 4 kernel, as the single-image path does."""
    L = _lib()
    ims = _images()
    b = L.Batch(ims, inner_iters=K, tile=tile, variant=variant)
    fs = [torch.from_numpy(m["f"]).cuda() for m in ims]
    b.load(fs)
    b.iterate(13)
    for k, m in enumerate(ims):
        u_b = b.get_u(k, torch.empty_like(fs[k]))
        p = L.make_params(m["height"], m["width"], m["height"] // tile, m["width"] // tile, fidelity=m["fidelity"],
                          alpha=m["alpha"], c1=m["c1"], c2=m["c2"], inner_iters=K)
        s = L.Solver(p)
        s.load(fs[k])
        s.iterate(13)
        u_s = s.get_u(torch.empty_like(fs[k]))
        torch.cuda.synchronize()
        assert torch.equal(u_b, u_s), k
        J = b.energy(k)
        assert abs(J - s.current_energy()) <= 1e-12 * abs(J)
    assert b.pixels() == sum(m["height"] * m["width"] for m in ims)


def test_batch_matches_oracle():
    L = _lib()
    ims = _images()[1:3]   # segmentation and TV-L1
    b = L.Batch(ims, inner_iters=10)
    fs = [torch.from_numpy(m["f"]).cuda() for m in ims]
    b.load(fs)
    b.iterate(20)
    for k, m in enumerate(ims):
        u = b.get_u(k, torch.empty_like(fs[k])).cpu().numpy().astype(np.float64)
        tau = 1.0 if m["fidelity"] == "seg" else 50.0
        pr = oracle.Problem(m["height"], m["width"], m["height"] // 128, m["width"] // 128, fidelity=m["fidelity"],
                            alpha=m["alpha"], c1=m["c1"], c2=m["c2"], tau=tau, inner=10)
        st = oracle.dd_run(pr, m["f"].astype(np.float64), 20)
        assert np.abs(u - st.u).max() <= 5e-4
        Jo = oracle.energy(pr, st.u, m["f"].astype(np.float64))
        assert abs(b.energy(k) - Jo) <= 1e-5 * abs(Jo)


def test_batch_variants_bitwise_on_the_full_workload():
    """The 4 x 4 and 2 x 4 batch kernels give the same bits on the benchmark's batch."""
    L = _lib()
    ims = synth.batch_workload(64, 0)
    fs = [torch.from_numpy(m["f"]).cuda() for m in ims]
    us = []
    for variant in (0, 2):
        b = L.Batch(ims, inner_iters=10, variant=variant)
        b.load(fs)
        b.iterate(3)
        us.append([b.get_u(k, torch.empty_like(fs[k])) for k in range(len(ims))])
        b.close()
    torch.cuda.synchronize()
    for k in range(len(ims)):
        assert torch.equal(us[0][k], us[1][k]), k


def test_full_batch_workload_parity():
    """The benchmark's 64-image batch (synth.batch_workload(64, 0): 168 Mpixel, short
    sides 256 to 2048, aspects 1:1, 2:1, 1:2, ROF and segmentation) in the benchmark's
    launch configuration (128 x 128 subdomains, K = 10, one graph): after 2 outer
    iterations every image matches the FP64 oracle (5e-4 in u, 1e-5 in J)."""
    L = _lib()
    ims = synth.batch_workload(64, 0)
    b = L.Batch(ims, inner_iters=10)
    fs = [torch.from_numpy(m["f"]).cuda() for m in ims]
    b.load(fs)
    b.iterate(2)
    torch.cuda.synchronize()
    for k, m in enumerate(ims):
        u = b.get_u(k, torch.empty_like(fs[k])).cpu().numpy().astype(np.float64)
        tau = 1.0 if m["fidelity"] == "seg" else 50.0
        pr = oracle.Problem(m["height"], m["width"], m["height"] // 128, m["width"] // 128, fidelity=m["fidelity"],
                            alpha=m["alpha"], c1=m["c1"], c2=m["c2"], tau=tau, inner=10)
        f64 = m["f"].astype(np.float64)
        st = oracle.dd_run(pr, f64, 2)
        assert np.abs(u - st.u).max() <= 5e-4, k
        Jo = oracle.energy(pr, st.u, f64)
        assert abs(b.energy(k) - Jo) <= 1e-5 * abs(Jo), k
    b.close()


def test_batch_rejects_bad_shapes():
    L = _lib()
    with pytest.raises(L.DDTVError) as e:
        L.Batch([dict(height=100, width=128, fidelity="l2", alpha=1.0)])
    assert e.value.code == L.EINVAL


def test_batch_graph_runs_compose():
    """dd_tv_batch_iterate(n) is one graph launch of n outer iterations (captured per n
    and start parity): 5 + 8 + 1 iterations give the bits of 14 in one call."""
    L = _lib()
    ims = _images()
    fs = [torch.from_numpy(m["f"]).cuda() for m in ims]
    outs = []
    for runs in ((14,), (5, 8, 1)):
        b = L.Batch(ims, inner_iters=10)
        b.load(fs)
        for n in runs:
            b.iterate(n)
        outs.append([b.get_u(k, torch.empty_like(fs[k])) for k in range(len(ims))])
        b.close()
    torch.cuda.synchronize()
    for u1, u2 in zip(*outs):
        assert torch.equal(u1, u2)
