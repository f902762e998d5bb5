"""The seeded generators: deterministic, in range, with the recipe's statistics."""
import numpy as np

import synth


def test_deterministic_and_seed_dependent():
    a, _ = synth.rof_image(64, 48, 12, 0.05, 3)
    b, _ = synth.rof_image(64, 48, 12, 0.05, 3)
    c, _ = synth.rof_image(64, 48, 12, 0.05, 4)
    assert a.dtype == np.float32 and a.shape == (64, 48)
    assert synth.array_digest(a) == synth.array_digest(b) != synth.array_digest(c)


def test_piecewise_constant_and_noise_level():
    f, clean = synth.rof_image(256, 256, 12, 0.05, 0)
    assert clean.min() >= 0.0 and clean.max() <= 1.0
    assert len(np.unique(clean)) <= 13                  # background + 12 shapes
    assert abs(np.std(f - clean) - 0.05) < 0.002


def test_salt_pepper_and_mask_rates():
    f, mask, clean = synth.tvl1_inpaint_image(512, 512, 20, 0.1, 0.2, 1)
    assert abs(mask.mean() - 0.2) < 0.01
    assert np.all(f[mask == 1] == 0.0)
    keep = mask == 0
    changed = f[keep] != clean[keep]
    assert abs(changed.mean() - 0.1 * (1 - np.mean((clean[keep] == 0) | (clean[keep] == 1)))) < 0.02
    assert set(np.unique(f[keep][changed])) <= {0.0, 1.0}


def test_batch_workload_shapes():
    """Config 4: 64 images with short side s in {256, 512, 1024, 2048} and aspect 1:1,
    2:1 or 1:2 (s x s, s x 2s, 2s x s), even ROF and odd segmentation; every side a
    multiple of 128 (the batch's subdomain side); the draw of seed 0 is deterministic."""
    ims = synth.batch_workload(64, 0)
    assert len(ims) == 64
    for i, m in enumerate(ims):
        h, w = m["height"], m["width"]
        s, l = min(h, w), max(h, w)
        assert s in (256, 512, 1024, 2048) and l in (s, 2 * s)
        assert h % 128 == 0 and w % 128 == 0 and m["f"].shape == (h, w)
        assert m["fidelity"] == ("l2" if i % 2 == 0 else "seg")
    assert sum(m["height"] * m["width"] for m in ims) == 168230912
    a, b = synth.batch_workload(3, 0), synth.batch_workload(3, 0)
    assert all(np.array_equal(x["f"], y["f"]) for x, y in zip(a, b))
