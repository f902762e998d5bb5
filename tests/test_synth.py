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
