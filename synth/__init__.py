"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module only draws random images, noise and masks.  It holds none of the
method's arithmetic, so both sides may import it without sharing any solver code.

Every image is a stand-in for the photographs of Section 5 (not available here):
a piecewise-constant scene of axis-aligned rectangles and disks with intensities
in [0, 1], then corrupted by Gaussian noise (denoising, Sections 5.1 and 5.2) or
salt-and-pepper noise (TV-L1, Sections 5.1 and 5.2), optionally with a random
inpainting domain D on which f is set to 0 (Section 3, inpainting models).

All draws come from ``numpy.random.Generator(PCG64(seed))`` in a fixed order, so
the same seed gives the same float32 array on every platform.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np

__all__ = [
    "piecewise_constant",
    "add_gaussian_noise",
    "add_salt_and_pepper",
    "bernoulli_mask",
    "rof_image",
    "tvl1_inpaint_image",
    "seg_image",
    "array_digest",
    "Workload",
    "WORKLOADS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def piecewise_constant(height: int, width: int, n_shapes: int, rng: np.random.Generator) -> np.ndarray:
    """Background U[0,1], then ``n_shapes`` shapes painted in order.

    Each shape draws, in this order: intensity U[0,1], kind (rectangle or disk,
    50/50), then its geometry.  Rectangle: height U[H/16, H/4], width U[W/16, W/4],
    top-left corner uniform over the image (clipped at the border).  Disk: radius
    U[min(H,W)/32, min(H,W)/8], centre uniform over the image.
    Returns float64 (the caller rounds to float32 once, at the end).
    """
    img = np.full((height, width), rng.uniform(0.0, 1.0), dtype=np.float64)
    for _ in range(n_shapes):
        val = rng.uniform(0.0, 1.0)
        kind = rng.integers(0, 2)
        if kind == 0:
            rh = int(rng.uniform(height / 16.0, height / 4.0))
            rw = int(rng.uniform(width / 16.0, width / 4.0))
            r0 = int(rng.integers(0, height))
            c0 = int(rng.integers(0, width))
            img[r0:r0 + max(rh, 1), c0:c0 + max(rw, 1)] = val
        else:
            m = min(height, width)
            rad = rng.uniform(m / 32.0, m / 8.0)
            cy = rng.uniform(0.0, height)
            cx = rng.uniform(0.0, width)
            y0, y1 = max(int(cy - rad) - 1, 0), min(int(cy + rad) + 2, height)
            x0, x1 = max(int(cx - rad) - 1, 0), min(int(cx + rad) + 2, width)
            if y1 <= y0 or x1 <= x0:
                continue
            yy = np.arange(y0, y1, dtype=np.float64)[:, None] + 0.5 - cy
            xx = np.arange(x0, x1, dtype=np.float64)[None, :] + 0.5 - cx
            inside = (yy * yy + xx * xx) <= rad * rad
            sub = img[y0:y1, x0:x1]
            sub[inside] = val
    return img


def add_gaussian_noise(img: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Additive N(0, sigma^2) noise, no clipping."""
    return img + sigma * rng.standard_normal(img.shape)


def add_salt_and_pepper(img: np.ndarray, density: float, rng: np.random.Generator) -> np.ndarray:
    """Each pixel, with probability ``density``, is replaced by 0 or 1 (50/50)."""
    hit = rng.uniform(0.0, 1.0, img.shape) < density
    salt = rng.uniform(0.0, 1.0, img.shape) < 0.5
    out = img.copy()
    out[hit] = salt[hit].astype(np.float64)
    return out


def bernoulli_mask(shape, prob: float, rng: np.random.Generator) -> np.ndarray:
    """uint8 mask of the inpainting domain D: 1 = pixel in D (value unknown)."""
    return (rng.uniform(0.0, 1.0, shape) < prob).astype(np.uint8)


def rof_image(height: int, width: int, n_shapes: int, sigma: float, seed: int):
    """(f, clean) float32 pair for L2 denoising: piecewise constant + Gaussian noise."""
    rng = _rng(seed)
    clean = piecewise_constant(height, width, n_shapes, rng)
    noisy = add_gaussian_noise(clean, sigma, rng)
    return noisy.astype(np.float32), clean.astype(np.float32)


def tvl1_inpaint_image(height: int, width: int, n_shapes: int, sp_density: float,
                       mask_prob: float, seed: int):
    """(f, mask, clean) for L1 inpainting + impulse denoising; f := 0 on D."""
    rng = _rng(seed)
    clean = piecewise_constant(height, width, n_shapes, rng)
    noisy = add_salt_and_pepper(clean, sp_density, rng)
    mask = bernoulli_mask(noisy.shape, mask_prob, rng)
    noisy[mask == 1] = 0.0
    return noisy.astype(np.float32), mask, clean.astype(np.float32)


def seg_image(height: int, width: int, n_shapes: int, sigma: float, seed: int):
    """(f, clean) for two-phase segmentation: same generator, Gaussian noise."""
    return rof_image(height, width, n_shapes, sigma, seed)


def array_digest(*arrays: np.ndarray) -> str:
    """sha256 over the raw bytes of the arrays (to detect generator drift)."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


@dataclass(frozen=True)
class Workload:
    """One named synthetic workload: image recipe and solver settings."""

    name: str
    height: int
    width: int
    n_shapes: int
    noise: float
    fidelity: str  # "l2", "l1", "seg"
    alpha: float
    sub_rows: int
    sub_cols: int
    outer: int
    inner: int
    sp_density: float = 0.0
    mask_prob: float = 0.0
    seed: int = 0

    def make(self, seed: int | None = None):
        """Returns (f, mask_or_None, clean)."""
        s = self.seed if seed is None else seed
        if self.fidelity == "l1" and self.mask_prob > 0:
            f, mask, clean = tvl1_inpaint_image(self.height, self.width, self.n_shapes,
                                                self.sp_density, self.mask_prob, s)
            return f, mask, clean
        f, clean = rof_image(self.height, self.width, self.n_shapes, self.noise, s)
        return f, None, clean


def batch_workload(n_images: int = 64, seed: int = 0):
    """The mixed batch: image i has short side s in {256, 512, 1024, 2048} and aspect in
    {1:1 (s x s), 2:1 landscape (s x 2s), 1:2 portrait (2s x s)} (both drawn uniformly;
    mean area 2.32 Mpixel); even i is ROF denoising
    (sigma 0.05, alpha 10), odd i two-phase segmentation of a noisy piecewise-constant
    image (sigma 0.05, c1 0.2, c2 0.8, alpha 20).  Returns a list of dicts with the
    image (float32), its shape, fidelity and parameters; image i uses seed 1000*seed+i."""
    rng = _rng(seed)
    out = []
    for i in range(n_images):
        side = int(rng.choice([256, 512, 1024, 2048]))
        aspect = int(rng.integers(0, 3))
        h, w = (side, side) if aspect == 0 else ((side, 2 * side) if aspect == 1 else (2 * side, side))
        shapes = max(4, (h * w) // (4096 * 4096 // 400))
        f, clean = rof_image(h, w, shapes, 0.05, 1000 * seed + i)
        if i % 2 == 0:
            out.append(dict(height=h, width=w, fidelity="l2", alpha=10.0, c1=0.0, c2=0.0, f=f, clean=clean))
        else:
            out.append(dict(height=h, width=w, fidelity="seg", alpha=20.0, c1=0.2, c2=0.8, f=f, clean=clean))
    return out


WORKLOADS = {
    # ROF denoising 128x128, 2x2 subdomains of 64x64, 200 outer x 10 inner
    "rof128": Workload("rof128", 128, 128, 12, 0.05, "l2", 10.0, 2, 2, 200, 10),
    # ROF denoising 4096x4096, 32x32 subdomains of 128x128, inner 10
    "rof4096": Workload("rof4096", 4096, 4096, 400, 0.1, "l2", 8.0, 32, 32, 0, 10),
    # TV-L1 inpainting + impulse denoising 2048x2048, 16x16 subdomains, 500 outer
    "tvl1_2048": Workload("tvl1_2048", 2048, 2048, 100, 0.0, "l1", 1.5, 16, 16, 500, 10,
                          sp_density=0.1, mask_prob=0.2),
}
