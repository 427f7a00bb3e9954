"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws images, filters,
codes and batch layouts.  Both the GPU path's tests and the oracle read what
it returns, so the two sides always see identical float32 values.

Recipe (stands in for the paper's fruit/city 100x100 images, ImageNet
100x100 patches and 256x256 test images, which are not available here):
* image: sum of 30 isotropic Gaussian blobs, centre uniform in [0,W)x[0,H),
  sigma ~ U[2, 8] px, amplitude ~ U[-1, 1], plus i.i.d. N(0, 0.05^2) noise,
  then the image mean is subtracted (the configs' preprocessing);
* filters: N(0, 1) per tap, each filter scaled to unit L2 norm;
* all draws from numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import numpy as np


def blob_image(rng: np.random.Generator, H: int, W: int, n_blobs: int = 30,
               noise_std: float = 0.05) -> np.ndarray:
    img = np.zeros((H, W), dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    xs = np.arange(W, dtype=np.float64)
    cy = rng.uniform(0.0, H, n_blobs)
    cx = rng.uniform(0.0, W, n_blobs)
    sig = rng.uniform(2.0, 8.0, n_blobs)
    amp = rng.uniform(-1.0, 1.0, n_blobs)
    for b in range(n_blobs):
        gy = np.exp(-((ys - cy[b]) ** 2) / (2.0 * sig[b] ** 2))
        gx = np.exp(-((xs - cx[b]) ** 2) / (2.0 * sig[b] ** 2))
        img += amp[b] * np.outer(gy, gx)
    img += rng.normal(0.0, noise_std, (H, W))
    img -= img.mean()
    return img.astype(np.float32)


def images(seed: int, H, W) -> np.ndarray:
    """Packed float32 images for per-image sizes H[n] x W[n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.concatenate([blob_image(rng, int(h), int(w)).ravel() for h, w in zip(H, W)])


def filters(seed: int, K: int, s: int = 11) -> np.ndarray:
    """Float32 [K][s][s] filters, N(0,1) taps, each scaled to unit norm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.normal(0.0, 1.0, (K, s * s))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32).reshape(K, s, s)


def sparse_codes(seed: int, n_pixels: int, K: int, density: float = 0.05,
                 scale: float = 0.5) -> np.ndarray:
    """Float32 [n_pixels][K] codes, each nonzero with probability `density`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.normal(0.0, scale, (n_pixels, K))
    z *= rng.random((n_pixels, K)) < density
    return z.astype(np.float32).ravel()


def uneven_sizes(seed: int, n_images: int, lo: int = 64, hi: int = 512):
    """Per-image (H, W), each independently uniform in {lo..hi}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = rng.integers(lo, hi + 1, n_images)
    W = rng.integers(lo, hi + 1, n_images)
    return H.astype(np.int32), W.astype(np.int32)


def observed_pixels(seed: int, n_pixels: int, fraction: float = 0.5) -> np.ndarray:
    """Inpainting observation mask: each pixel observed (1) independently with
    the given probability (the paper's experiment observes 50% at random)."""
    rng = np.random.default_rng(seed)
    return (rng.random(n_pixels) < fraction).astype(np.uint8)
