"""Shared helpers of the test suite: seeded inputs, running both sides."""
from __future__ import annotations

import numpy as np

from oracle import reference as R
from paper_1909_00145_gb300 import inputs as I


def make_case(H, W, K, s=11, seed=0, code_density=None):
    """Seeded float32 images, filters and (optionally) random sparse codes."""
    H = np.atleast_1d(H)
    W = np.atleast_1d(W)
    x = I.images(seed + 1, H, W)
    d = I.filters(seed + 2, K, s)
    npx = int((H.astype(np.int64) * W).sum())
    z = (I.sparse_codes(seed + 3, npx, K, density=code_density)
         if code_density is not None else np.zeros(npx * K, dtype=np.float32))
    return x, d, z


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_bits(cfg: R.Config, batch: R.Batch, t: int) -> np.ndarray:
    """Oracle mask packed the way scsc_mask returns it: [pixel][ceil(K/32)] u32."""
    m = R.mask_batch(cfg, batch, t).reshape(-1, cfg.K).astype(np.uint64)
    kw = (cfg.K + 31) // 32
    out = np.zeros((m.shape[0], kw), dtype=np.uint64)
    for k in range(cfg.K):
        out[:, k // 32] |= m[:, k] << np.uint64(k % 32)
    return out.astype(np.uint32).ravel()


def support_jaccard(a, b) -> float:
    """Jaccard index of the nonzero sets of two code vectors (1 when both are
    all zero): the support agreement of two solutions of the lasso."""
    sa = np.asarray(a).ravel() != 0
    sb = np.asarray(b).ravel() != 0
    union = int(np.count_nonzero(sa | sb))
    return 1.0 if union == 0 else int(np.count_nonzero(sa & sb)) / union


def measured(name: str, **vals) -> None:
    """Print a measured error next to its test (visible with pytest -s)."""
    print("MEASURED " + name + " " + " ".join(f"{k}={v:.3e}" for k, v in vals.items()))
