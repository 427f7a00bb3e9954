"""The rewritings the online dictionary step's kernels compute, checked on the
CPU against the FP64 oracle and plain linear algebra (no GPU, no library).

- Eq. 7's sum of Z^T Z over an image's patches equals the cross-correlations
  of the code maps at the lag between two columns, minus the products whose
  patch centre lies outside the image (the border correction).  The same for
  Z^T x over the centres inside the image.
- A product with the symmetric C from its upper 128 x 128 block triangle: each
  block's row products go to slot J of panel I and its column products to slot
  I of panel J, every (slot, row) written once, and the slots add up to C v.
- The closed-form map from a block number to its (I, J) of the upper triangle,
  and the bound on the number of correlation segments.
"""
import math

import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case


def _codes(z, K, H, W, off):
    """Codes of one image as [K][H][W] from the [pixel][K] layout."""
    return z[off * K:(off + H * W) * K].reshape(H, W, K).transpose(2, 0, 1).astype(np.float64)


def _surrogates_by_correlation(K, s, Hs, Ws, x, z, border=True):
    """sum_n Z_n^T Z_n and Z_n^T x_n as cross-correlations of the code maps
    plus (unless border is False) the border correction, in FP64."""
    c = (s - 1) // 2
    M, D = s * s, 2 * s - 1
    KM = K * M
    C = np.zeros((KM, KM))
    B = np.zeros(KM)
    off = 0
    for H, W in zip(Hs, Ws):
        zi = _codes(z, K, H, W, off)
        xi = x[off:off + H * W].reshape(H, W).astype(np.float64)
        off += H * W
        # T[k][k2][dy][dx] = sum over r1 with r1 + (dy, dx) in the image
        T = np.zeros((K, K, D, D))
        for dy in range(-(s - 1), s):
            for dx in range(-(s - 1), s):
                y0, y1 = max(0, -dy), min(H, H - dy)
                x0, x1 = max(0, -dx), min(W, W - dx)
                if y0 >= y1 or x0 >= x1:
                    continue
                a = zi[:, y0:y1, x0:x1]
                b = zi[:, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
                T[:, :, dy + s - 1, dx + s - 1] = np.einsum("kyx,lyx->kl", a, b)
        for k in range(K):
            ys, xs = np.nonzero(zi[k])
            for u in range(s):
                for v in range(s):
                    a = k * M + u * s + v
                    for k2 in range(K):
                        for u2 in range(s):
                            for v2 in range(s):
                                C[a, k2 * M + u2 * s + v2] += T[k, k2, u - u2 + s - 1,
                                                               v - v2 + s - 1]
                    for y1_, x1_ in zip(ys, xs):
                        zv = zi[k, y1_, x1_]
                        qy, qx = y1_ - c + u, x1_ - c + v
                        if 0 <= qy < H and 0 <= qx < W:
                            B[a] += zv * xi[qy, qx]
                            continue
                        if not border:
                            continue
                        # centre outside: the products the correlation counted
                        for u2 in range(s):
                            for v2 in range(s):
                                ry, rx = qy + c - u2, qx + c - v2
                                if 0 <= ry < H and 0 <= rx < W:
                                    C[a, u2 * s + v2::M][:K] -= zv * zi[:, ry, rx]
    return C, B


@pytest.mark.parametrize("K,s,Hs,Ws,density", [(3, 5, [9, 12], [12, 7], 0.2),
                                                (2, 3, [4, 6], [5, 3], 0.5),
                                                (2, 5, [3], [4], 0.6)])
def test_correlation_form_equals_patch_sum(K, s, Hs, Ws, density):
    """Eq. 7's per-patch sums against the correlation form, including images
    smaller than the filter (every centre near a border)."""
    x, _, z = make_case(Hs, Ws, K, s, seed=91, code_density=density)
    cfg = R.Config(K=K, s=s, seed=3)
    st = R.OnlineState(cfg)
    st.update(R.Batch(H=Hs, W=Ws, ids=list(range(len(Hs)))), x, z)  # t = 1: mean over images
    C, B = _surrogates_by_correlation(K, s, Hs, Ws, x, z)
    n = len(Hs)
    scale = max(1.0, np.abs(st.C).max())
    assert np.abs(C / n - st.C).max() <= 1e-12 * scale
    assert np.abs(B / n - st.B).max() <= 1e-12 * max(1.0, np.abs(st.B).max())
    # the border term matters on these sizes: the correlations alone differ
    C0, _ = _surrogates_by_correlation(K, s, Hs, Ws, x, z, border=False)
    assert np.abs(C0 / n - st.C).max() > 1e-3 * scale


def _upper_offset(I, NP):
    return I * NP - I * (I - 1) // 2


def _upper_block(b, NP):
    tn = 2.0 * NP + 1.0
    I = int((tn - math.sqrt(tn * tn - 8.0 * b)) * 0.5)
    I = min(max(I, 0), NP - 1)
    while I > 0 and _upper_offset(I, NP) > b:
        I -= 1
    while I + 1 < NP and _upper_offset(I + 1, NP) <= b:
        I += 1
    return I, I + (b - _upper_offset(I, NP))


@pytest.mark.parametrize("NP", [1, 2, 3, 29, 379, 1000])
def test_upper_block_map_covers_the_triangle_once(NP):
    seen = set()
    for b in range(NP * (NP + 1) // 2):
        I, J = _upper_block(b, NP)
        assert 0 <= I <= J < NP
        seen.add((I, J))
    assert len(seen) == NP * (NP + 1) // 2


@pytest.mark.parametrize("n", [75, 128, 300, 675])
def test_half_triangle_product_slots(n):
    """C v from the upper block triangle: the slot scheme of the products with
    the online surrogate, every (slot, row) written exactly once."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    Cm = A + A.T
    v = rng.standard_normal(n)
    blk = 128
    NP = (n + blk - 1) // blk
    part = np.full((NP, n), np.nan)
    for b in range(NP * (NP + 1) // 2):
        I, J = _upper_block(b, NP)
        rows = slice(I * blk, min(n, (I + 1) * blk))
        cols = slice(J * blk, min(n, (J + 1) * blk))
        assert np.all(np.isnan(part[J, rows]))
        part[J, rows] = Cm[rows, cols] @ v[cols]
        if I != J:
            assert np.all(np.isnan(part[I, cols]))
            part[I, cols] = Cm[rows, cols].T @ v[rows]
    assert not np.any(np.isnan(part))
    np.testing.assert_allclose(part.sum(axis=0), Cm @ v, rtol=1e-12, atol=1e-12)


def test_correlation_segment_bound():
    """sum_k ceil(count_k / L) <= floor(nnz / L) + K: the grid and the slice
    buffer sized from nnz alone hold every segment, for skewed counts too."""
    rng = np.random.default_rng(2)
    for L in (1, 7, 256, 1024):
        for _ in range(200):
            K = int(rng.integers(1, 513))
            counts = (rng.pareto(1.2, K) * rng.integers(1, 2000)).astype(np.int64)
            segs = int(((counts + L - 1) // L).sum())
            assert segs <= int(counts.sum()) // L + K
