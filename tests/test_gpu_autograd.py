"""Differentiation wrapper: torch.autograd.Function over the library's masked
synthesis, whose backward runs the library's adjoint kernels.

Checked against the FP64 oracle's analytic gradients on the C2 shape (16
images 128x128, K = 100), against FP64 central differences of the oracle's
loss, and against the adjoint identity <Dz, r> = <z, D^T r>, for
p in {0.1, 0.25, 0.5, 1}.
"""
import numpy as np
import pytest

from oracle import reference as R
from paper_1909_00145_gb300 import inputs as I
from tests.helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402
from paper_1909_00145_gb300.autograd import synthesis  # noqa: E402

P_GRID = [(1, 10), (1, 4), (1, 2), (1, 1)]


def gpu_grads(ctx, batch, x, z, d, t):
    zt = torch.from_numpy(z).cuda().requires_grad_(True)
    dt = torch.from_numpy(np.ascontiguousarray(d)).cuda().requires_grad_(True)
    xt = torch.from_numpy(x).cuda()
    xhat = synthesis(zt, dt, ctx, batch, t, True)
    loss = 0.5 * ((xhat - xt) ** 2).sum()
    loss.backward()
    return xhat.detach().cpu().numpy(), zt.grad.cpu().numpy(), dt.grad.cpu().numpy().ravel()


@pytest.mark.parametrize("p", P_GRID)
def test_backward_matches_oracle_gradients_c2(p):
    K, s = 100, 11
    n = 16 if p == (1, 4) else 4
    H, W = [128] * n, [128] * n
    x = I.images(21, H, W)
    d = I.filters(22, K, s)
    z = I.sparse_codes(23, int(np.dot(H, W)), K, density=0.05)
    ctx = scsc.Context(K, s, p=p, seed=5)
    b = scsc.Batch(H, W)
    xhat, gz, gd = gpu_grads(ctx, b, x, z, d, t=3)
    cfg = R.Config(K=K, s=s, p_num=p[0], p_den=p[1], seed=5)
    rb = R.Batch(H=H, W=W, ids=list(range(n)))
    m = R.mask_batch(cfg, rb, 3).astype(bool)
    zm = np.where(m, z, 0.0)
    xo = R.synthesis_batch(cfg, rb, zm, d)
    r = xo - x
    gz_o = np.where(m, np.concatenate([R.adjoint(d, rb.image(r, i), K, s, 128, 128)
                                       for i in range(n)]), 0.0)
    gd_o = sum(R.filter_gradient(rb.image(r, i), rb.image(zm, i, K), K, s, 128, 128)
               for i in range(n))
    assert rel_l2(xhat, xo) < 1e-5
    assert rel_l2(gz, gz_o) < 1e-5
    assert rel_l2(gd, gd_o) < 1e-5
    assert np.all(gz[~m] == 0)


def _local_loss(z, d, x, K, s, H, W, a, bb, m):
    """0.5 ||D(m.z) - x||^2 restricted to the pixels a code at (a, bb) reaches:
    the synthesis is taken on a crop with a margin of 2c, exact inside."""
    c = (s - 1) // 2
    y0, y1 = max(0, a - 2 * c), min(H, a + 2 * c + 1)
    x0, x1 = max(0, bb - 2 * c), min(W, bb + 2 * c + 1)
    zz = (np.where(m, z, 0.0)).reshape(H, W, K)[y0:y1, x0:x1, :].copy()
    xh = R.synthesis(d, zz.ravel(), K, s, y1 - y0, x1 - x0).reshape(y1 - y0, x1 - x0)
    wy0, wy1 = max(0, a - c) - y0, min(H, a + c + 1) - y0
    wx0, wx1 = max(0, bb - c) - x0, min(W, bb + c + 1) - x0
    rr = xh[wy0:wy1, wx0:wx1] - x.reshape(H, W)[y0 + wy0:y0 + wy1, x0 + wx0:x0 + wx1]
    return 0.5 * float(np.sum(rr * rr))


@pytest.mark.parametrize("p", P_GRID)
def test_backward_matches_fp64_central_differences(p):
    K, s = 100, 11
    # codes: one 128x128 image, 50 coordinates, local exact loss differences
    H = W = 128
    x = I.images(31, [H], [W]).astype(np.float64)
    d = I.filters(32, K, s).astype(np.float64)
    z = I.sparse_codes(33, H * W, K, density=0.05).astype(np.float64)
    ctx = scsc.Context(K, s, p=p, seed=7)
    b = scsc.Batch([H], [W])
    _, gz, _ = gpu_grads(ctx, b, x.astype(np.float32), z.astype(np.float32), d.astype(np.float32), 2)
    cfg = R.Config(K=K, s=s, p_num=p[0], p_den=p[1], seed=7)
    m = R.mask_image(cfg, 2, 0, H, W).ravel().astype(bool)
    rng = np.random.default_rng(0)
    idx = rng.choice(H * W * K, 50, replace=False)
    scale = np.abs(gz).max()
    for i in idx:
        pix, k = divmod(int(i), K)
        a, bb = divmod(pix, W)
        h = 1e-6 * max(1.0, abs(z[i]))
        zp, zm_ = z.copy(), z.copy()
        zp[i] += h
        zm_[i] -= h
        fd = (_local_loss(zp, d, x, K, s, H, W, a, bb, m) -
              _local_loss(zm_, d, x, K, s, H, W, a, bb, m)) / (2 * h)
        assert abs(gz[i] - fd) <= 1e-4 * scale, (i, gz[i], fd)
    # filters: a small image, 50 coordinates, full loss differences
    H2 = W2 = 40
    x2 = I.images(34, [H2], [W2]).astype(np.float64)
    z2 = I.sparse_codes(35, H2 * W2, K, density=0.1).astype(np.float64)
    b2 = scsc.Batch([H2], [W2])
    _, _, gd = gpu_grads(ctx, b2, x2.astype(np.float32), z2.astype(np.float32),
                         d.astype(np.float32), 4)
    m2 = R.mask_image(cfg, 4, 0, H2, W2).ravel().astype(bool)
    zm2 = np.where(m2, z2, 0.0)

    def loss(dd):
        rr = R.synthesis(dd, zm2, K, s, H2, W2) - x2
        return 0.5 * float(np.dot(rr, rr))

    scale = np.abs(gd).max()
    for i in rng.choice(K * s * s, 50, replace=False):
        dv = d.ravel().copy()
        h = 1e-6 * max(1.0, abs(dv[i]))
        dp, dm = dv.copy(), dv.copy()
        dp[i] += h
        dm[i] -= h
        fd = (loss(dp) - loss(dm)) / (2 * h)
        assert abs(gd[i] - fd) <= 1e-4 * scale, (i, gd[i], fd)


@pytest.mark.parametrize("p", P_GRID)
def test_adjoint_identity_through_autograd(p):
    K, s, H, W = 100, 11, [128, 96], [128, 160]
    z = torch.from_numpy(I.sparse_codes(41, int(np.dot(H, W)), K, density=0.05)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(I.filters(42, K, s))).cuda()
    r = torch.randn(int(np.dot(H, W)), generator=torch.Generator().manual_seed(1)).cuda()
    ctx = scsc.Context(K, s, p=p, seed=9)
    b = scsc.Batch(H, W)
    zt = z.clone().requires_grad_(True)
    dt = d.clone().requires_grad_(True)
    xhat = synthesis(zt, dt, ctx, b, 6, True)
    (xhat * r).sum().backward()
    lhs = float((xhat.double() * r.double()).sum())
    assert abs(lhs - float((zt.grad.double() * z.double()).sum())) <= 1e-5 * abs(lhs)
    # the masked synthesis is bilinear: <D(m.z) d, r> = <d, Z^T r>
    assert abs(lhs - float((dt.grad.double() * d.double()).sum())) <= 1e-5 * abs(lhs)
