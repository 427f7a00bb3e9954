"""The paper's ADMM code solver (Sec. 3.2: rho = 10 lambda, over-relaxation
1.8, the QP substep by conjugate gradient) on the GPU against the oracle's
ADMM, image by image; and ADMM and proximal gradient reaching the same LASSO
optimum of Eq. 3 on the GPU."""
import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_both(K, s, H, W, p, lam, n_iters, cg_iters, seed, t=1, warm=None):
    x, d, _ = make_case(H, W, K, s, seed=seed)
    npx = int(np.dot(H, W))
    z0 = np.zeros(npx * K, np.float32) if warm is None else warm
    ids = list(range(7, 7 + len(H)))
    ctx = scsc.Context(K, s, lam=lam, p=p, seed=seed + 50)
    b = scsc.Batch(H, W, ids=ids)
    z = dev(z0)
    ctx.code_step_admm(b, dev(x), dev(d), z, t, n_iters, cg_iters)
    ctx.sync()
    cfg = R.Config(K=K, s=s, lam=lam, p_num=p[0], p_den=p[1], seed=seed + 50)
    rb = R.Batch(H=H, W=W, ids=ids)
    zo = np.zeros(npx * K)
    for n in range(len(H)):
        m = R.mask_image(cfg, t, ids[n], H[n], W[n]).ravel()
        o = int(rb.off[n]) * K
        zi = R.admm_image(cfg, d, rb.image(x, n), rb.image(z0, n, K), m, H[n], W[n], n_iters,
                          cg_iters=cg_iters)
        zo[o:o + zi.size] = zi
    fg = ctx.objective(b, dev(x), z, dev(d))
    fo = R.objective(cfg, rb, x, zo, d)
    return z.cpu().numpy(), zo, fg, fo


def test_admm_c1_shape_matches_oracle():
    """One 100x100 image, K = 16, p = 1/2, lambda = 1: 10 ADMM iterations with
    30 CG steps each."""
    zg, zo, fg, fo = run_both(16, 11, [100], [100], (1, 2), 1.0, 10, 30, seed=1)
    assert fg == pytest.approx(fo, rel=1e-5)
    assert rel_l2(zg, zo) < 1e-3


def test_admm_ragged_batch_and_warm_start():
    K, s, H, W = 8, 7, [30, 17, 40], [50, 33, 129]
    npx = int(np.dot(H, W))
    warm = make_case(H, W, K, s, seed=9, code_density=0.1)[2]
    zg, zo, fg, fo = run_both(K, s, H, W, (1, 3), 0.5, 5, 20, seed=3, t=2, warm=warm)
    assert fg == pytest.approx(fo, rel=1e-5)
    assert rel_l2(zg, zo) < 1e-3
    assert npx * K == zg.size


def test_admm_and_pg_reach_the_same_optimum():
    K, s, H, W = 4, 5, [16], [20]
    x, d, _ = make_case(H, W, K, s, seed=5)
    b = scsc.Batch(H, W)
    za = torch.zeros(H[0] * W[0] * K, device="cuda")
    zp = torch.zeros_like(za)
    ctx = scsc.Context(K, s, lam=0.2, p=(1, 2), seed=6)
    ctx.code_step_admm(b, dev(x), dev(d), za, 1, 300, 40)
    ctx.code_step(b, dev(x), dev(d), zp, 1, 4000)
    ctx.sync()
    fa = ctx.objective(b, dev(x), za, dev(d))
    fp = ctx.objective(b, dev(x), zp, dev(d))
    assert fa == pytest.approx(fp, rel=2e-5)
