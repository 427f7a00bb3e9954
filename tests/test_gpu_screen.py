"""Safe screening of the code problem (Sec. 5) on the GPU against the oracle.

The test itself is a decision taken in floating point: the GPU takes it in
FP32 (FP64 per-image reductions), the oracle in FP64.  The removed sets must
agree except for coordinates whose oracle statistic lies within BAND of the
threshold 1 - 1e-4; gaps, codes and objectives are compared to FP32
tolerances.  Every test runs through the C-ABI entries scsc_screen and
scsc_code_step_screened."""
import numpy as np
import pytest

import bench
from oracle import reference as R
from tests.helpers import make_case, measured, oracle_bits, rel_l2, support_jaccard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402

THRESH = 1.0 - 1e-4
BAND = 1e-3


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def unpack_bits(bits, K):
    kw = (K + 31) // 32
    w = bits.reshape(-1, kw).astype(np.uint32)
    k = np.arange(K)
    return ((w[:, k // 32] >> (k % 32).astype(np.uint32)) & 1).astype(np.uint8).ravel()


def lam_max(cfg, rb, x, d, t):
    """max over the sampled set of |(D^T x)_j|, image by image (oracle)."""
    out = []
    for n in range(rb.n):
        H, W = int(rb.H[n]), int(rb.W[n])
        m = R.mask_image(cfg, t, int(rb.ids[n]), H, W).ravel()
        c = R.adjoint(d, rb.image(x, n), cfg.K, cfg.s, H, W)
        out.append(float(np.abs(c[m == 1]).max()))
    return out


def case(K, s, H, W, p, seed, frac, t=1):
    x, d, _ = make_case(H, W, K, s, seed=seed)
    ids = list(range(3, 3 + len(H)))
    rb = R.Batch(H=H, W=W, ids=ids)
    cfg0 = R.Config(K=K, s=s, lam=1.0, p_num=p[0], p_den=p[1], seed=seed + 10)
    lam = frac * min(lam_max(cfg0, rb, x, d, t))
    cfg = R.Config(K=K, s=s, lam=lam, p_num=p[0], p_den=p[1], seed=seed + 10)
    return x, d, ids, rb, cfg


def compare_removed(removed_gpu, removed_orc, stat_orc):
    """Equal decisions outside the rounding band around the threshold."""
    diff = removed_gpu != removed_orc
    assert np.all(np.abs(stat_orc[diff] - THRESH) < BAND), stat_orc[diff]
    assert diff.sum() <= max(2, 1e-3 * removed_orc.size)


@pytest.mark.parametrize("K,s,H,W,p,frac,pre_iters", [
    (16, 5, [24, 17], [20, 33], (1, 2), 0.85, 30),
    (40, 7, [40], [36], (1, 3), 0.7, 100),
    (100, 11, [48, 33], [40, 47], (1, 4), 0.85, 100),
])
def test_screen_matches_oracle(K, s, H, W, p, frac, pre_iters):
    """One test on FP32 codes taken after some oracle PG iterations: per-image
    gaps, survivor counts, the removed sets and the zeroed codes."""
    x, d, ids, rb, cfg = case(K, s, H, W, p, seed=K + s, frac=frac)
    z0 = R.code_step(cfg, rb, x, d, np.zeros(rb.total_pixels * K), t=1,
                     n_iters=pre_iters).astype(np.float32)
    bits0 = oracle_bits(cfg, rb, 1)
    ctx = scsc.Context(K, s, lam=cfg.lam, p=p, seed=cfg.seed)
    b = scsc.Batch(H, W, ids=ids)
    zg, bg = dev(z0), dev(bits0.view(np.int32))
    gaps, kept = ctx.screen(b, dev(x), dev(d), zg, bg)
    ctx.sync()
    zg, mg = zg.cpu().numpy(), unpack_bits(bg.cpu().numpy().view(np.uint32), K)
    m0 = R.mask_batch(cfg, rb, 1).ravel()
    for n in range(rb.n):
        Hn, Wn = int(rb.H[n]), int(rb.W[n])
        zo, mo, gap_o, stat = R.screen_image(cfg, d, rb.image(x, n), rb.image(z0, n, K),
                                             rb.image(m0, n, K), Hn, Wn)
        mgn = rb.image(mg, n, K)
        m0n = rb.image(m0, n, K)
        compare_removed((m0n == 1) & (mgn == 0), (m0n == 1) & (mo == 0), stat)
        assert kept[n] == int(mgn.sum())
        assert gaps[n] == pytest.approx(gap_o, rel=1e-4, abs=1e-6 * R.objective(
            cfg, R.Batch(H=[Hn], W=[Wn], ids=[ids[n]]), rb.image(x, n), rb.image(z0, n, K), d))
        zgn = rb.image(zg, n, K)
        assert not zgn[mgn == 0].any()
        np.testing.assert_array_equal(zgn[mgn == 1], rb.image(z0, n, K)[mgn == 1])
    assert (m0.sum() - mg.sum()) > 0.1 * m0.sum()  # the case removes coordinates


def test_screen_above_lambda_max_removes_everything():
    x, d, ids, rb, cfg = case(16, 5, [30, 21], [26, 40], (1, 2), seed=4, frac=1.05)
    # frac applies to the smaller lambda_max: lift lambda above both images'
    lam = 1.05 * max(lam_max(cfg, rb, x, d, 1))
    ctx = scsc.Context(16, 5, lam=lam, p=(1, 2), seed=cfg.seed)
    b = scsc.Batch([30, 21], [26, 40], ids=ids)
    z = torch.zeros(rb.total_pixels * 16, device="cuda")
    bits = ctx.mask(b, 1)
    gaps, kept = ctx.screen(b, dev(x), dev(d), z, bits)
    assert np.all(kept == 0) and not bits.any().item()
    assert np.all(np.abs(gaps) < 1e-6 * float((x.astype(np.float64) ** 2).sum()))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_code_step_screened_matches_oracle(prec):
    """60 PG iterations with a test every 15 on a ragged 3-image batch (fixed
    step): codes, active sets and the last gaps against the oracle's screened
    step."""
    K, s, H, W, p = 24, 7, [40, 23, 64], [36, 51, 30], (1, 2)
    x, d, ids, rb, cfg = case(K, s, H, W, p, seed=7, frac=0.85)
    step = 1.0 / (1.01 * R.lipschitz_codes(cfg, d, max(H), max(W)))
    zo, mo, gaps_o = R.code_step_screened(cfg, rb, x, d, np.zeros(rb.total_pixels * K), t=1,
                                          n_iters=60, screen_every=15, step=step)
    ctx = scsc.Context(K, s, lam=cfg.lam, p=p, seed=cfg.seed, prec=prec, step=step)
    b = scsc.Batch(H, W, ids=ids)
    z = torch.zeros(rb.total_pixels * K, device="cuda")
    gaps, kept = ctx.code_step_screened(b, dev(x), dev(d), z, 1, 60, 15)
    zg = z.cpu().numpy()
    fo = R.objective(cfg, rb, x, zo, d)
    fg = R.objective(cfg, rb, x, zg, d)
    m0 = R.mask_batch(cfg, rb, 1).ravel()
    if prec == "fp32":
        assert rel_l2(zg, zo) < 1e-4
        assert fg == pytest.approx(fo, rel=1e-5)
        np.testing.assert_allclose(gaps, gaps_o, rtol=1e-3, atol=1e-6 * fo)
        # survivors agree up to coordinates decided inside the rounding band
        assert np.abs(kept - [int(rb.image(mo, n, K).sum()) for n in range(rb.n)]).max() <= 2
    else:
        measured("screen_bf16", rel=rel_l2(zg, zo), jac=support_jaccard(zg, zo))
        # 60 iterations: measured 1.1e-2, identical supports
        assert rel_l2(zg, zo) < 2.5e-2
        assert support_jaccard(zg, zo) >= 0.985
        assert fg == pytest.approx(fo, rel=1e-3)
        assert abs(int(kept.sum()) - int(mo.sum())) <= 0.02 * m0.sum()
    assert mo.sum() < 0.9 * m0.sum()  # the oracle's run removed coordinates
    # Eq. 4 and the removed coordinates: zero codes off the surviving set
    assert not zg[m0 == 0].any()


def test_code_step_screened_zero_iterations_applies_eq4_only():
    K, s, H, W = 8, 5, [20], [20]
    x, d, z0 = make_case(H, W, K, s, seed=2, code_density=0.2)
    ctx = scsc.Context(K, s, lam=0.5, p=(1, 2), seed=1)
    b = scsc.Batch(H, W, ids=[0])
    z = dev(z0)
    ctx.code_step_screened(b, dev(x), dev(d), z, 1, 0, 5)
    m = R.mask_image(R.Config(K=K, s=s, p_num=1, p_den=2, seed=1), 1, 0, 20, 20).ravel()
    np.testing.assert_array_equal(z.cpu().numpy(), np.where(m == 1, z0, 0.0).astype(np.float32))
    with pytest.raises(scsc.ScscError):
        ctx.code_step_screened(b, dev(x), dev(d), z, 1, 5, 0)


def test_c3_full_batch_screened_step_sampled_images():
    """The 64 x 256^2 batch (K = 100, p = 1/4, lambda = 1) in the bench's
    precision: 4 iterations with a test every 2 and a fixed step; two images
    against the oracle's screened step (at this lambda and iteration count the
    gap is far above the level at which the sphere removes coordinates)."""
    wl = bench.WORKLOADS["c3"]
    H, W, ids, x, d = bench.make_inputs(wl, 0)
    K = wl["K"]
    step = 1.0 / 200.0
    ctx = scsc.Context(K, 11, 1.0, wl["p"], seed=0, prec="bf16", step=step)
    b = scsc.Batch(H, W, ids)
    z = torch.zeros(b.total_pixels * K, device="cuda")
    gaps, kept = ctx.code_step_screened(b, dev(x), dev(d), z, 1, 4, 2)
    cfg = R.Config(K=K, s=11, lam=1.0, p_num=wl["p"][0], p_den=wl["p"][1], seed=0)
    rb = R.Batch(H=H, W=W, ids=ids)
    for k in [0, 37]:
        rk = R.Batch(H=[H[k]], W=[W[k]], ids=[ids[k]])
        xk = np.ascontiguousarray(rb.image(x, k))
        zo, mo, go = R.code_step_screened(cfg, rk, xk, d, np.zeros(int(H[k]) * int(W[k]) * K),
                                          t=1, n_iters=4, screen_every=2, step=step)
        zk = z[int(rb.off[k]) * K:(int(rb.off[k]) + int(H[k]) * int(W[k])) * K].cpu().numpy()
        fo = R.objective(cfg, rk, xk, zo, d)
        assert R.objective(cfg, rk, xk, zk, d) == pytest.approx(fo, rel=1e-3)
        assert gaps[k] == pytest.approx(go[0], rel=1e-2)
        assert kept[k] == int(mo.sum())
