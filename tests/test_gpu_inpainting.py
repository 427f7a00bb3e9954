"""Inpainting (Sec. 4.3): the code update with the data term over observed
pixels only, against the oracle; FP32 and BF16 paths; the paper's setting
(50% of pixels observed at random, lambda = 0.4) with and without code
subsampling, on a ragged batch, plus a sampled image of the full-size
inpainting workload (ten 256x256 images, 50 iterations) in the launch
configuration bench.py times."""
import numpy as np
import pytest

import bench
from oracle import reference as R
from paper_1909_00145_gb300 import inputs as I
from tests.helpers import make_case, measured, rel_l2, support_jaccard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("p", [(1, 1), (1, 2)])
def test_observed_code_step_matches_oracle(prec, p):
    K, s, H, W = 24, 11, [64, 40, 30], [140, 64, 30]
    x, d, _ = make_case(H, W, K, s, seed=12)
    npx = int(np.dot(H, W))
    obs = I.observed_pixels(13, npx, 0.5)
    ids = [3, 4, 5]
    cfg = R.Config(K=K, s=s, lam=0.4, p_num=p[0], p_den=p[1], seed=17)
    rb = R.Batch(H=H, W=W, ids=ids)
    zo = R.code_step_observed(cfg, rb, x, d, np.zeros(npx * K), obs, 1, 12)
    ctx = scsc.Context(K, s, lam=0.4, p=p, seed=17, prec=prec)
    b = scsc.Batch(H, W, ids=ids)
    z = torch.zeros(npx * K, device="cuda")
    xt, dt, ot = dev(x), dev(d), dev(obs)
    ctx.code_step_observed(b, xt, dt, z, ot, 1, 12)
    ctx.sync()
    fo = R.objective_observed(cfg, rb, x, zo, d, obs)
    fg = ctx.objective_observed(b, xt, z, dt, ot)
    tol = 1e-5 if prec == "fp32" else 1e-3
    assert fg == pytest.approx(fo, rel=tol)
    zg = z.cpu().numpy()
    measured("inpaint_" + prec, rel=rel_l2(zg, zo), jac=support_jaccard(zg, zo))
    if prec == "fp32":
        assert rel_l2(zg, zo) < 1e-4
    else:
        assert rel_l2(zg, zo) < 1.2e-2  # measured 4.6e-3 .. 5.0e-3
        assert support_jaccard(zg, zo) >= 0.985
    # the unobserved pixels really are out of the data term: the plain
    # objective of the same codes is larger
    assert ctx.objective(b, xt, z, dt) > fg


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_observed_none_is_the_plain_code_step(prec):
    K, s, H, W = 16, 7, [50], [150]
    x, d, _ = make_case(H, W, K, s, seed=2)
    b = scsc.Batch(H, W)
    outs = []
    for observed in (None, "call"):
        ctx = scsc.Context(K, s, lam=0.5, p=(1, 3), seed=4, prec=prec,
                           flags=scsc.SCSC_FLAG_NO_AUTOTUNE)
        z = torch.zeros(H[0] * W[0] * K, device="cuda")
        if observed is None:
            ctx.code_step_observed(b, dev(x), dev(d), z, None, 2, 6)
        else:
            ctx.code_step(b, dev(x), dev(d), z, 2, 6)
        ctx.sync()
        outs.append(z.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_inpainting_workload_sampled_image(prec):
    wl = bench.WORKLOADS["inpaint"]
    H, W, ids, x, d = bench.make_inputs(wl, 0)
    obs = bench.make_observed(wl, 0, H, W)
    K, n_iters = wl["K"], wl["n_iters"]
    step = 1.0 / 200.0
    ctx = scsc.Context(K, 11, wl["lam"], wl["p"], seed=0, prec=prec, step=step,
                       stream=torch.cuda.Stream())
    b = scsc.Batch(H, W, ids)
    z = torch.zeros(b.total_pixels * K, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(ctx.stream):
        ctx.code_step_observed(b, dev(x), dev(d), z, dev(obs), 1, n_iters)
        ctx.sync()
    cfg = R.Config(K=K, s=11, lam=wl["lam"], p_num=wl["p"][0], p_den=wl["p"][1], seed=0)
    rb = R.Batch(H=H, W=W, ids=ids)
    k = 6
    rk = R.Batch(H=[H[k]], W=[W[k]], ids=[ids[k]])
    xk, ok = rb.image(x, k), rb.image(obs, k)
    zo = R.code_step_observed(cfg, rk, xk, d, np.zeros(int(H[k]) * int(W[k]) * K), ok, 1,
                              n_iters, step=step)
    o = int(rb.off[k]) * K
    zk = z[o:o + zo.size].cpu().numpy()
    fo = R.objective_observed(cfg, rk, xk, zo, d, ok)
    fg = R.objective_observed(cfg, rk, xk, zk, d, ok)
    assert fg == pytest.approx(fo, rel=1e-5 if prec == "fp32" else 1e-3)
    measured("inpaint_full_" + prec, rel=rel_l2(zk, zo), jac=support_jaccard(zk, zo))
    if prec == "fp32":
        assert rel_l2(zk, zo) < 1e-4
    else:
        # the longer run drifts further than the 12-iteration case above:
        # measured 1.1e-2, Jaccard 0.995
        assert rel_l2(zk, zo) < 2.5e-2
        assert support_jaccard(zk, zo) >= 0.985
