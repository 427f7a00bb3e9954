"""Parity at the benchmark's full sizes, in the launch configuration that
bench.py times: one library call over the whole batch (persistent tensor
kernels, CUDA-graph replay, autotuned variant).

Code updates are independent per image once the step size is fixed, so the
oracle recomputes sampled images of the full batch one by one:
- the 64 x 256^2 batch (K=100, p=1/4) and the 512-image uneven batch
  (H, W in {64..512}), with a fixed step so that the oracle needs no power
  iteration on the full domain, a few iterations each;
- the sampled images' masks bit-exact and their codes zero off the mask
  (Eq. 4) after the full 100-iteration update with the computed step size;
- batch invariance at full size: an image's codes from the 64-image launch
  equal those of a launch over that image alone, bit for bit;
- the benchmark's own step (64 x 256^2, 100 iterations at the computed
  1/L_z) on two sampled images against the oracle, and the same step teacher-
  forced: the oracle takes the GPU's codes after iteration 50 and performs
  iteration 51, so that the comparison sees one step's arithmetic rather than
  100 steps of drift.
"""
import numpy as np
import pytest

import bench
from oracle import reference as R
from tests.helpers import measured, rel_l2, support_jaccard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402

STEP = 1.0 / 200.0  # a fixed step below 1/L_z of the benchmark filters (L_z = 131.5 on 256 x 256)


def gpu_code_step(wl, H, W, ids, x, d, prec, n_iters, t=1, step=0.0, flags=0):
    K = wl["K"]
    ctx = scsc.Context(K, 11, 1.0, wl["p"], seed=0, prec=prec, step=step, flags=flags,
                       stream=torch.cuda.Stream())
    batch = scsc.Batch(H, W, ids)
    xt = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    z = torch.zeros(batch.total_pixels * K, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(ctx.stream):
        ctx.code_step(batch, xt, dt, z, t, n_iters)
        ctx.sync()
    return ctx, batch, z


def image_codes(z, rb, k, K):
    """Codes of image k of a device code vector, on the host."""
    o = int(rb.off[k]) * K
    return z[o:o + int(rb.H[k]) * int(rb.W[k]) * K].cpu().numpy()


def oracle_image(wl, H, W, ids, x, d, k, n_iters, t=1):
    K = wl["K"]
    cfg = R.Config(K=K, s=11, lam=1.0, p_num=wl["p"][0], p_den=wl["p"][1], seed=0)
    rb = R.Batch(H=H, W=W, ids=ids)
    rk = R.Batch(H=[H[k]], W=[W[k]], ids=[ids[k]])
    xk = np.ascontiguousarray(rb.image(x, k))
    zk = R.code_step(cfg, rk, xk, d, np.zeros(int(H[k]) * int(W[k]) * K), t, n_iters, step=STEP)
    return cfg, rb, rk, xk, zk


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("name,sample,n_iters", [("c3", [0, 37], 4), ("c5", [5, 300], 3)])
def test_full_batch_sampled_images_match_oracle(name, sample, n_iters, prec):
    wl = bench.WORKLOADS[name]
    H, W, ids, x, d = bench.make_inputs(wl, 0)
    _, _, zg = gpu_code_step(wl, H, W, ids, x, d, prec, n_iters, step=STEP)
    K = wl["K"]
    for k in sample:
        cfg, rb, rk, xk, zo = oracle_image(wl, H, W, ids, x, d, k, n_iters)
        zk = image_codes(zg, rb, k, K)
        fo = R.objective(cfg, rk, xk, zo, d)
        fg = R.objective(cfg, rk, xk, zk, d)
        if prec == "fp32":
            assert fg == pytest.approx(fo, rel=1e-5), (k, fg, fo)
            assert rel_l2(zk, zo) < 1e-4
        else:
            measured(f"full_{name}_{k}", rel=rel_l2(zk, zo), jac=support_jaccard(zk, zo),
                     obj=abs(fg - fo) / abs(fo))
            assert fg == pytest.approx(fo, rel=1e-3), (k, fg, fo)
            # measured 4.9e-3 .. 5.3e-3 and Jaccard >= 0.994 on these images
            assert rel_l2(zk, zo) < 1.2e-2
            assert support_jaccard(zk, zo) >= 0.985


def test_c3_full_update_masks_and_eq4_zeros():
    wl = bench.WORKLOADS["c3"]
    H, W, ids, x, d = bench.make_inputs(wl, 0)
    ctx, batch, zg = gpu_code_step(wl, H, W, ids, x, d, "bf16", wl["n_iters"], t=3)
    K, kw = wl["K"], (wl["K"] + 31) // 32
    bits = ctx.mask(batch, 3).cpu().numpy().view(np.uint32).reshape(-1, kw)
    cfg = R.Config(K=K, s=11, lam=1.0, p_num=wl["p"][0], p_den=wl["p"][1], seed=0)
    rb = R.Batch(H=H, W=W, ids=ids)
    for k in [0, 21, 63]:
        mo = R.mask_image(cfg, 3, int(ids[k]), int(H[k]), int(W[k])).reshape(-1, K)
        o, npx = int(rb.off[k]), int(H[k]) * int(W[k])
        words = bits[o:o + npx]
        mg = ((words[:, np.arange(K) // 32] >> (np.arange(K) % 32).astype(np.uint32)) & 1)
        assert np.array_equal(mg.astype(np.uint8), mo)
        zk = image_codes(zg, rb, k, K).reshape(-1, K)
        assert not zk[mo == 0].any()
        assert np.isfinite(zk).all() and zk.any()


def test_c3_batch_invariance_bit_exact():
    """The 64-image launch (bench's configuration) and a launch over one of
    its images alone give that image the same codes: every row item's
    arithmetic is independent of how items are spread over the CTAs."""
    wl = bench.WORKLOADS["c3"]
    H, W, ids, x, d = bench.make_inputs(wl, 0)
    _, batch, zg = gpu_code_step(wl, H, W, ids, x, d, "bf16", wl["n_iters"], t=2)
    k = 37
    rb = R.Batch(H=H, W=W, ids=ids)
    xk = np.ascontiguousarray(rb.image(x, k))
    _, _, z1 = gpu_code_step(wl, H[k:k + 1], W[k:k + 1], ids[k:k + 1], xk, d, "bf16",
                             wl["n_iters"], t=2, flags=scsc.SCSC_FLAG_NO_AUTOTUNE)
    assert np.array_equal(image_codes(zg, rb, k, wl["K"]), z1.cpu().numpy())


def test_c3_benchmark_step_against_oracle_and_teacher_forced():
    wl = bench.WORKLOADS["c3"]
    H, W, ids, x, d = bench.make_inputs(wl, 0)
    K, n_iters, sample = wl["K"], wl["n_iters"], [0, 37]
    cfg = R.Config(K=K, s=11, lam=1.0, p_num=wl["p"][0], p_den=wl["p"][1], seed=0)
    rb = R.Batch(H=H, W=W, ids=ids)
    rk = R.Batch(H=[H[k] for k in sample], W=[W[k] for k in sample], ids=[ids[k] for k in sample])
    xk = np.concatenate([rb.image(x, k) for k in sample])
    # the step both sides compute: 1/L_z of the 256 x 256 domain
    alpha_o = 1.0 / R.lipschitz_codes(cfg, d, int(H[0]), int(W[0]))
    ctx = scsc.Context(K, 11, 1.0, wl["p"], seed=0, prec="bf16", stream=torch.cuda.Stream())
    batch = scsc.Batch(H, W, ids)
    xt = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    alpha_g = 1.0 / ctx.lipschitz_codes(batch, dt)
    assert alpha_g == pytest.approx(alpha_o, rel=1e-4)

    def gpu(z, its):
        torch.cuda.synchronize()
        with torch.cuda.stream(ctx.stream):
            ctx.code_step(batch, xt, dt, z, 1, its)
            ctx.sync()
        return z

    def sampled(z):
        return np.concatenate([image_codes(z, rb, k, K) for k in sample])

    # the whole benchmark step from zero codes
    zg = sampled(gpu(torch.zeros(batch.total_pixels * K, device="cuda"), n_iters))
    zo = R.code_step(cfg, rk, xk, d, np.zeros(zg.size), 1, n_iters, step=alpha_o)
    fo, fg = R.objective(cfg, rk, xk, zo, d), R.objective(cfg, rk, xk, zg, d)
    measured("c3_step100", rel=rel_l2(zg, zo), jac=support_jaccard(zg, zo), obj=abs(fg - fo) / abs(fo))
    assert fg == pytest.approx(fo, rel=1e-3)
    # after 100 iterations the two paths have drifted apart along the
    # lasso's flat directions (measured 2.7e-2, objective 3.4e-5, support
    # Jaccard 0.996); one step from the same state is the tight check below
    assert rel_l2(zg, zo) < 5.5e-2
    assert support_jaccard(zg, zo) >= 0.99
    # teacher forcing: both sides take iteration 51 from the GPU's codes after 50
    z50 = gpu(torch.zeros(batch.total_pixels * K, device="cuda"), n_iters // 2)
    z50_k = sampled(z50)
    z51g = sampled(gpu(z50.clone(), 1))
    z51o = R.code_step(cfg, rk, xk, d, z50_k, 1, 1, step=alpha_o)
    measured("c3_teacher51", rel=rel_l2(z51g, z51o), jac=support_jaccard(z51g, z51o),
             moved=rel_l2(z51o, z50_k))
    # one BF16 iteration: measured 1.7e-3 (the step itself moves the codes by
    # 1.1e-2), identical supports
    assert rel_l2(z51g, z51o) < 4e-3
    assert support_jaccard(z51g, z51o) >= 0.995
    ctx.close()
