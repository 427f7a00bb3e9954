"""Outer iterations of Alg. 1 on the GPU against the oracle, with the filters
updated in place between code steps: the code step's step size (stencils and
power iteration, replayed from a cached CUDA graph keyed by the filter
pointer) must follow the new filters."""
import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_step_size_follows_filters_updated_in_place():
    """L_z of 2d is 4 L_z of d, bit for bit (scaling by 2 is exact in every
    step of the stencil build and the power iteration), with the same device
    buffer rescaled in place between the two calls."""
    K, s, H, W = 16, 11, [70], [90]
    _, d, _ = make_case(H, W, K, s, seed=2)
    ctx = scsc.Context(K, s, seed=5)
    b = scsc.Batch(H, W)
    dt = dev(d)
    l1 = ctx.lipschitz_codes(b, dt)
    dt.mul_(2.0)
    l2 = ctx.lipschitz_codes(b, dt)
    assert l2 == 4.0 * l1
    cfg = R.Config(K=K, s=s, seed=5)
    assert l1 == pytest.approx(R.lipschitz_codes(cfg, d, H[0], W[0]), rel=2e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_two_outer_iterations_of_alg1(prec):
    """t = 1, 2: code step (computed step size) then the batch dictionary
    step, the filters overwritten in place; objective after each step."""
    K, s, H, W, p = 12, 7, [40, 29], [36, 51], (1, 2)
    x, d0, _ = make_case(H, W, K, s, seed=4)
    ctx = scsc.Context(K, s, lam=0.5, p=p, seed=9, prec=prec)
    b = scsc.Batch(H, W)
    xt, dt = dev(x), dev(d0)
    zt = torch.zeros(b.total_pixels * K, device="cuda")
    cfg = R.Config(K=K, s=s, lam=0.5, p_num=p[0], p_den=p[1], seed=9)
    rb = R.Batch(H=H, W=W, ids=[0, 1])
    zo, do = np.zeros(rb.total_pixels * K), d0.astype(np.float64).ravel()
    tol = 1e-5 if prec == "fp32" else 1e-3
    for t in (1, 2):
        ctx.code_step(b, xt, dt, zt, t, 15)
        zo = R.code_step(cfg, rb, x, do, zo, t, 15)
        assert ctx.objective(b, xt, zt, dt) == pytest.approx(R.objective(cfg, rb, x, zo, do),
                                                             rel=tol)
        ctx.dict_step(b, xt, zt, dt, scsc.SCSC_DICT_BATCH, t)
        # the oracle's dictionary step from the GPU's codes (teacher forcing),
        # so that only this step's error is measured
        do = R.dict_step_batch(cfg, rb, x, zt.cpu().numpy(), do)
        if prec == "fp32":
            assert rel_l2(dt.cpu().numpy(), do) < 1e-4
        else:
            assert rel_l2(dt.cpu().numpy(), do) < 1e-2
        do = dt.cpu().numpy().astype(np.float64).ravel()
        zo = zt.cpu().numpy().astype(np.float64)
