"""The allocation-free objective entry point, called through the C ABI.

Callers inside stream capture, or whose memory pool already owns the whole
device, cannot allocate; scsc_objective_noalloc serves them from scratch
built into the library.  Its result must match scsc_objective's on the same
inputs, on two calls in a row (the second call reuses the scratch the first
one left behind), and the FP64 oracle's objective (Eq. 1).  Kept in a file
that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


@pytest.mark.parametrize("K,s,lam,H,W,n", [(24, 11, 0.8, 70, 90, 3), (13, 5, 1.3, 33, 64, 2)])
def test_objective_noalloc_matches_objective_and_oracle_on_two_calls(K, s, lam, H, W, n):
    ctx = scsc.Context(K, s, lam=lam)
    b = scsc.Batch([H] * n, [W] * n)
    ob = R.Batch([H] * n, [W] * n, np.arange(n))
    cfg = R.Config(K, s, lam)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (1, 2):
        x, d, z = make_case([H] * n, [W] * n, K, s, seed=seed, code_density=0.1)
        xt = torch.from_numpy(x).cuda()
        zt = torch.from_numpy(z).cuda()
        dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
        ref = ctx.objective(b, xt, zt, dt)
        scsc.scsc_objective_noalloc(K, s, lam, n, H, W, xt, zt, dt, out)
        torch.cuda.synchronize()
        got = out.item()
        assert got == pytest.approx(ref, rel=1e-6)
        # FP32 synthesis against the FP64 oracle: the FP32 path's bound
        assert got == pytest.approx(R.objective(cfg, ob, x, z, d), rel=1e-5)


def test_objective_noalloc_at_exactly_its_scratch_size():
    # 65,536 tiles of 32 x 32 pixels, the largest batch the scratch holds
    K, s, lam, n, H, W = 1, 1, 0.5, 64, 1024, 1024
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(n * H * W, device="cuda", generator=g)
    z = torch.randn(n * H * W * K, device="cuda", generator=g)
    d = torch.full((K,), 0.75, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    scsc.scsc_objective_noalloc(K, s, lam, n, H, W, x, z, d, out)
    torch.cuda.synchronize()
    # s = 1, K = 1: D z = 0.75 z exactly, so Eq. 1 has a closed form
    r = (0.75 * z.double() - x.double())
    want = 0.5 * float((r * r).sum()) + lam * float(z.double().abs().sum())
    assert out.item() == pytest.approx(want, rel=1e-9)


def test_objective_noalloc_rejects_batches_beyond_its_scratch():
    # called on the C entry point directly: the binding's own buffer checks
    # would reject these 1-element tensors before the library sees them
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros(1, dtype=torch.float32, device="cuda")
    cfg = scsc.scsc_config(4, 3, 1.0, 1, 1, 0, scsc.SCSC_FP32, 0.0, 0)
    st = scsc.lib().scsc_objective_noalloc(ctypes.byref(cfg), 65537, 32, 32, f.data_ptr(),
                                           f.data_ptr(), f.data_ptr(), t.data_ptr(), None)
    assert st == scsc.SCSC_EINVAL
