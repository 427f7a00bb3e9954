"""The allocation-free objective entry point, called through the C ABI.

Callers inside stream capture, or whose memory pool already owns the whole
device, cannot allocate; scsc_objective_noalloc serves them from scratch
built into the library.  Its result must match scsc_objective's on the same
inputs, on two calls in a row (the second call reuses the scratch the first
one left behind).  Kept in a file that pytest collects last.
"""
import numpy as np
import pytest

from tests.helpers import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def test_objective_noalloc_matches_objective_on_two_calls():
    K, s, lam = 24, 11, 0.8
    H, W, n = 70, 90, 3
    ctx = scsc.Context(K, s, lam=lam)
    b = scsc.Batch([H] * n, [W] * n)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (1, 2):
        x, d, z = make_case([H] * n, [W] * n, K, s, seed=seed, code_density=0.1)
        xt = torch.from_numpy(x).cuda()
        zt = torch.from_numpy(z).cuda()
        dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
        ref = ctx.objective(b, xt, zt, dt)
        scsc.scsc_objective_noalloc(K, s, lam, n, H, W, xt, zt, dt, out)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=1e-6)


def test_objective_noalloc_rejects_batches_beyond_its_scratch():
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(scsc.ScscError) as e:
        scsc.scsc_objective_noalloc(4, 3, 1.0, 65537, 32, 32, f, f, f, t)
    assert e.value.status == scsc.SCSC_EINVAL
