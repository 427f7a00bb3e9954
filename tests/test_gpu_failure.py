"""Failure detection on the GPU without a fault: a bounded wait that nothing
completes (an mbarrier that nothing arrives on) gives up at its limit and
raises an error word that the host reads as SCSC_ETIMEOUT; the device stays
usable for the next call."""
import time

import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    L = scsc.lib()
    assert L.scsc_diag_wait_timeout(0.0) == scsc.SCSC_EINVAL
    t0 = time.perf_counter()
    assert L.scsc_diag_wait_timeout(20.0) == scsc.SCSC_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.02
    # a code step right after, on the tensor path, still matches the oracle
    K, s, H, W = 16, 7, [40], [50]
    x, d, _ = make_case(H, W, K, s, seed=5)
    ctx = scsc.Context(K, s, lam=0.6, p=(1, 2), seed=4, prec="bf16")
    b = scsc.Batch(H, W)
    xt = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    zt = torch.zeros(b.total_pixels * K, device="cuda")
    ctx.code_step(b, xt, dt, zt, 1, 8)
    ctx.sync()
    cfg = R.Config(K=K, s=s, lam=0.6, p_num=1, p_den=2, seed=4)
    rb = R.Batch(H=H, W=W, ids=[0])
    zo = R.code_step(cfg, rb, x, d, np.zeros(b.total_pixels * K), 1, 8)
    assert ctx.objective(b, xt, zt, dt) == pytest.approx(R.objective(cfg, rb, x, zo, d), rel=1e-3)
