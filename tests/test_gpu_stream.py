"""Alg. 2 (SOCSC) as a stream of mini-batches on the GPU, teacher-forced
against the oracle: at every mini-batch the oracle takes the GPU's filters
for the code step (Eq. 3-4) and the GPU's codes and filters for the online
dictionary step (Eq. 7-8), so each step's own error is measured without the
drift of the trajectories."""
import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case, rel_l2, support_jaccard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_alg2_stream_teacher_forced(prec):
    """Three mini-batches of two new images each (the stream's images 0-5),
    K = 12 filters of 7 x 7, p = 1/4, 10 PG iterations per mini-batch."""
    K, s, H, W, p, lam, iters = 12, 7, [30, 26], [34, 40], (1, 4), 0.5, 10
    ctx = scsc.Context(K, s, lam=lam, p=p, seed=21, prec=prec)
    cfg = R.Config(K=K, s=s, lam=lam, p_num=p[0], p_den=p[1], seed=21)
    state = R.OnlineState(cfg)
    _, d0, _ = make_case(H, W, K, s, seed=23)
    dt = dev(d0)
    npx = int(np.sum(np.multiply(H, W)))
    for t in (1, 2, 3):
        ids = [2 * (t - 1), 2 * (t - 1) + 1]
        b = scsc.Batch(H, W, ids=ids)
        rb = R.Batch(H=H, W=W, ids=ids)
        x, _, _ = make_case(H, W, K, s, seed=30 + t)
        xt = dev(x)
        d_now = host(dt).astype(np.float64).ravel()
        # code step from zero codes with the GPU's filters on both sides
        zt = torch.zeros(npx * K, device="cuda")
        ctx.code_step(b, xt, dt, zt, t, iters)
        zo = R.code_step(cfg, rb, x, d_now, np.zeros(npx * K), t, iters)
        zg = host(zt)
        if prec == "fp32":
            assert rel_l2(zg, zo) < 1e-4
        else:
            assert rel_l2(zg, zo) < 1e-2
            assert support_jaccard(zg, zo) >= 0.985
        # online dictionary step from the GPU's codes and filters
        state.update(rb, x, zg)
        d_o = state.dict_step(d_now)
        ctx.dict_step(b, xt, zt, dt, scsc.SCSC_DICT_ONLINE, t)
        assert rel_l2(host(dt), d_o) < 1e-5
        assert np.all(np.linalg.norm(host(dt).reshape(K, -1), axis=1) <= 1 + 1e-6)
