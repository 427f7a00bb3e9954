"""Boundary behaviour of the C ABI on the GPU: non-finite inputs are reported
as SCSC_ENONFINITE at the next synchronising call (no trap, the context stays
usable), and the variant of Sec. 3.1 that keeps the unsampled codes
(SCSC_FLAG_UNSAMPLED_KEEP) matches the oracle's variant."""
import numpy as np
import pytest

from oracle import reference as R
from tests.helpers import make_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1909_00145_gb300 import scsc  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("where", ["x", "z", "d"])
def test_nonfinite_input_is_reported_and_cleared(prec, where):
    K, s, H, W = 12, 5, [30, 20], [70, 140]
    x, d, z = make_case(H, W, K, s, seed=3, code_density=0.1)
    bad = {"x": x.copy(), "z": z.copy(), "d": d.copy()}
    bad[where].ravel()[7] = np.nan if where != "d" else np.inf
    ctx = scsc.Context(K, s, p=(1, 2), seed=1, prec=prec)
    b = scsc.Batch(H, W)
    zt = dev(bad["z"])
    ctx.code_step(b, dev(bad["x"]), dev(bad["d"]), zt, 1, 3)
    with pytest.raises(scsc.ScscError) as e:
        ctx.sync()
    assert e.value.status == scsc.SCSC_ENONFINITE
    ctx.sync()  # reported once, then cleared
    # the context still works: a clean step matches the oracle
    zt = dev(z)
    ctx.code_step(b, dev(x), dev(d), zt, 1, 3)
    ctx.sync()
    cfg = R.Config(K=K, s=s, lam=1.0, p_num=1, p_den=2, seed=1)
    rb = R.Batch(H=H, W=W, ids=[0, 1])
    zo = R.code_step(cfg, rb, x, d, z, 1, 3)
    tol = 1e-5 if prec == "fp32" else 1e-3
    assert ctx.objective(b, dev(x), zt, dev(d)) == pytest.approx(R.objective(cfg, rb, x, zo, d),
                                                                  rel=tol)


def test_nonfinite_input_to_the_objective_is_returned_by_it():
    K, s, H, W = 6, 3, [16], [24]
    x, d, z = make_case(H, W, K, s, seed=4, code_density=0.2)
    z[5] = np.inf
    ctx = scsc.Context(K, s)
    b = scsc.Batch(H, W)
    with pytest.raises(scsc.ScscError) as e:
        ctx.objective(b, dev(x), dev(z), dev(d))
    assert e.value.status == scsc.SCSC_ENONFINITE


@pytest.mark.parametrize("prec,tol_z", [("fp32", 1e-4), ("bf16", 2e-2)])
@pytest.mark.parametrize("p", [(1, 3), (1, 1)])
def test_unsampled_keep_variant_matches_the_oracle(prec, tol_z, p):
    K, s, H, W = 20, 7, [37, 24], [131, 60]
    x, d, z0 = make_case(H, W, K, s, seed=9, code_density=0.15)
    ids = [3, 4]
    ctx = scsc.Context(K, s, lam=0.6, p=p, seed=5, prec=prec, flags=scsc.SCSC_FLAG_UNSAMPLED_KEEP)
    b = scsc.Batch(H, W, ids)
    zt = dev(z0)
    ctx.code_step(b, dev(x), dev(d), zt, 2, 10)
    ctx.sync()
    zg = zt.cpu().numpy()
    cfg = R.Config(K=K, s=s, lam=0.6, p_num=p[0], p_den=p[1], seed=5)
    rb = R.Batch(H=H, W=W, ids=ids)
    zo = R.code_step(cfg, rb, x, d, z0, 2, 10, keep=True)
    m = R.mask_batch(cfg, rb, 2).astype(bool)
    # codes off the sampled set are returned exactly as they came in
    assert np.array_equal(zg[~m], z0[~m])
    assert rel_l2(zg[m], zo[m]) < tol_z
    fo = R.objective(cfg, rb, x, zo, d)
    assert ctx.objective(b, dev(x), zt, dev(d)) == pytest.approx(
        fo, rel=1e-5 if prec == "fp32" else 1e-3)
    if p == (1, 1):
        # every coordinate sampled: the same update as Eq. 4's
        ze = R.code_step(cfg, rb, x, d, z0, 2, 10)
        assert rel_l2(zo, ze) < 1e-12
