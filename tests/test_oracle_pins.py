"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, a published test vector,
a library routine (scipy.signal convolution, numpy eigvalsh, scipy optimize),
brute force on tiny inputs, or an invariant the paper states.  CPU only.
"""
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.signal

from oracle import reference as R
from paper_1909_00145_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def explicit_synthesis_matrix(d, H, W):
    """A (H*W x H*W*K) with A z = sum_k d_k * z_k, columns built by
    scipy.signal.convolve2d(mode='same') of unit code images."""
    K, s, _ = d.shape
    A = np.zeros((H * W, H * W * K))
    for y in range(H):
        for x in range(W):
            e = np.zeros((H, W))
            e[y, x] = 1.0
            for k in range(K):
                A[:, (y * W + x) * K + k] = scipy.signal.convolve2d(e, d[k], mode="same").ravel()
    return A


def explicit_code_matrix(z, K, s, H, W):
    """Z (H*W x K*s*s) with Z d = sum_k d_k * z_k, columns from unit filters."""
    zz = z.reshape(H, W, K)
    Z = np.zeros((H * W, K * s * s))
    for k in range(K):
        for u in range(s):
            for v in range(s):
                e = np.zeros((s, s))
                e[u, v] = 1.0
                Z[:, k * s * s + u * s + v] = scipy.signal.convolve2d(zz[:, :, k], e, mode="same").ravel()
    return Z


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ hash / mask

def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for inp, out in rows:
        assert R.splitmix64(int(inp, 16)) == int(out, 16)


def test_mask_key_order_golden_value():
    """The hash chain's key order (seed, then t, then n, then the coordinate
    index) and the strict threshold test, against a value derived from the
    published SplitMix64 vectors (derivation in the fixture)."""
    kv = dict(l.split() for l in open(os.path.join(GOLDEN, "mask_key_order.txt"))
              if l.strip() and not l.startswith("#"))
    seed, t, n = int(kv["seed"], 16), int(kv["t"], 16), int(kv["n"], 16)
    H, W, k, y, x = (int(kv[c]) for c in "HWkyx")
    hi = int(kv["hash"], 16) >> 32
    K = 2
    for p_num, want in ((hi, 0), (hi + 1, 1)):
        cfg = R.Config(K=K, p_num=p_num, p_den=2**32 - 1, seed=seed)
        m = R.mask_image(cfg, t, n, H, W)
        assert m[y, x, k] == want, (p_num, want)


def test_mask_p_one_is_identity_and_p_zero_is_empty():
    # Sec. 3.1: p = 1 makes M^t the identity.
    full = R.mask_image(R.Config(K=7, p_num=1, p_den=1, seed=5), 3, 11, 9, 13)
    assert full.all()
    none = R.mask_image(R.Config(K=7, p_num=0, p_den=1, seed=5), 3, 11, 9, 13)
    assert not none.any()


@pytest.mark.parametrize("p_num,p_den", [(1, 4), (1, 2), (1, 10), (3, 7)])
def test_mask_bernoulli_rate_within_5_sigma(p_num, p_den):
    cfg = R.Config(K=16, p_num=p_num, p_den=p_den, seed=123)
    m = R.mask_image(cfg, 1, 0, 64, 64)
    n = m.size
    p = p_num / p_den
    assert abs(m.mean() - p) <= 5 * np.sqrt(p * (1 - p) / n)
    # independence across filters: the per-filter rates agree with p too
    per_k = m.reshape(-1, 16).mean(axis=0)
    assert np.all(np.abs(per_k - p) <= 5 * np.sqrt(p * (1 - p) / (n / 16)))


def test_mask_is_fresh_per_iteration_and_per_image():
    cfg = R.Config(K=8, p_num=1, p_den=2, seed=9)
    a = R.mask_image(cfg, 1, 0, 20, 20)
    b = R.mask_image(cfg, 2, 0, 20, 20)
    c = R.mask_image(cfg, 1, 1, 20, 20)
    d = R.mask_image(R.Config(K=8, p_num=1, p_den=2, seed=10), 1, 0, 20, 20)
    for other in (b, c, d):
        agree = (a == other).mean()
        assert 0.4 < agree < 0.6  # independent Bernoulli(1/2) masks agree half the time
    assert np.array_equal(a, R.mask_image(cfg, 1, 0, 20, 20))  # deterministic


# ------------------------------------------------------------------ operators

def test_delta_filter_reproduces_codes():
    """K=1 and d = delta at the centre: D = I, so D z = z, D^T r = r,
    lambda_max(D D^T) = 1, and one PG step from 0 is soft(alpha x, alpha lam)."""
    s, H, W = 11, 17, 23
    d = np.zeros((1, s, s))
    d[0, 5, 5] = 1.0
    z = rng(1).normal(size=H * W)
    assert np.array_equal(R.synthesis(d, z, 1, s, H, W), z)
    assert np.array_equal(R.adjoint(d, z, 1, s, H, W), z)
    cfg = R.Config(K=1, s=s, lam=0.3, p_num=1, p_den=2, seed=4)
    assert R.lipschitz_codes(cfg, d, H, W) == pytest.approx(1.01, rel=1e-14)
    x = I.images(3, [H], [W]).astype(np.float64)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    znew = R.code_step(cfg, batch, x, d, np.zeros(H * W), t=1, n_iters=1)
    m = R.mask_image(cfg, 1, 0, H, W).ravel().astype(bool)
    alpha = 1.0 / 1.01
    expect = np.where(m, np.sign(x) * np.maximum(np.abs(alpha * x) - alpha * 0.3, 0.0), 0.0)
    np.testing.assert_allclose(znew, expect, rtol=0, atol=1e-14)


def test_shifted_deltas_fix_index_conventions():
    """d_0 = delta at (c+1, c), d_1 = delta at (c, c+2): the synthesis is z_0
    shifted down one row plus z_1 shifted right two columns, zero filled."""
    s, H, W, c = 11, 9, 12, 5
    d = np.zeros((2, s, s))
    d[0, c + 1, c] = 1.0
    d[1, c, c + 2] = 1.0
    z = rng(2).normal(size=H * W * 2).reshape(H, W, 2)
    expect = np.zeros((H, W))
    expect[1:, :] += z[:-1, :, 0]
    expect[:, 2:] += z[:, :-2, 1]
    np.testing.assert_array_equal(R.synthesis(d, z.ravel(), 2, s, H, W).reshape(H, W), expect)


@pytest.mark.parametrize("K,s,H,W", [(3, 5, 13, 17), (2, 11, 9, 14), (4, 3, 6, 5)])
def test_operators_match_scipy_convolution(K, s, H, W):
    d = I.filters(7, K, s).astype(np.float64)
    z = rng(3).normal(size=H * W * K)
    r = rng(4).normal(size=H * W)
    zz = z.reshape(H, W, K)
    conv = sum(scipy.signal.convolve2d(zz[:, :, k], d[k], mode="same") for k in range(K))
    np.testing.assert_allclose(R.synthesis(d, z, K, s, H, W), conv.ravel(), rtol=0, atol=1e-13)
    corr = np.stack([scipy.signal.correlate2d(r.reshape(H, W), d[k], mode="same")
                     for k in range(K)], axis=-1)
    np.testing.assert_allclose(R.adjoint(d, r, K, s, H, W), corr.ravel(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("K,s,H,W", [(3, 5, 13, 17), (5, 11, 20, 16)])
def test_adjoint_identities(K, s, H, W):
    """<Dz, r> = <z, D^T r> and <Z d, r> = <d, Z^T r> (synthesis is bilinear)."""
    d = rng(5).normal(size=K * s * s)
    z = rng(6).normal(size=H * W * K)
    r = rng(7).normal(size=H * W)
    lhs = np.dot(R.synthesis(d, z, K, s, H, W), r)
    assert abs(lhs - np.dot(z, R.adjoint(d, r, K, s, H, W))) <= 1e-13 * max(1.0, abs(lhs))
    assert abs(lhs - np.dot(d, R.filter_gradient(r, z, K, s, H, W))) <= 1e-13 * max(1.0, abs(lhs))


@pytest.mark.parametrize("K,s,H,W,p", [(3, 5, 13, 17, 0.25), (5, 11, 20, 16, 0.1),
                                       (4, 3, 2, 9, 1.0), (2, 7, 6, 5, 0.0)])
def test_adjoint_at_sampled_coordinates(K, s, H, W, p):
    """The gradient of Eq. 3 in its sampled variables: the explicit matrix's
    rows A^T r at the sampled coordinates, bit for bit the dense adjoint's
    values there, and nothing written elsewhere."""
    d = rng(11).normal(size=K * s * s)
    r = rng(12).normal(size=H * W)
    mask = (rng(13).random(H * W * K) < p).astype(np.uint8)
    g = R.adjoint_sampled(d, r, mask, K, s, H, W)
    on = mask.astype(bool)
    assert np.array_equal(g[on], R.adjoint(d, r, K, s, H, W)[on])
    assert np.all(np.isnan(g[~on]))
    if H * W <= 64:
        A = explicit_synthesis_matrix(d.reshape(K, s, s), H, W)
        np.testing.assert_allclose(g[on], (A.T @ r)[on], atol=1e-13)


def test_brute_force_8x8_operators_and_lipschitz():
    K, s, H, W = 2, 5, 8, 8
    d = I.filters(1, K, s).astype(np.float64)
    A = explicit_synthesis_matrix(d, H, W)
    z = rng(8).normal(size=H * W * K)
    r = rng(9).normal(size=H * W)
    np.testing.assert_allclose(R.synthesis(d, z, K, s, H, W), A @ z, atol=1e-13)
    np.testing.assert_allclose(R.adjoint(d, r, K, s, H, W), A.T @ r, atol=1e-13)
    Z = explicit_code_matrix(z, K, s, H, W)
    np.testing.assert_allclose(Z @ d.ravel(), A @ z, atol=1e-13)
    np.testing.assert_allclose(R.filter_gradient(r, z, K, s, H, W), Z.T @ r, atol=1e-13)
    # power iteration: Rayleigh quotient never exceeds lambda_max, and is close
    lam = np.linalg.eigvalsh(A @ A.T).max()
    cfg = R.Config(K=K, s=s, seed=3)
    est = R.lipschitz_codes(cfg, d, H, W) / 1.01
    assert est <= lam * (1 + 1e-12)
    assert est >= 0.99 * lam
    batch = R.Batch(H=[H], W=[W], ids=[0])
    lz = np.linalg.eigvalsh(Z.T @ Z).max()
    estd = R.lipschitz_filters(cfg, batch, z) / 1.01
    assert lz * 0.95 <= estd <= lz * (1 + 1e-12)


def test_brute_force_8x8_kkt_after_many_pg_steps():
    """Eq. 3 is a LASSO over the sampled coordinates: after many proximal
    gradient steps the KKT conditions hold, checked with the explicit A."""
    K, s, H, W = 2, 5, 8, 8
    lam = 0.05
    d = I.filters(1, K, s).astype(np.float64)
    x = I.images(2, [H], [W]).astype(np.float64)
    cfg = R.Config(K=K, s=s, lam=lam, p_num=1, p_den=2, seed=21)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    z = R.code_step(cfg, batch, x, d, np.zeros(H * W * K), t=1, n_iters=20000)
    A = explicit_synthesis_matrix(d, H, W)
    m = R.mask_image(cfg, 1, 0, H, W).ravel().astype(bool)
    g = A.T @ (A @ z - x)
    assert np.all(z[~m] == 0)
    nz = m & (z != 0)
    zero = m & (z == 0)
    assert nz.sum() > 0
    np.testing.assert_allclose(g[nz], -lam * np.sign(z[nz]), atol=1e-9)
    assert np.all(np.abs(g[zero]) <= lam + 1e-9)


def test_subsampled_pg_matches_explicit_matrix_pg():
    """p = 1 (M = I) gives plain PG on the full LASSO; p < 1 gives PG on the
    sampled columns of A (Eq. 3), both written here with the explicit A."""
    K, s, H, W = 3, 5, 8, 9
    d = I.filters(11, K, s).astype(np.float64)
    x = I.images(12, [H], [W]).astype(np.float64)
    A = explicit_synthesis_matrix(d, H, W)
    batch = R.Batch(H=[H], W=[W], ids=[4])
    alpha = 1.0 / (1.01 * np.linalg.eigvalsh(A @ A.T).max())
    z0 = rng(13).normal(size=H * W * K) * 0.1
    for p_num, p_den in [(1, 1), (1, 3)]:
        cfg = R.Config(K=K, s=s, lam=0.02, p_num=p_num, p_den=p_den, seed=2)
        got = R.code_step(cfg, batch, x, d, z0, t=5, n_iters=30, step=alpha)
        m = R.mask_image(cfg, 5, 4, H, W).ravel().astype(bool)
        z = np.where(m, z0, 0.0)
        for _ in range(30):
            v = z - alpha * (A.T @ (A @ z - x))
            z = np.where(m, np.sign(v) * np.maximum(np.abs(v) - alpha * cfg.lam, 0.0), 0.0)
        np.testing.assert_allclose(got, z, rtol=0, atol=1e-12)
        if p_num == p_den:
            assert m.all()


def test_keep_variant_matches_explicit_matrix_pg_with_fixed_unsampled_codes():
    """Sec. 3.1's other reading: the unsampled codes remain unchanged and the
    sampled ones take proximal-gradient steps on the full residual, written
    here with the explicit A; p = 1 is the Eq. 4 update and p = 0 leaves the
    codes as they are."""
    K, s, H, W = 3, 5, 8, 9
    d = I.filters(21, K, s).astype(np.float64)
    x = I.images(22, [H], [W]).astype(np.float64)
    A = explicit_synthesis_matrix(d, H, W)
    batch = R.Batch(H=[H], W=[W], ids=[6])
    alpha = 1.0 / (1.01 * np.linalg.eigvalsh(A @ A.T).max())
    z0 = rng(23).normal(size=H * W * K) * 0.1
    cfg = R.Config(K=K, s=s, lam=0.03, p_num=1, p_den=3, seed=4)
    got = R.code_step(cfg, batch, x, d, z0, t=2, n_iters=25, step=alpha, keep=True)
    m = R.mask_image(cfg, 2, 6, H, W).ravel().astype(bool)
    z = z0.copy()
    for _ in range(25):
        v = z - alpha * (A.T @ (A @ z - x))
        z = np.where(m, np.sign(v) * np.maximum(np.abs(v) - alpha * cfg.lam, 0.0), z)
    np.testing.assert_allclose(got, z, rtol=0, atol=1e-12)
    assert np.array_equal(got[~m], z0[~m]) and (~m).sum() > 0
    # the same sampled codes as the Eq. 4 update on x' = x - D z_{not S}
    z_off = np.where(m, 0.0, z0)
    eq4 = R.code_step(cfg, batch, x - A @ z_off, d, z0, t=2, n_iters=25, step=alpha)
    np.testing.assert_allclose(got[m], eq4[m], rtol=0, atol=1e-12)
    full = R.Config(K=K, s=s, lam=0.03, p_num=1, p_den=1, seed=4)
    assert np.array_equal(R.code_step(full, batch, x, d, z0, 2, 7, step=alpha, keep=True),
                          R.code_step(full, batch, x, d, z0, 2, 7, step=alpha))
    none = R.Config(K=K, s=s, lam=0.03, p_num=0, p_den=1, seed=4)
    assert np.array_equal(R.code_step(none, batch, x, d, z0, 2, 7, step=alpha, keep=True), z0)


# ------------------------------------------------------------------ prox / projection

def test_soft_threshold_is_the_prox_of_the_l1_norm():
    tau = 0.7
    for v in np.concatenate([np.linspace(-3, 3, 61), [tau, -tau, 0.0]]):
        got = R.soft_threshold(float(v), tau)
        res = scipy.optimize.minimize_scalar(lambda w: 0.5 * (w - v) ** 2 + tau * abs(w),
                                             bounds=(-5, 5), method="bounded",
                                             options={"xatol": 1e-12})
        assert abs(got - res.x) <= 1e-6
    assert R.soft_threshold(tau, tau) == 0.0 and R.soft_threshold(-tau, tau) == 0.0
    assert R.soft_threshold(2.0, tau) == pytest.approx(1.3, abs=1e-15)


def test_unit_ball_projection():
    K, M = 6, 25
    v = rng(14).normal(size=K * M) * np.repeat([0.1, 0.5, 1.0, 2.0, 10.0, 0.0], M)
    p = R.project_filters(v, K, M)
    norms = np.linalg.norm(p.reshape(K, M), axis=1)
    assert np.all(norms <= 1 + 1e-15)
    np.testing.assert_array_equal(R.project_filters(p, K, M), p)  # idempotent
    vin = v.reshape(K, M)
    for k in range(K):
        nk = np.linalg.norm(vin[k])
        if nk <= 1:
            np.testing.assert_array_equal(p.reshape(K, M)[k], vin[k])
        else:
            np.testing.assert_allclose(p.reshape(K, M)[k], vin[k] / nk, rtol=1e-15)
            # the projection is the closest point of the ball
            w = rng(15).normal(size=(200, M))
            w /= np.maximum(1.0, np.linalg.norm(w, axis=1, keepdims=True))
            assert np.linalg.norm(vin[k] - p.reshape(K, M)[k]) <= np.min(
                np.linalg.norm(w - vin[k], axis=1)) + 1e-12


# ------------------------------------------------------------------ gradients

def test_finite_difference_gradients_of_the_data_term():
    """D^T r and Z^T r are the gradients of 0.5 ||Dz - x||^2 in z and d."""
    K, s, H, W = 3, 5, 7, 9
    d = rng(16).normal(size=K * s * s)
    z = rng(17).normal(size=H * W * K)
    x = rng(18).normal(size=H * W)

    def f(dd, zz):
        r = R.synthesis(dd, zz, K, s, H, W) - x
        return 0.5 * np.dot(r, r)

    r = R.synthesis(d, z, K, s, H, W) - x
    gz = R.adjoint(d, r, K, s, H, W)
    gd = R.filter_gradient(r, z, K, s, H, W)
    pick = rng(19)
    for i in pick.choice(z.size, 20, replace=False):
        h = 1e-6 * max(1.0, abs(z[i]))
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        assert (f(d, zp) - f(d, zm)) / (2 * h) == pytest.approx(gz[i], rel=1e-6, abs=1e-6)
    for i in pick.choice(d.size, 20, replace=False):
        h = 1e-6 * max(1.0, abs(d[i]))
        dp, dm = d.copy(), d.copy()
        dp[i] += h
        dm[i] -= h
        assert (f(dp, z) - f(dm, z)) / (2 * h) == pytest.approx(gd[i], rel=1e-6, abs=1e-6)


# ------------------------------------------------------------------ solvers

def test_admm_and_pg_reach_the_same_lasso_optimum():
    """Eq. 3 is a standard LASSO: the paper's ADMM (rho = 10 lambda,
    alpha = 1.8, CG inner solve) and proximal gradient agree at convergence."""
    K, s, H, W = 2, 3, 10, 10
    cfg = R.Config(K=K, s=s, lam=0.2, p_num=1, p_den=2, seed=31)
    d = I.filters(5, K, s).astype(np.float64)
    x = I.images(6, [H], [W]).astype(np.float64)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    m = R.mask_image(cfg, 1, 0, H, W)
    z_pg = R.code_step(cfg, batch, x, d, np.zeros(H * W * K), t=1, n_iters=20000)
    z_admm = R.admm_image(cfg, d, x, np.zeros(H * W * K), m, H, W, n_iters=400, cg_iters=500)
    f_pg = R.objective(cfg, batch, x, z_pg, d)
    f_admm = R.objective(cfg, batch, x, z_admm, d)
    assert f_pg == pytest.approx(f_admm, rel=1e-8)
    np.testing.assert_allclose(z_pg, z_admm, atol=1e-5)


def test_objective_is_monotone_over_pg_and_dict_steps():
    K, s, H, W = 4, 7, 24, 20
    cfg = R.Config(K=K, s=s, lam=0.5, p_num=1, p_den=2, seed=8)
    d = I.filters(3, K, s)
    x = I.images(4, [H], [W])
    batch = R.Batch(H=[H], W=[W], ids=[0])
    z = np.zeros(H * W * K)
    f_prev = R.objective(cfg, batch, x, z, d)
    for it in range(15):
        # re-entering with the same t keeps M^t, so this continues PG
        z = R.code_step(cfg, batch, x, d, z, t=1, n_iters=1)
        f = R.objective(cfg, batch, x, z, d)
        assert f <= f_prev * (1 + 1e-14)
        f_prev = f
    d2 = R.dict_step_batch(cfg, batch, x, z, d)
    assert R.objective(cfg, batch, x, z, d2) <= f_prev * (1 + 1e-14)
    assert np.all(np.linalg.norm(d2.reshape(K, -1), axis=1) <= 1 + 1e-15)


def test_dict_step_with_all_zero_codes_keeps_filters():
    K, s, H, W = 3, 5, 6, 6
    cfg = R.Config(K=K, s=s)
    d = I.filters(1, K, s).astype(np.float64)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    x = I.images(1, [H], [W])
    assert R.lipschitz_filters(cfg, batch, np.zeros(H * W * K)) == 0.0
    np.testing.assert_array_equal(R.dict_step_batch(cfg, batch, x, np.zeros(H * W * K), d),
                                  d.ravel())


# ------------------------------------------------------------------ online surrogates

def test_online_surrogates_match_batch_gradient_and_explicit_matrix():
    """Eq. 7 at t = 1 with one image: C d - B = Z^T (Z d - x), the batch
    filter gradient; C = Z^T Z with the explicit Z, symmetric PSD."""
    K, s, H, W = 2, 5, 9, 8
    cfg = R.Config(K=K, s=s, lam=0.1, seed=3)
    d = I.filters(2, K, s).astype(np.float64).ravel()
    x = I.images(3, [H], [W]).astype(np.float64)
    z = I.sparse_codes(4, H * W, K, density=0.3).astype(np.float64)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    st = R.OnlineState(cfg)
    st.update(batch, x, z)
    Z = explicit_code_matrix(z, K, s, H, W)
    np.testing.assert_allclose(st.C, Z.T @ Z, atol=1e-12)
    np.testing.assert_allclose(st.B, Z.T @ x, atol=1e-12)
    np.testing.assert_allclose(st.C @ d - st.B, R.filter_gradient_batch(cfg, batch, x, z, d),
                               atol=1e-11)
    assert np.array_equal(st.C, st.C.T)
    assert np.linalg.eigvalsh(st.C).min() >= -1e-10
    lam = np.linalg.eigvalsh(st.C).max()
    assert 0.95 * lam <= st.lipschitz() / 1.01 <= lam * (1 + 1e-12)
    # t = 2 with a mini-batch of two images: C^2 = C^1/2 + mean(Z_n^T Z_n)/2
    x2 = I.images(5, [H, H], [W, W]).astype(np.float64)
    z2 = I.sparse_codes(6, 2 * H * W, K, density=0.3).astype(np.float64)
    b2 = R.Batch(H=[H, H], W=[W, W], ids=[1, 2])
    C1 = st.C.copy()
    st.update(b2, x2, z2)
    Za = explicit_code_matrix(z2[:H * W * K], K, s, H, W)
    Zb = explicit_code_matrix(z2[H * W * K:], K, s, H, W)
    np.testing.assert_allclose(st.C, 0.5 * C1 + 0.25 * (Za.T @ Za + Zb.T @ Zb), atol=1e-12)
    dn = st.dict_step(d)
    assert np.all(np.linalg.norm(dn.reshape(K, -1), axis=1) <= 1 + 1e-15)
    # Eq. 8's objective does not increase under the projected step
    q = lambda v: 0.5 * v @ st.C @ v - v @ st.B
    assert q(dn) <= q(d) + 1e-12


def test_dense_power_iteration_matches_eigvalsh():
    a = rng(20).normal(size=(30, 30))
    C = a @ a.T
    est = R.lib().orc_power_dense(30, R._p(np.ascontiguousarray(C)), 1, R.TAG_LC, 200)
    assert est == pytest.approx(np.linalg.eigvalsh(C).max(), rel=1e-9)


# ------------------------------------------------------------------ inpainting (observed pixels)

def test_observed_all_ones_equals_the_plain_update_and_objective():
    K, s, H, W = 3, 5, 12, 15
    d = I.filters(4, K, s).astype(np.float64)
    x = I.images(5, [H], [W]).astype(np.float64)
    z0 = I.sparse_codes(6, H * W, K, density=0.2).astype(np.float64)
    cfg = R.Config(K=K, s=s, lam=0.3, p_num=2, p_den=3, seed=8)
    batch = R.Batch(H=[H], W=[W], ids=[2])
    ones = np.ones(H * W, dtype=np.uint8)
    za = R.code_step(cfg, batch, x, d, z0, t=2, n_iters=7, step=0.01)
    zb = R.code_step_observed(cfg, batch, x, d, z0, ones, t=2, n_iters=7, step=0.01)
    assert np.array_equal(za, zb)
    assert R.objective(cfg, batch, x, za, d) == R.objective_observed(cfg, batch, x, za, d, ones)


def test_observed_none_leaves_pure_shrinkage():
    """With no observed pixel the gradient vanishes: each PG step only shrinks
    the sampled codes by alpha * lambda (closed form), and Eq. 4 zeroes the
    rest."""
    K, s, H, W = 2, 3, 9, 7
    d = I.filters(1, K, s).astype(np.float64)
    x = I.images(2, [H], [W]).astype(np.float64)
    z0 = rng(4).normal(size=H * W * K)
    cfg = R.Config(K=K, s=s, lam=0.2, p_num=1, p_den=2, seed=3)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    n, alpha = 5, 0.1
    z = R.code_step_observed(cfg, batch, x, d, z0, np.zeros(H * W, np.uint8), 1, n, step=alpha)
    m = R.mask_image(cfg, 1, 0, H, W).ravel().astype(bool)
    want = np.where(m, np.sign(z0) * np.maximum(np.abs(z0) - n * alpha * cfg.lam, 0.0), 0.0)
    np.testing.assert_allclose(z, want, atol=1e-15)
    assert R.objective_observed(cfg, batch, x, z, d, np.zeros(H * W, np.uint8)) == \
        pytest.approx(cfg.lam * np.abs(z).sum(), rel=1e-15)


def test_observed_pg_step_matches_explicit_matrices_8x8():
    """One step z <- soft(z - alpha A^T O (A z - x), alpha lambda) on the
    sampled set, with the explicit synthesis matrix A and O = diag(obs)."""
    K, s, H, W = 2, 5, 8, 8
    d = I.filters(1, K, s).astype(np.float64)
    x = I.images(2, [H], [W]).astype(np.float64)
    z0 = rng(11).normal(size=H * W * K) * 0.3
    obs = (rng(12).random(H * W) < 0.5).astype(np.uint8)
    cfg = R.Config(K=K, s=s, lam=0.05, p_num=1, p_den=2, seed=21)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    alpha = 0.02
    z1 = R.code_step_observed(cfg, batch, x, d, z0, obs, 1, 1, step=alpha)
    A = explicit_synthesis_matrix(d, H, W)
    m = R.mask_image(cfg, 1, 0, H, W).ravel().astype(bool)
    zm = np.where(m, z0, 0.0)
    v = zm - alpha * (A.T @ (obs * (A @ zm - x)))
    want = np.where(m, np.sign(v) * np.maximum(np.abs(v) - alpha * cfg.lam, 0.0), 0.0)
    np.testing.assert_allclose(z1, want, atol=1e-13)
    f = R.objective_observed(cfg, batch, x, z1, d, obs)
    assert f == pytest.approx(0.5 * np.sum(obs * (x - A @ z1) ** 2) + cfg.lam * np.abs(z1).sum(),
                              rel=1e-13)


# ------------------------------------------------------------------ Gauss-Seidel dictionary pass

def test_gauss_seidel_with_one_filter_is_the_jacobi_step():
    K, s, H, W = 1, 5, 14, 12
    x, d = I.images(3, [H], [W]).astype(np.float64), I.filters(4, K, s).astype(np.float64)
    z = I.sparse_codes(5, H * W, K, density=0.2).astype(np.float64)
    cfg = R.Config(K=K, s=s, seed=2)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    np.testing.assert_allclose(R.dict_step_gauss_seidel(cfg, batch, x, z, d),
                               R.dict_step_batch(cfg, batch, x, z, d), rtol=0, atol=1e-14)


def test_gauss_seidel_equals_jacobi_when_blocks_do_not_interact():
    """Filters whose code maps lie far apart (more than 2(s-1) pixels) have
    Z_j^T Z_k = 0: each block's residual update leaves the next blocks'
    gradients unchanged, so one sequential pass equals the simultaneous step."""
    K, s, H, W = 2, 5, 10, 30
    d = I.filters(6, K, s).astype(np.float64)
    x = I.images(7, [H], [W]).astype(np.float64)
    z = np.zeros((H, W, K))
    z[:, :8, 0] = rng(1).normal(size=(H, 8))
    z[:, 20:, 1] = rng(2).normal(size=(H, 10))
    cfg = R.Config(K=K, s=s, seed=3)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    np.testing.assert_allclose(R.dict_step_gauss_seidel(cfg, batch, x, z.ravel(), d),
                               R.dict_step_batch(cfg, batch, x, z.ravel(), d), atol=1e-13)


def test_gauss_seidel_matches_explicit_matrices_and_descends():
    K, s, H, W = 3, 5, 8, 8
    d = I.filters(8, K, s).astype(np.float64).ravel()
    x = I.images(9, [H], [W]).astype(np.float64)
    z = rng(10).normal(size=H * W * K)
    cfg = R.Config(K=K, s=s, seed=4)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    got = R.dict_step_gauss_seidel(cfg, batch, x, z, d)
    Z = explicit_code_matrix(z, K, s, H, W)
    L = R.lipschitz_filters(cfg, batch, z)
    M = s * s
    want = d.copy()
    f0 = 0.5 * np.sum((Z @ want - x) ** 2)
    for k in range(K):
        g = Z[:, k * M:(k + 1) * M].T @ (Z @ want - x)
        v = want[k * M:(k + 1) * M] - g / L
        want[k * M:(k + 1) * M] = v / max(1.0, np.linalg.norm(v))
        f1 = 0.5 * np.sum((Z @ want - x) ** 2)
        assert f1 <= f0 * (1 + 1e-12)  # a step of 1/L on one block never increases Eq. 5
        f0 = f1
    np.testing.assert_allclose(got, want, atol=1e-12)


# ------------------------------------------------------------------ safe screening (Sec. 5)

def _screen_problem(frac):
    """10 x 10 image, K = 3 filters of 5 x 5, p = 1/2; lambda = frac x lambda_max
    of the sampled set (lambda_max = max_S |a_j . x| from the explicit matrix)."""
    K, s, H, W = 3, 5, 10, 10
    d = I.filters(5, K, s).astype(np.float64)
    x = I.images(6, [H], [W]).astype(np.float64)
    A = explicit_synthesis_matrix(d.reshape(K, s, s), H, W)
    m = R.mask_image(R.Config(K=K, s=s, p_num=1, p_den=2, seed=31), 1, 0, H, W).ravel()
    S = np.flatnonzero(m)
    lam_max = float(np.abs(A[:, S].T @ x).max())
    cfg = R.Config(K=K, s=s, lam=frac * lam_max, p_num=1, p_den=2, seed=31)
    return cfg, d, x, A, m, S, lam_max, H, W


@pytest.mark.parametrize("frac", [0.2, 0.5, 0.8])
def test_screening_never_removes_a_coordinate_of_the_solution(frac):
    """Safety: every coordinate the test removes, at iterates near and far from
    the optimum, is zero in the solution of Eq. 3 on the sampled set (30,000
    PG iterations); close to the optimum it removes almost all zeros."""
    cfg, d, x, A, m, S, _, H, W = _screen_problem(frac)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    z_star = R.code_step(cfg, batch, x, d, np.zeros(m.size), t=1, n_iters=30000)
    zeros = (m == 1) & (z_star == 0)
    for its in [0, 5, 20, 100, 1000]:
        z0 = R.code_step(cfg, batch, x, d, np.zeros(m.size), t=1, n_iters=its)
        z, mm, gap, stat = R.screen_image(cfg, d, x, z0, m, H, W)
        removed = (m == 1) & (mm == 0)
        assert not np.any(removed & ~zeros), (its, np.abs(z_star[removed]).max())
        assert gap >= 0.0 and not np.any(z[removed])
        assert np.isnan(stat[m == 0]).all()
    assert removed.sum() >= 0.9 * zeros.sum()
    assert gap < 1e-4


def test_screening_above_lambda_max_removes_every_coordinate():
    """For lambda > lambda_max the solution is z = 0 and the gap at z = 0 is 0,
    so the test removes the whole sampled set."""
    cfg, d, x, A, m, S, lam_max, H, W = _screen_problem(1.05)
    z, mm, gap, _ = R.screen_image(cfg, d, x, np.zeros(m.size), m, H, W)
    assert gap == pytest.approx(0.0, abs=1e-12)
    assert not mm.any() and not z.any()


@pytest.mark.parametrize("frac", [0.7, 0.9])
def test_screening_at_zero_contains_the_safe_rule(frac):
    """At z = 0 the sphere test removes every coordinate the SAFE rule of
    El Ghaoui et al. removes: |a_j . x| < lambda - ||a_j|| ||x|| (lambda_max -
    lambda) / lambda_max (taken with 1% room for the test's margins)."""
    cfg, d, x, A, m, S, lam_max, H, W = _screen_problem(frac)
    lam = cfg.lam
    corr = A.T @ x
    norms = np.linalg.norm(A, axis=0)
    safe = np.zeros(m.size, bool)
    safe[S] = np.abs(corr[S]) < lam - norms[S] * np.linalg.norm(x) * (lam_max - lam) / lam_max \
        - 0.01 * lam
    assert safe.any()
    _, mm, _, _ = R.screen_image(cfg, d, x, np.zeros(m.size), m, H, W)
    assert not np.any(safe & (mm == 1))


def test_screening_statistic_matches_explicit_matrix():
    """Gap, dual point and the per-coordinate statistic from the explicit
    matrix (columns by scipy convolve2d, column norms from those columns)."""
    cfg, d, x, A, m, S, _, H, W = _screen_problem(0.5)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    z0 = R.code_step(cfg, batch, x, d, np.zeros(m.size), t=1, n_iters=20)
    _, _, gap, stat = R.screen_image(cfg, d, x, z0, m, H, W)
    lam = cfg.lam
    rho = x - A @ z0
    scale = max(lam, float(np.abs(A[:, S].T @ rho).max()))
    theta = rho / scale
    primal = 0.5 * rho @ rho + lam * np.abs(z0).sum()
    dual = 0.5 * x @ x - 0.5 * lam ** 2 * np.sum((theta - x / lam) ** 2)
    assert gap == pytest.approx(primal - dual, rel=1e-10)
    radius = np.sqrt(2 * (primal - dual + 1e-6 * (primal + 0.5 * x @ x))) / lam
    want = np.abs(A[:, S].T @ theta) + radius * np.linalg.norm(A[:, S], axis=0)
    np.testing.assert_allclose(stat[S], want, rtol=1e-10)


def test_screened_code_step_reaches_the_unscreened_optimum():
    """Screening every 50 iterations changes the iterates but not the limit:
    both runs end at the solution of Eq. 3, and the active set keeps its
    support while shrinking."""
    cfg, d, x, A, m, S, _, H, W = _screen_problem(0.4)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    z_plain = R.code_step(cfg, batch, x, d, np.zeros(m.size), t=1, n_iters=4000)
    z_scr, active, gaps = R.code_step_screened(cfg, batch, x, d, np.zeros(m.size), t=1,
                                               n_iters=4000, screen_every=50)
    np.testing.assert_allclose(z_scr, z_plain, atol=1e-9)
    assert np.all(active[z_plain != 0] == 1)
    assert active.sum() < m.sum() and np.all(active <= m)
    assert gaps[0] >= 0.0


@pytest.mark.parametrize("seed", [101, 202, 303, 404])
def test_screening_safety_on_random_small_problems(seed):
    """Safety over random shapes, filters, sampling rates and lambdas: at
    random iterates (including random codes off the optimum), no coordinate
    the test removes is nonzero in the solution (2·10^4 PG iterations)."""
    g = np.random.default_rng(seed)
    K, s = int(g.integers(2, 4)), int(g.choice([3, 5]))
    H, W = int(g.integers(6, 11)), int(g.integers(6, 11))
    d = I.filters(seed, K, s).astype(np.float64)
    x = I.images(seed + 1, [H], [W]).astype(np.float64)
    p_den = int(g.choice([1, 2, 3]))
    base = R.Config(K=K, s=s, lam=1.0, p_num=1, p_den=p_den, seed=seed)
    m = R.mask_image(base, 1, 0, H, W).ravel()
    A = explicit_synthesis_matrix(d.reshape(K, s, s), H, W)
    lam_max = float(np.abs(A[:, m == 1].T @ x).max())
    cfg = R.Config(K=K, s=s, lam=float(g.uniform(0.2, 0.95)) * lam_max, p_num=1, p_den=p_den,
                   seed=seed)
    batch = R.Batch(H=[H], W=[W], ids=[0])
    z_star = R.code_step(cfg, batch, x, d, np.zeros(m.size), t=1, n_iters=20000)
    zeros = (m == 1) & (z_star == 0)
    starts = [R.code_step(cfg, batch, x, d, np.zeros(m.size), t=1, n_iters=int(n))
              for n in g.integers(0, 400, size=3)]
    starts.append(g.normal(scale=0.1, size=m.size) * m)
    for z0 in starts:
        _, mm, gap, _ = R.screen_image(cfg, d, x, z0, m, H, W)
        removed = (m == 1) & (mm == 0)
        assert gap >= 0.0
        assert not np.any(removed & ~zeros)
