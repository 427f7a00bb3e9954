"""Batch-level FP64 oracle: Algorithm 1 (SBCSC) and Algorithm 2 (SOCSC) steps.

TEST INFRASTRUCTURE ONLY.  Composes the per-image C routines of
``scsc_oracle.c`` over a batch of images.  Every array crossing into C is
converted to contiguous float64 here; inputs may be float32 (the GPU's input
values) and are widened exactly.

Layouts match the library: a batch packs images at ``off[n]`` pixels
(row-major H x W), codes at ``off[n] * K`` ([H][W][K]), filters [K][s][s].

Readings of the paper used here (each also listed in the design notes):
* the code problem (Eq. 3) is solved by proximal gradient with constant step
  1/L_z, L_z = 1.01 x the 50-step power-iteration estimate of
  lambda_max(D D^T) on the batch's largest (H, W) domain;
* the warm start of the sampled codes is the previous codes restricted to the
  sampled set; unsampled codes are zero after the step (Eq. 4);
* the batch dictionary step (Eq. 5) is one Jacobi projected-gradient step
  d_k <- P(d_k - G_k / L_d), L_d from the same power-iteration rule on
  sum_n Z_n^T Z_n;
* the online surrogates (Eq. 7) average Z^T Z and Z^T x over the mini-batch,
  t counts mini-batches from 1, and Eq. 8 takes one projected-gradient step
  with L_C from the power-iteration rule on C^t.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import lib

POWER_ITERS = 50
L_SAFETY = 1.01
TAG_LZ = 0x4C  # start vector tag of the code-step power iteration
TAG_LD = 0x44  # dictionary (batch) power iteration
TAG_LC = 0x43  # online surrogate power iteration


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Batch:
    """Images of possibly different sizes packed back to back."""
    H: np.ndarray
    W: np.ndarray
    ids: np.ndarray  # global image index n used by the subsampling hash
    off: np.ndarray = field(init=False)

    def __post_init__(self):
        self.H = np.asarray(self.H, dtype=np.int32)
        self.W = np.asarray(self.W, dtype=np.int32)
        self.ids = np.asarray(self.ids, dtype=np.int64)
        sizes = self.H.astype(np.int64) * self.W.astype(np.int64)
        self.off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)

    @property
    def n(self) -> int:
        return len(self.H)

    @property
    def total_pixels(self) -> int:
        return int((self.H.astype(np.int64) * self.W).sum())

    def image(self, a: np.ndarray, n: int, per_pixel: int = 1) -> np.ndarray:
        o = int(self.off[n]) * per_pixel
        return a[o:o + int(self.H[n]) * int(self.W[n]) * per_pixel]


@dataclass
class Config:
    K: int
    s: int = 11
    lam: float = 1.0
    p_num: int = 1
    p_den: int = 1
    seed: int = 0


# ---------------------------------------------------------------- primitives

def splitmix64(v: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(v & (2**64 - 1))))


def mask_image(cfg: Config, t: int, n: int, H: int, W: int) -> np.ndarray:
    out = np.empty(H * W * cfg.K, dtype=np.uint8)
    lib().orc_mask_image(cfg.seed, t, n, cfg.K, H, W, cfg.p_num, cfg.p_den, _p(out))
    return out.reshape(H, W, cfg.K)


def mask_batch(cfg: Config, batch: Batch, t: int) -> np.ndarray:
    """Flat [sum_n H_n W_n K] 0/1 mask of outer iteration t."""
    return np.concatenate([mask_image(cfg, t, int(batch.ids[n]), int(batch.H[n]),
                                      int(batch.W[n])).ravel() for n in range(batch.n)])


def synthesis(d, z, K: int, s: int, H: int, W: int) -> np.ndarray:
    d, z = _f64(d), _f64(z)
    out = np.empty(H * W)
    lib().orc_synthesis(K, s, H, W, _p(d), _p(z), _p(out))
    return out


def adjoint(d, r, K: int, s: int, H: int, W: int) -> np.ndarray:
    d, r = _f64(d), _f64(r)
    out = np.empty(H * W * K)
    lib().orc_adjoint(K, s, H, W, _p(d), _p(r), _p(out))
    return out


def adjoint_sampled(d, r, mask, K: int, s: int, H: int, W: int, fill=np.nan) -> np.ndarray:
    """The adjoint at the sampled coordinates; `fill` elsewhere."""
    d, r = _f64(d), _f64(r)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.full(H * W * K, fill)
    lib().orc_adjoint_sampled(K, s, H, W, _p(d), _p(r), _p(m), _p(out))
    return out


def filter_gradient(r, z, K: int, s: int, H: int, W: int) -> np.ndarray:
    r, z = _f64(r), _f64(z)
    out = np.empty(K * s * s)
    lib().orc_filter_gradient(K, s, H, W, _p(r), _p(z), _p(out))
    return out


def soft_threshold(v: float, tau: float) -> float:
    return float(lib().orc_soft_threshold(v, tau))


def project_filters(d, K: int, M: int) -> np.ndarray:
    d = _f64(d).copy()
    lib().orc_project_filters(K, M, _p(d))
    return d


# ---------------------------------------------------------------- batch level

def synthesis_batch(cfg: Config, batch: Batch, z, d) -> np.ndarray:
    z, d = _f64(z), _f64(d)
    return np.concatenate([synthesis(d, batch.image(z, n, cfg.K), cfg.K, cfg.s,
                                     int(batch.H[n]), int(batch.W[n])) for n in range(batch.n)])


def objective(cfg: Config, batch: Batch, x, z, d) -> float:
    """Eq. 1 summed over the images of the batch."""
    x, z, d = _f64(x), _f64(z), _f64(d)
    tot = 0.0
    for n in range(batch.n):
        tot += lib().orc_objective_image(cfg.K, cfg.s, int(batch.H[n]), int(batch.W[n]), _p(d),
                                         _p(np.ascontiguousarray(batch.image(z, n, cfg.K))),
                                         _p(np.ascontiguousarray(batch.image(x, n))), cfg.lam)
    return float(tot)


def lipschitz_codes(cfg: Config, d, H: int, W: int) -> float:
    """L_z = 1.01 * power-iteration estimate of lambda_max(D D^T) on H x W."""
    d = _f64(d)
    lam = lib().orc_power_ddt(cfg.K, cfg.s, H, W, _p(d), cfg.seed, TAG_LZ, POWER_ITERS)
    return L_SAFETY * float(lam)


def lipschitz_filters(cfg: Config, batch: Batch, z) -> float:
    """L_d = 1.01 * power-iteration estimate of lambda_max(sum_n Z_n^T Z_n)."""
    z = _f64(z)
    lam = lib().orc_power_ztz(batch.n, _p(batch.off), _p(batch.H), _p(batch.W), cfg.K, cfg.s,
                              _p(z), cfg.seed, TAG_LD, POWER_ITERS)
    return L_SAFETY * float(lam)


def code_step(cfg: Config, batch: Batch, x, d, z, t: int, n_iters: int,
              step: float | None = None, keep: bool = False) -> np.ndarray:
    """One outer iteration of the code update (Alg. 1 lines 4-7 / Alg. 2
    lines 5-7): draw M^t, solve Eq. 3 by n_iters proximal-gradient steps from
    the warm start, return the Eq. 4 codes.  ``step`` overrides 1/L_z.
    ``keep``: the variant where codes off the sampled set keep their values
    (Sec. 3.1, the rest remain unchanged) instead of Eq. 4's zeros."""
    x, d = _f64(x), _f64(d)
    z = _f64(z).copy()
    if step is None:
        L = lipschitz_codes(cfg, d, int(batch.H.max()), int(batch.W.max()))
        alpha = 1.0 / L if L > 0 else 0.0
    else:
        alpha = float(step)
    for n in range(batch.n):
        H, W = int(batch.H[n]), int(batch.W[n])
        m = mask_image(cfg, t, int(batch.ids[n]), H, W).ravel()
        zi = np.ascontiguousarray(batch.image(z, n, cfg.K))
        xi = np.ascontiguousarray(batch.image(x, n))
        update = lib().orc_code_update_image_keep if keep else lib().orc_code_update_image
        update(cfg.K, cfg.s, H, W, _p(d), _p(xi), _p(zi), _p(m), alpha, cfg.lam, n_iters)
        o = int(batch.off[n]) * cfg.K
        z[o:o + zi.size] = zi
    return z


def objective_observed(cfg: Config, batch: Batch, x, z, d, obs) -> float:
    """Eq. 1 with the data term over observed pixels only (inpainting, Sec.
    4.3); obs: one 0/1 byte per pixel of the batch."""
    x, z, d = _f64(x), _f64(z), _f64(d)
    obs = np.ascontiguousarray(obs, dtype=np.uint8).ravel()
    tot = 0.0
    for n in range(batch.n):
        H, W = int(batch.H[n]), int(batch.W[n])
        tot += lib().orc_objective_image_observed(
            cfg.K, cfg.s, H, W, _p(d), _p(np.ascontiguousarray(batch.image(z, n, cfg.K))),
            _p(np.ascontiguousarray(batch.image(x, n))),
            _p(np.ascontiguousarray(batch.image(obs, n))), cfg.lam)
    return float(tot)


def code_step_observed(cfg: Config, batch: Batch, x, d, z, obs, t: int, n_iters: int,
                       step: float | None = None) -> np.ndarray:
    """code_step with the data term over observed pixels only (inpainting,
    Sec. 4.3).  The step is 1/L_z of the unmasked operator unless given: a
    valid step, since ||O D|| <= ||D|| for the 0/1 diagonal O."""
    x, d = _f64(x), _f64(d)
    z = _f64(z).copy()
    obs = np.ascontiguousarray(obs, dtype=np.uint8).ravel()
    if step is None:
        L = lipschitz_codes(cfg, d, int(batch.H.max()), int(batch.W.max()))
        alpha = 1.0 / L if L > 0 else 0.0
    else:
        alpha = float(step)
    for n in range(batch.n):
        H, W = int(batch.H[n]), int(batch.W[n])
        m = mask_image(cfg, t, int(batch.ids[n]), H, W).ravel()
        zi = np.ascontiguousarray(batch.image(z, n, cfg.K))
        xi = np.ascontiguousarray(batch.image(x, n))
        oi = np.ascontiguousarray(batch.image(obs, n))
        lib().orc_code_update_image_observed(cfg.K, cfg.s, H, W, _p(d), _p(xi), _p(zi), _p(m),
                                             _p(oi), alpha, cfg.lam, n_iters)
        o = int(batch.off[n]) * cfg.K
        z[o:o + zi.size] = zi
    return z


def filter_gradient_batch(cfg: Config, batch: Batch, x, z, d) -> np.ndarray:
    """G = sum_n Z_n^T (D z_n - x_n), the gradient of Eq. 5's objective."""
    x, z, d = _f64(x), _f64(z), _f64(d)
    G = np.zeros(cfg.K * cfg.s * cfg.s)
    for n in range(batch.n):
        H, W = int(batch.H[n]), int(batch.W[n])
        zi = batch.image(z, n, cfg.K)
        r = synthesis(d, zi, cfg.K, cfg.s, H, W) - batch.image(x, n)
        G += filter_gradient(r, zi, cfg.K, cfg.s, H, W)
    return G


def dict_step_batch(cfg: Config, batch: Batch, x, z, d) -> np.ndarray:
    """Eq. 5 by one projected-gradient step on all filters (Alg. 1 line 8)."""
    d = _f64(d).ravel()
    G = filter_gradient_batch(cfg, batch, x, z, d)
    L = lipschitz_filters(cfg, batch, z)
    M = cfg.s * cfg.s
    dn = d - G / L if L > 0 else d.copy()
    return project_filters(dn, cfg.K, M)


def dict_step_gauss_seidel(cfg: Config, batch: Batch, x, z, d) -> np.ndarray:
    """Eq. 5 by one pass of projected block coordinate descent (Sec. 3.2): for
    k = 1..K in order, G_k = sum_n Z_{n,k}^T r_n with the current residuals,
    d_k <- P(d_k - G_k / L_d), then r_n <- r_n + Z_{n,k} (d_k^new - d_k^old).
    L_d is the batch step's power-iteration estimate of lambda_max(sum_n
    Z_n^T Z_n), an upper bound of every block's lambda_max(Z_k^T Z_k)."""
    d = _f64(d).ravel().copy()
    x, z = _f64(x), _f64(z)
    K, s = cfg.K, cfg.s
    M = s * s
    L = lipschitz_filters(cfg, batch, z)
    r = [synthesis(d, batch.image(z, n, K), K, s, int(batch.H[n]), int(batch.W[n]))
         - batch.image(x, n) for n in range(batch.n)]
    for k in range(K):
        G = np.zeros(M)
        for n in range(batch.n):
            H, W = int(batch.H[n]), int(batch.W[n])
            G += filter_gradient(r[n], batch.image(z, n, K), K, s, H, W)[k * M:(k + 1) * M]
        old = d[k * M:(k + 1) * M].copy()
        new = old - G / L if L > 0 else old.copy()
        new = project_filters(new, 1, M)
        delta = np.zeros(K * M)
        delta[k * M:(k + 1) * M] = new - old
        for n in range(batch.n):
            H, W = int(batch.H[n]), int(batch.W[n])
            r[n] = r[n] + synthesis(delta, batch.image(z, n, K), K, s, H, W)
        d[k * M:(k + 1) * M] = new
    return d


class OnlineState:
    """Surrogates C^t, B^t of Eq. 7 (mean over the mini-batch) and Eq. 8."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        KM = cfg.K * cfg.s * cfg.s
        self.C = np.zeros((KM, KM))
        self.B = np.zeros(KM)
        self.t = 0

    def update(self, batch: Batch, x, z) -> None:
        """C^t = (t-1)/t C^{t-1} + (1/t) mean_n Z_n^T Z_n; B^t likewise."""
        self.t += 1
        t = self.t
        x, z = _f64(x), _f64(z)
        self.C *= (t - 1) / t
        self.B *= (t - 1) / t
        scale = 1.0 / (t * batch.n)
        for n in range(batch.n):
            H, W = int(batch.H[n]), int(batch.W[n])
            zi = np.ascontiguousarray(batch.image(z, n, self.cfg.K))
            xi = np.ascontiguousarray(batch.image(x, n))
            lib().orc_surrogate_accumulate(self.cfg.K, self.cfg.s, H, W, _p(zi), _p(xi), scale,
                                           _p(self.C), _p(self.B))

    def lipschitz(self) -> float:
        n = self.C.shape[0]
        lam = lib().orc_power_dense(n, _p(self.C), self.cfg.seed, TAG_LC, POWER_ITERS)
        return L_SAFETY * float(lam)

    def dict_step(self, d) -> np.ndarray:
        """One projected-gradient step on Eq. 8 from the warm start d^{t-1}."""
        d = _f64(d).ravel()
        L = self.lipschitz()
        grad = self.C @ d - self.B
        dn = d - grad / L if L > 0 else d.copy()
        return project_filters(dn, self.cfg.K, self.cfg.s * self.cfg.s)


def admm_image(cfg: Config, d, x, z, mask, H: int, W: int, n_iters: int,
               rho: float | None = None, alpha_r: float = 1.8,
               cg_iters: int = 200) -> np.ndarray:
    """ADMM on Eq. 3 for one image (rho = 10 lambda, alpha = 1.8 by default)."""
    d, x = _f64(d), _f64(x)
    z = _f64(z).copy()
    m = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    rho = 10.0 * cfg.lam if rho is None else rho
    lib().orc_admm_image(cfg.K, cfg.s, H, W, _p(d), _p(x), _p(z), _p(m), cfg.lam, rho,
                         alpha_r, n_iters, cg_iters)
    return z


def screen_image(cfg: Config, d, x, z, mask, H: int, W: int):
    """Duality-gap sphere test on Eq. 3 for one image (Sec. 5: safe screening
    of the code LASSO).  Returns (z, mask, gap, stat): the codes and active
    set with the coordinates proven zero removed, the duality gap at the
    input codes, and the per-coordinate statistic (NaN off the input set)."""
    d, x = _f64(d), _f64(x)
    z = _f64(z).copy()
    m = np.ascontiguousarray(mask, dtype=np.uint8).ravel().copy()
    stat = np.empty(H * W * cfg.K)
    gap = ctypes.c_double(0.0)
    lib().orc_screen_image(cfg.K, cfg.s, H, W, _p(d), _p(x), _p(z), _p(m), cfg.lam,
                           ctypes.byref(gap), _p(stat))
    return z, m, float(gap.value), stat


def code_step_screened(cfg: Config, batch: Batch, x, d, z, t: int, n_iters: int,
                       screen_every: int, step: float | None = None):
    """code_step with the screening test run on each image's active set before
    iterations 0, e, 2e, ... (e = screen_every; 0 = never).  Returns (z,
    active mask [sum_n H_n W_n K], per-image gap of the last test)."""
    x, d = _f64(x), _f64(d)
    z = _f64(z).copy()
    if step is None:
        L = lipschitz_codes(cfg, d, int(batch.H.max()), int(batch.W.max()))
        alpha = 1.0 / L if L > 0 else 0.0
    else:
        alpha = float(step)
    masks, gaps = [], []
    for n in range(batch.n):
        H, W = int(batch.H[n]), int(batch.W[n])
        m = np.ascontiguousarray(mask_image(cfg, t, int(batch.ids[n]), H, W).ravel())
        zi = np.ascontiguousarray(batch.image(z, n, cfg.K))
        xi = np.ascontiguousarray(batch.image(x, n))
        gap = ctypes.c_double(0.0)
        lib().orc_code_update_image_screened(cfg.K, cfg.s, H, W, _p(d), _p(xi), _p(zi), _p(m),
                                             alpha, cfg.lam, n_iters, screen_every,
                                             ctypes.byref(gap))
        o = int(batch.off[n]) * cfg.K
        z[o:o + zi.size] = zi
        masks.append(m)
        gaps.append(float(gap.value))
    return z, np.concatenate(masks) if masks else np.zeros(0, np.uint8), np.array(gaps)
