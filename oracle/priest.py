"""Oracle of the projection-guided sampler (Paper III, Algorithm 3) -- TEST
INFRASTRUCTURE ONLY, FP64 numpy.

One outer iteration, in the order of Algorithm 3:
  draw samples from N(mu, Sigma)        (Philox4x32-10 + Box-Muller, or given z)
  project each sample                   (am.solve in projection mode, eq. matrix_vec)
  residuals r, ConstraintEliteSet       (N_proj lowest r)
  c_aug = c_1 + w_r r, EliteSet         (N_elite lowest c_aug among them)
  mean / covariance update              (eqs. update_mean, update_covariance)
Reading: weights c_m = exp(-(c_aug,m - delta) / gamma) (the printed exponent
has the opposite sign, which would favour bad samples); the covariance is taken
about the new mean as printed; ties in the selections go to the lower index.

Parity status: philox pinned by the generator's published known-answer
vectors; box_muller by a Kolmogorov-Smirnov test against scipy's normal CDF;
sample by the empirical covariance; select by Python's sorted() on
(key, index); refit by the uniform-weight special case (elite sample mean and
numpy.cov). step/run compose these with am.solve.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import am

M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11)."""
    c0, c1, c2, c3 = (int(x) & MASK for x in ctr)
    k0, k1 = (int(x) & MASK for x in key)
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
        k0, k1 = (k0 + W0) & MASK, (k1 + W1) & MASK
    return c0, c1, c2, c3


def u01(x):
    return (np.asarray(x, np.float64) + 0.5) * 2.0 ** -32


def box_muller(u1, u2):
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)


def philox_normals(B, D, seed, iteration):
    """Standard normal draws [B, D]: counter (i, iteration, q, 0), one call per 4 dims."""
    key = (seed & MASK, (seed >> 32) & MASK)
    z = np.zeros((B, D))
    for i in range(B):
        for q in range(0, (D + 1) // 2, 2):
            w = philox4x32_10((i, iteration, q, 0), key)
            for h in range(2):
                a, b = box_muller(u01(w[2 * h]), u01(w[2 * h + 1]))
                d0 = 2 * (q + h)
                if d0 < D:
                    z[i, d0] = a
                if d0 + 1 < D:
                    z[i, d0 + 1] = b
    return z


def sample(mu, sigma, z, eps):
    """Draw line of Algorithm 3: xi_i = mu + L z_i with L L^T = Sigma + eps I."""
    S = 0.5 * (sigma + sigma.T) + eps * np.eye(sigma.shape[0])
    L = np.linalg.cholesky(S)
    return mu[None, :] + z @ L.T


def costs(batch, xi_bar, residual, w_r=1.0, p=0):
    """c_1 = sum_t ||p''(t)||^2 on the grid (acceleration cost) and c_aug = c_1 + w_r r."""
    n_p, T = int(batch.n_steps[p]), float(batch.duration[p])
    _, _, Pdd = am.bernstein(n_p, T)
    acc = np.einsum("ti,bdi->btd", Pdd, xi_bar.reshape(xi_bar.shape[0], batch.dim, 11))
    c1 = (acc ** 2).sum(axis=(1, 2))
    r = np.max(residual, axis=1)
    r = np.where(np.isnan(r), np.inf, r)
    return r, c1 + w_r * r


def select(r, caug, n_proj, n_elite):
    """ConstraintEliteSet (n_proj lowest r) then EliteSet (n_elite lowest c_aug
    among them); ascending keys, ties to the lower index."""
    idx = np.arange(len(r))
    proj = np.lexsort((idx, r))[:n_proj]
    elite = proj[np.lexsort((proj, caug[proj]))][:n_elite]
    return proj, elite


def refit(xi_bar, caug, elite, mu, sigma, gamma, sig):
    """Eqs. update_mean and update_covariance over the EliteSet."""
    c = caug[elite]
    w = np.exp(-(c - c.min()) / gamma)
    X = xi_bar[elite]
    mu_new = (1.0 - sig) * mu + sig * (w[:, None] * X).sum(0) / w.sum()
    Dv = X - mu_new[None, :]
    cov = (w[:, None, None] * Dv[:, :, None] * Dv[:, None, :]).sum(0) / w.sum()
    sigma_new = (1.0 - sig) * sigma + sig * cov
    return mu_new, sigma_new, X[0].copy(), float(c.min())


@dataclasses.dataclass
class SamplerConfig:
    n_inner: int = 20
    n_proj: int = 2991
    n_elite: int = 410
    gamma: float = 1.0
    sigma_lr: float = 0.5
    eps: float = 1e-6
    w_res: float = 1.0
    seed: int = 0


def step(batch, cfg: SamplerConfig, iteration, mu, sigma, z=None):
    """One outer iteration of Algorithm 3 on problem 0 of `batch` (projection mode)."""
    B, D = batch.n_traj, batch.dim * 11
    if z is None:
        z = philox_normals(B, D, cfg.seed, iteration)
    xi = sample(mu, sigma, z, cfg.eps)
    proj = am.solve(batch, cfg.n_inner, tol=-1.0, cost_mode=1,
                    xi0=xi.reshape(B, batch.dim, 11))
    xb = proj["xi"].reshape(B, D)
    r, caug = costs(batch, xb, proj["residual"], cfg.w_res)
    pidx, elite = select(r, caug, cfg.n_proj, cfg.n_elite)
    mu2, sigma2, best, best_c = refit(xb, caug, elite, mu, sigma, cfg.gamma, cfg.sigma_lr)
    return dict(samples=xi, projected=xb, residual=r, cost_aug=caug, proj_idx=pidx,
                elite_idx=elite, mu=mu2, sigma=sigma2, best=best, best_cost=best_c)
