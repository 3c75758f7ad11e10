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

c_1 may carry the two extra terms of the BARN cost (Section 5): the squared
curvature c_kappa = ((y'' x' - x'' y') / (x'^2 + y'^2)^1.5)^2, read with y' in the
second square of the denominator where the print repeats x', and in 3D as its
spatial counterpart ||p' x p''||^2 / ||p'||^6 (0 where ||p'|| < 1e-3, so that
the rest start, where the speed is zero up to rounding, adds nothing); and the
path term c_p = the distance of p(t) from its orthogonal projection onto the
straight segment from the problem's start to its goal (clamped to the segment).
Both enter with weights w_curv, w_path (the paper's cost has unit weights).

The decentralised form (D-PRIEST, Section 5) refines n_dist distributions in
parallel: the batch splits into n_dist contiguous groups, each drawn from and
refitting its own (mu, Sigma); draws still use the sample's index in the whole
batch, and one projection solve covers all groups.

Parity status: philox pinned by the generator's published known-answer
vectors; box_muller by a Kolmogorov-Smirnov test against scipy's normal CDF;
sample by the empirical covariance; select by Python's sorted() on
(key, index); refit by the uniform-weight special case (elite sample mean and
numpy.cov); the curvature term by the parabola (t, t^2), whose curvature has a
closed form (also in a tilted 3D plane), and by a straight line with varying
speed (zero curvature); the path term by offset and overshooting lines with
known distances. step/step_multi compose
these with am.solve; step_multi with n_dist = 1 is step.
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


def curvature_sq(vel, acc):
    """c_kappa per grid point: ||v x a||^2 / ||v||^6 (planar: the squared signed
    curvature); 0 where the speed is below 1e-3. vel, acc: [..., dim]."""
    v = np.zeros(vel.shape[:-1] + (3,))
    a = np.zeros_like(v)
    v[..., :vel.shape[-1]] = vel
    a[..., :acc.shape[-1]] = acc
    cr = np.cross(v, a)
    v2 = (v ** 2).sum(-1)
    out = np.zeros_like(v2)
    ok = v2 > 1e-6
    out[ok] = (cr[ok] ** 2).sum(-1) / v2[ok] ** 3
    return out


def path_distance(pos, start, goal):
    """c_p per grid point: distance of pos [..., dim] from its projection onto the
    segment start -> goal."""
    start, goal = np.asarray(start, np.float64), np.asarray(goal, np.float64)
    d = goal - start
    L2 = float(d @ d)
    u = np.zeros(pos.shape[:-1]) if L2 == 0.0 else np.clip((pos - start) @ d / L2, 0.0, 1.0)
    return np.linalg.norm(pos - (start + u[..., None] * d), axis=-1)


def costs(batch, xi_bar, residual, w_r=1.0, p=0, w_curv=0.0, w_path=0.0):
    """c_1 = sum_t (||p''||^2 + w_curv c_kappa + w_path c_p) on the grid and
    c_aug = c_1 + w_r r."""
    n_p, T = int(batch.n_steps[p]), float(batch.duration[p])
    P, Pd, Pdd = am.bernstein(n_p, T)
    X = xi_bar.reshape(xi_bar.shape[0], batch.dim, 11)
    acc = np.einsum("ti,bdi->btd", Pdd, X)
    c1 = (acc ** 2).sum(axis=(1, 2))
    if w_curv:
        vel = np.einsum("ti,bdi->btd", Pd, X)
        c1 = c1 + w_curv * curvature_sq(vel, acc).sum(1)
    if w_path:
        pos = np.einsum("ti,bdi->btd", P, X)
        c1 = c1 + w_path * path_distance(pos, batch.start[p], batch.goal[p]).sum(1)
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
    w_curv: float = 0.0
    w_path: float = 0.0


def step(batch, cfg: SamplerConfig, iteration, mu, sigma, z=None):
    """One outer iteration of Algorithm 3 on problem 0 of `batch` (projection mode)."""
    B, D = batch.n_traj, batch.dim * 11
    if z is None:
        z = philox_normals(B, D, cfg.seed, iteration)
    xi = sample(mu, sigma, z, cfg.eps)
    proj = am.solve(batch, cfg.n_inner, tol=-1.0, cost_mode=1,
                    xi0=xi.reshape(B, batch.dim, 11))
    xb = proj["xi"].reshape(B, D)
    r, caug = costs(batch, xb, proj["residual"], cfg.w_res, w_curv=cfg.w_curv,
                    w_path=cfg.w_path)
    pidx, elite = select(r, caug, cfg.n_proj, cfg.n_elite)
    mu2, sigma2, best, best_c = refit(xb, caug, elite, mu, sigma, cfg.gamma, cfg.sigma_lr)
    return dict(samples=xi, projected=xb, residual=r, cost_aug=caug, proj_idx=pidx,
                elite_idx=elite, mu=mu2, sigma=sigma2, best=best, best_cost=best_c)


def step_multi(batch, cfg: SamplerConfig, iteration, mus, sigmas, z=None):
    """One outer iteration of D-PRIEST: len(mus) distributions over contiguous
    groups of the batch's samples (mus [n_dist, D], sigmas [n_dist, D, D])."""
    n_dist = len(mus)
    B, D = batch.n_traj, batch.dim * 11
    assert B % n_dist == 0
    Bg = B // n_dist
    if z is None:
        z = philox_normals(B, D, cfg.seed, iteration)
    xi = np.concatenate([sample(mus[g], sigmas[g], z[g * Bg:(g + 1) * Bg], cfg.eps)
                         for g in range(n_dist)])
    proj = am.solve(batch, cfg.n_inner, tol=-1.0, cost_mode=1,
                    xi0=xi.reshape(B, batch.dim, 11))
    xb = proj["xi"].reshape(B, D)
    r, caug = costs(batch, xb, proj["residual"], cfg.w_res, w_curv=cfg.w_curv,
                    w_path=cfg.w_path)
    out = dict(samples=xi, projected=xb, residual=r, cost_aug=caug, proj_idx=[], elite_idx=[],
               mu=[], sigma=[], best=[], best_cost=[])
    for g in range(n_dist):
        sl = slice(g * Bg, (g + 1) * Bg)
        pidx, elite = select(r[sl], caug[sl], cfg.n_proj, cfg.n_elite)
        m2, s2, best, bc = refit(xb[sl], caug[sl], elite, mus[g], sigmas[g], cfg.gamma,
                                 cfg.sigma_lr)
        for k, v in (("proj_idx", pidx), ("elite_idx", elite), ("mu", m2), ("sigma", s2),
                     ("best", best), ("best_cost", bc)):
            out[k].append(v)
    for k in ("proj_idx", "elite_idx", "mu", "sigma", "best", "best_cost"):
        out[k] = np.array(out[k])
    return out
