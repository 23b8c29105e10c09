"""Projected Gauss-Seidel for the frictional contact problem (FP64).

Eq. "constraint system" with lambda~ = h^2 lambda:
    delta = delta_free + W lambda~,
    0 <= delta_n  _|_  lambda~_n >= 0                       (Eq. "signorini's law")
    Coulomb friction in the isotropic disc ||lambda~_t|| <= mu lambda~_n
                                                             (Eq. "coulomb's law",
                                                              3-D reading)
Eq. "PGS" / Alg. 1: contacts are visited in ascending index; contact a sees
the residual r_a = delta_free_a + sum_b W_ab lambda~_b with the newest values
of every lambda~_b, then solves its local problem.

Local rule (the paper only names the two laws):
  1. normal:  lambda_n <- max(0, lambda_n - r_n / W_nn)
  2. update the tangential residual with the change of lambda_n
  3. tangent: lambda_t <- lambda_t - r_t / w_t,  w_t = (W_t1t1 + W_t2t2) / 2
  4. project lambda_t onto the disc of radius mu * lambda_n.
Stopping (Alg. 1): eps = ||lambda^i - lambda^(i-1)|| / ||lambda^i|| (0 when
lambda^i = 0); stop when eps <= tol for a positive tol.  A sweep that changes
no lambda~ at all is a fixed point of the iteration (every later sweep repeats
it exactly), so the solve also stops there: this is Alg. 1's test with
PGS_error = 0.
"""
from __future__ import annotations

import numpy as np


def local_solve(lam: np.ndarray, r: np.ndarray, Wblk: np.ndarray, mu: float) -> np.ndarray:
    """One contact's Signorini-Coulomb update from the current residual r (3,),
    its 3x3 diagonal block Wblk and the current lambda~ (3,)."""
    ln_old = lam[0]
    ln = max(0.0, ln_old - r[0] / Wblk[0, 0])
    dn = ln - ln_old
    rt = r[1:] + Wblk[1:, 0] * dn
    wt = 0.5 * (Wblk[1, 1] + Wblk[2, 2])
    lt = lam[1:] - rt / wt
    lim = mu * ln
    nt = float(np.hypot(lt[0], lt[1]))
    if ln <= 0.0:
        lt = np.zeros(2)
    elif nt > lim:
        lt = lt * (lim / nt)
    return np.array([ln, lt[0], lt[1]])


def pgs(W: np.ndarray, delta: np.ndarray, mu: np.ndarray, lam0=None, sweeps: int = 50, tol: float = 0.0):
    """Returns (lambda~ (3m,), sweeps_done, eps_last)."""
    m = mu.size
    lam = np.zeros(3 * m) if lam0 is None else np.array(lam0, dtype=np.float64)
    eps = 0.0
    done = 0
    for _ in range(sweeps):
        prev = lam.copy()
        for a in range(m):
            sl = slice(3 * a, 3 * a + 3)
            r = delta[sl] + W[sl, :] @ lam
            lam[sl] = local_solve(lam[sl], r, W[sl, sl], float(mu[a]))
        done += 1
        nrm = float(np.linalg.norm(lam))
        eps = float(np.linalg.norm(lam - prev)) / nrm if nrm > 0 else 0.0
        if np.array_equal(lam, prev) or (tol > 0 and eps <= tol):
            break
    return lam, done, eps


def residuals(W: np.ndarray, delta: np.ndarray, lam: np.ndarray, mu: np.ndarray, rel: float = 1e-9) -> dict:
    """Complementarity and friction residuals of a solution (max over contacts).

    With d = delta + W lambda~ (the gaps the solution leaves):
    normal: |min(d_n, lambda_n)| (Eq. "signorini's law"); cone:
    max(0, ||lambda_t|| - mu lambda_n) (Eq. "coulomb's law", disc reading);
    stick (lambda_n > 0 inside the cone): ||d_t||, the sliding a sticking
    contact must not have; slip (on the cone within ``rel``, as ``classify``
    decides): the part of d_t not anti-parallel to lambda_t plus any component
    along it (maximal dissipation: a slipping contact slides against its
    friction force).
    """
    d = (delta + W @ lam).reshape(-1, 3)
    L = lam.reshape(-1, 3)
    normal = np.abs(np.minimum(d[:, 0], L[:, 0]))
    nt = np.linalg.norm(L[:, 1:], axis=1)
    lim = mu * L[:, 0]
    cone = np.maximum(0.0, nt - lim)
    # the same states as classify(): on the cone (slip) when ||lambda_t|| >=
    # mu lambda_n (1 - rel), which includes a frictionless contact (mu = 0)
    on_cone = (L[:, 0] > 0) & (nt >= lim * (1 - rel))
    stick = (L[:, 0] > 0) & ~on_cone
    res_stick = np.where(stick, np.linalg.norm(d[:, 1:], axis=1), 0.0)
    that = np.where(nt[:, None] > 0, L[:, 1:] / np.where(nt > 0, nt, 1.0)[:, None], 0.0)
    along = np.einsum("ij,ij->i", d[:, 1:], that)
    perp = np.linalg.norm(d[:, 1:] - along[:, None] * that, axis=1)
    # with a zero friction force (mu lambda_n = 0) Coulomb's law leaves the
    # sliding d_t free: no slip residual
    res_slip = np.where(on_cone & (nt > 0), perp + np.maximum(0.0, along), 0.0)
    return {"normal": float(normal.max(initial=0.0)), "cone": float(cone.max(initial=0.0)),
            "stick": float(res_stick.max(initial=0.0)), "slip": float(res_slip.max(initial=0.0))}


SEPARATED, STICK, SLIP = 0, 1, 2


def classify(lam: np.ndarray, mu: np.ndarray, rel: float = 1e-9) -> np.ndarray:
    """Per-contact state: 0 separated (lambda_n = 0), 1 stick (strictly inside
    the cone), 2 slip (on the cone within ``rel``)."""
    L = lam.reshape(-1, 3)
    nt = np.linalg.norm(L[:, 1:], axis=1)
    lim = mu * L[:, 0]
    out = np.full(L.shape[0], STICK, dtype=np.int64)
    out[nt >= lim * (1.0 - rel)] = SLIP
    out[L[:, 0] <= 0] = SEPARATED
    return out
