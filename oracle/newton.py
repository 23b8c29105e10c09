"""The recursive corrective-motion loop, standard (Alg. 2) and fast (Alg. 3).

Both loops take the same inputs: the system matrix A, the barycentric
mapping (nodes, bary), friction coefficients, the proximity positions p_0
after the free motion and a ``linearize(p, k) -> (C_k, delta_k)`` callback
(Alg. 2/3 step 1, collision linearisation supplied by the scene).

Newton reading (incremental, as Alg. 2/3 are written): iteration k solves a
fresh PGS for the increment lambda~_k on the gaps delta_k measured at
p_(k-1); only iteration 1 may be warm-started (from the previous time step).

Standard scheme (Alg. 2), with A_k = A_0 (Sec. 5):
    J_k = C_k H,  W_k = J_k A^-1 J_k^T,  lambda~_k = PGS(W_k, delta_k),
    dq_k = A^-1 J_k^T lambda~_k,  q_k = q_(k-1) + dq_k,  p_k = p_0 + H q_k.
Fast scheme (Alg. 3; Eqs. "schur complemnt reformulated",
"recursive motion correction 7" and "recursive motion correction 3"):
    W_H = H A^-1 H^T once,  W_k = C_k W_H C_k^T,  lambda~_k = PGS(W_k, delta_k),
    p_k = p_(k-1) + W_H C_k^T lambda~_k,  u = sum_k C_k^T lambda~_k,
    dq = A^-1 H^T u  (one solve per time step).
"""
from __future__ import annotations

import numpy as np

from . import delassus as dl
from .pgs import pgs


def standard_scheme(A, nodes, bary, mu, p0, linearize, n_newton, sweeps, tol=0.0, lam0=None, solver=None):
    n = A.shape[0]
    solver = solver or dl.SystemSolver(A)
    H = dl.mapping_matrix(nodes, bary, n)
    p = np.array(p0, dtype=np.float64).reshape(-1)
    q = np.zeros(n)
    hist = []
    for k in range(n_newton):
        C, delta = linearize(p.reshape(-1, 3), k)
        J = dl.jacobian(C, H)
        Z = solver.solve(J.T.toarray())
        W = np.asarray(J @ Z)
        lam, done, eps = pgs(W, delta, mu, lam0 if k == 0 else None, sweeps, tol)
        q = q + Z @ lam
        p = np.asarray(p0, dtype=np.float64).reshape(-1) + H @ q
        hist.append({"C": C, "delta": delta, "W": W, "lam": lam, "p": p.copy(), "sweeps": done, "eps": eps})
    return {"dq": q, "p": p, "iters": hist}


def zero_increment_residual(delta):
    """Normal complementarity residual of lambda~ = 0 at the gaps delta
    (Eq. "signorini's law"): max over contacts of |min(delta_n, 0)|.  When it
    is zero, lambda~ = 0 solves the next iteration's problem (a zero normal
    force also forces zero friction in the cone of Eq. "coulomb's law")."""
    dn = np.asarray(delta, dtype=np.float64)[0::3]
    return float(np.max(np.maximum(0.0, -dn), initial=0.0))


def fast_scheme(A, nodes, bary, mu, p0, linearize, n_newton, sweeps, tol=0.0, lam0=None, solver=None, WH=None,
                newton_tol=0.0):
    """``WH`` (optional): W_H = H A^-1 H^T already formed by the caller, e.g.
    from column blocks of dl.compliance_mapping solved in parallel (W_H is
    column-separable); formed here otherwise.

    ``newton_tol`` > 0 ends the Newton loop early: before iteration k >= 2 the
    gaps at p_(k-1) are linearised and, when the residual of a zero increment
    there (zero_increment_residual) is at most newton_tol, the loop stops (the
    next solve would have nothing to correct); 0 runs all n_newton iterations."""
    n = A.shape[0]
    solver = solver or dl.SystemSolver(A)
    H = dl.mapping_matrix(nodes, bary, n)
    if WH is None:
        WH = dl.compliance_mapping(solver, H)
    p = np.array(p0, dtype=np.float64).reshape(-1)
    u = np.zeros(H.shape[0])
    hist = []
    for k in range(n_newton):
        C, delta = linearize(p.reshape(-1, 3), k)
        if k >= 1 and newton_tol > 0 and zero_increment_residual(delta) <= newton_tol:
            break
        W = dl.delassus_fast(C, WH)
        lam, done, eps = pgs(W, delta, mu, lam0 if k == 0 else None, sweeps, tol)
        uk = np.einsum("aji,aj->ai", C, lam.reshape(-1, 3)).reshape(-1)     # C_k^T lambda~_k
        p = p + WH @ uk
        u += uk
        hist.append({"C": C, "delta": delta, "W": W, "lam": lam, "p": p.copy(), "sweeps": done, "eps": eps})
    dq = dl.correct_motion(solver, H, u)
    return {"dq": dq, "p": p, "WH": WH, "u": u, "iters": hist}
