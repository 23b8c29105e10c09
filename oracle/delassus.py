"""Constraint matrices in FP64: H, C, J, W = J A^-1 J^T, W_H and C W_H C^T.

Sec. 3.4 (Eq. "schur complement"): the constraint-space operator is
W = J A^-1 J^T; with lambda~ = h^2 lambda the integrated gap reads
delta = delta_free + W lambda~.
Sec. 5 (Eqs. "contact jacobian deconstruction", "jacobian directions",
"isolate directions", "schur complemnt reformulated"): J = C H with C block
diagonal (one 3x3 block of rows n, t1, t2 per contact) and H = dG/dq, so
W = C (H A^-1 H^T) C^T = C W_H C^T.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def mapping_matrix(nodes: np.ndarray, bary: np.ndarray, n: int) -> sp.csr_matrix:
    """H = dG/dq for a barycentric mapping (Eq. "geometrical mapping").

    Row 3*a + d of H holds bary[a, i] at DOF 3*nodes[a, i] + d: the proximity
    point of contact a is sum_i bary[a, i] * q(node i).
    """
    m = nodes.shape[0]
    rows, cols, vals = [], [], []
    for a in range(m):
        for d in range(3):
            for i in range(4):
                rows.append(3 * a + d)
                cols.append(3 * int(nodes[a, i]) + d)
                vals.append(float(bary[a, i]))
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * m, n))


def direction_matrix(C: np.ndarray) -> sp.csr_matrix:
    """Block-diagonal C (Eq. "jacobian directions"), one 3x3 block per contact."""
    return sp.csr_matrix(sp.block_diag([sp.csr_matrix(C[a]) for a in range(C.shape[0])], format="csr"))


def jacobian(C: np.ndarray, H: sp.csr_matrix) -> sp.csr_matrix:
    """J = C H (Eq. "isolate directions")."""
    return (direction_matrix(C) @ H).tocsr()


class SystemSolver:
    """A^-1 applied through a sparse LU factorisation of A (computed once:
    the hypothesis A_k = A_0 of Sec. 5).

    ``ordering`` is SuperLU's column ordering.  "COLAMD" (default) picks a
    fill-reducing order itself; "NATURAL" keeps the order A is given in (no
    pivoting, for an SPD A already in a fill-reducing order such as the
    fixture's nested dissection), which factors the 60k-DOF scenes several
    times faster.  A^-1 B does not depend on the ordering beyond rounding."""

    def __init__(self, A: sp.spmatrix, ordering: str = "COLAMD"):
        self.n = A.shape[0]
        if ordering == "NATURAL":
            self.lu = spla.splu(sp.csc_matrix(A), permc_spec="NATURAL", diag_pivot_thresh=0.0,
                                options=dict(SymmetricMode=True))
        else:
            self.lu = spla.splu(sp.csc_matrix(A), permc_spec=ordering)

    def solve(self, B: np.ndarray) -> np.ndarray:
        B = np.asarray(B, dtype=np.float64)
        return self.lu.solve(B)


def delassus_standard(solver: SystemSolver, J: sp.spmatrix) -> np.ndarray:
    """W = J A^-1 J^T formed directly (Eq. "schur complement"; Alg. 2 step 2)."""
    Z = solver.solve(J.T.toarray())          # n x 3m
    return np.asarray(J @ Z)


def compliance_mapping(solver: SystemSolver, H: sp.spmatrix) -> np.ndarray:
    """W_H = H A^-1 H^T (Eq. "schur complemnt reformulated")."""
    Z = solver.solve(H.T.toarray())
    return np.asarray(H @ Z)


def compliance_columns(A: sp.spmatrix, nodes: np.ndarray, bary: np.ndarray, cols: np.ndarray,
                       ordering: str = "COLAMD") -> np.ndarray:
    """Columns ``cols`` of W_H = H A^-1 H^T: H (A^-1 H^T[:, cols]), the
    definition restricted to some columns (one process's share when W_H is
    formed by column blocks in parallel)."""
    n = A.shape[0]
    H = mapping_matrix(nodes, bary, n)
    Z = SystemSolver(A, ordering).solve(H.T[:, cols].toarray())
    return np.asarray(H @ Z)


def delassus_fast(C: np.ndarray, WH: np.ndarray) -> np.ndarray:
    """W = C W_H C^T (Eq. "schur complemnt reformulated"; Alg. 3 step 2)."""
    Cm = direction_matrix(C)
    return np.asarray((Cm @ (Cm @ WH).T).T)


def correct_motion(solver: SystemSolver, H: sp.spmatrix, u: np.ndarray) -> np.ndarray:
    """dq = A^-1 H^T u with u = sum_k C_k^T lambda~_k
    (Eq. "recursive motion correction 3" with J_k = C_k H)."""
    return solver.solve(H.T @ u)
