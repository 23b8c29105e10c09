"""Linear tetrahedral finite elements and the implicit system matrix.

The system matrix follows the backward-Euler linearisation of Sec. 3.1
(Eq. "dynamic equation soft"):  A = M + h B + h^2 K  with Rayleigh damping
B = alpha_M M + alpha_K K and a lumped mass matrix.  At the rest state the
corotational element reduces to the linear one, so K is the linear
constant-strain stiffness.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def lame(E: float, nu: float) -> tuple[float, float]:
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def tet_stiffness(X: np.ndarray, T: np.ndarray, E: float, nu: float):
    """Element stiffness matrices (T, 12, 12) and volumes (T,).

    DOF order inside an element is 3 * local_vertex + axis.
    """
    lam, mu = lame(E, nu)
    Dm = np.stack([X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]], X[T[:, 3]] - X[T[:, 0]]], axis=2)
    vol = np.linalg.det(Dm) / 6.0
    if np.any(vol <= 0):
        raise ValueError("degenerate or inverted tetrahedron")
    Ginv = np.linalg.inv(Dm)                       # rows are grad N_1..N_3
    grads = np.concatenate([-Ginv.sum(axis=1, keepdims=True), Ginv], axis=1)   # (T, 4, 3)
    # K_e[3i+a, 3j+b] = V (lam g_i[a] g_j[b] + mu g_i[b] g_j[a] + mu delta_ab g_i . g_j)
    gg = np.einsum("tia,tjb->tiajb", grads, grads)
    dot = np.einsum("tia,tja->tij", grads, grads)
    Ke = lam * gg + mu * gg.transpose(0, 1, 4, 3, 2) \
        + mu * np.einsum("tij,ab->tiajb", dot, np.eye(3))
    Ke = Ke.reshape(-1, 12, 12) * vol[:, None, None]
    return Ke, vol


def assemble(X, T, E=1e5, nu=0.45, rho=1000.0, h=0.01, alpha_m=0.1, alpha_k=0.1,
             anchor_nodes=None, anchor_k=0.0):
    """Assemble (A, M_diag, K) in CSR form over DOFs 3 * node + axis.

    ``anchor_nodes`` get a grounding spring of stiffness ``anchor_k`` (N/m)
    on each axis, added to K (an attached organ instead of a free body).
    """
    n_nodes = X.shape[0]
    n = 3 * n_nodes
    Ke, vol = tet_stiffness(X, T, E, nu)
    dofs = (3 * T[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
    rows = np.repeat(dofs, 12, axis=1).ravel()
    cols = np.tile(dofs, (1, 12)).ravel()
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    K = 0.5 * (K + K.T)
    if anchor_nodes is not None and len(anchor_nodes) and anchor_k > 0:
        kd = np.zeros(n)
        kd[(3 * np.asarray(anchor_nodes)[:, None] + np.arange(3)).ravel()] = anchor_k
        K = K + sp.diags(kd)
    mnode = np.zeros(n_nodes)
    np.add.at(mnode, T.ravel(), np.repeat(rho * vol / 4.0, 4))
    mdiag = np.repeat(mnode, 3)
    M = sp.diags(mdiag)
    A = ((1.0 + h * alpha_m) * M + (h * alpha_k + h * h) * K).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A, mdiag, K.tocsr()
