"""Supernodal multifrontal LDL^T factorisation of an SPD matrix (FP64).

Produces the factor in the panel layout a caller hands to the constraint
library: for every supernode s of width w and below-row count r, a
column-major (w + r) x w panel whose first w rows hold the unit lower
triangular diagonal block (ones on the diagonal, zeros above it) and whose
last r rows hold L[R_s, cols(s)].  D holds the pivots.

Each supernode assembles its frontal matrix from the entries of A and the
update matrices of its children, factors the leading w x w block with a
dense Cholesky and passes its Schur complement to its parent.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .ordering import Symbolic


@dataclass
class Factor:
    sym: Symbolic
    val_ptr: np.ndarray     # (nsuper+1,) offsets of each panel in Lpanels
    Lpanels: np.ndarray     # float64, concatenated column-major panels
    D: np.ndarray           # (n,) pivots

    def panel(self, s: int) -> np.ndarray:
        w = self.sym.width(s)
        r = self.sym.rows(s).size
        v = self.Lpanels[self.val_ptr[s]:self.val_ptr[s + 1]]
        return v.reshape(w, w + r).T          # (w + r, w) view, column-major storage

    def to_sparse_L(self) -> sp.csr_matrix:
        """Unit lower triangular L as a sparse matrix (for checks)."""
        sym = self.sym
        ri, ci, vv = [], [], []
        for s in range(sym.nsuper):
            c0, c1 = sym.super_ptr[s], sym.super_ptr[s + 1]
            rows = np.concatenate([np.arange(c0, c1), sym.rows(s)])
            P = self.panel(s)
            rr, cc = np.nonzero(P)
            ri.append(rows[rr])
            ci.append(c0 + cc)
            vv.append(P[rr, cc])
        n = sym.n
        return sp.csr_matrix((np.concatenate(vv), (np.concatenate(ri), np.concatenate(ci))), shape=(n, n))


def multifrontal_ldlt(A_perm: sp.csr_matrix, sym: Symbolic) -> Factor:
    n = sym.n
    ns = sym.nsuper
    Acsc = sp.tril(A_perm, format="csc")
    D = np.zeros(n)
    val_ptr = np.zeros(ns + 1, dtype=np.int64)
    for s in range(ns):
        w = sym.width(s)
        val_ptr[s + 1] = val_ptr[s] + w * (w + sym.rows(s).size)
    Lpanels = np.zeros(int(val_ptr[-1]))
    updates: dict[int, np.ndarray] = {}
    children: list[list[int]] = [[] for _ in range(ns)]
    for s in range(ns):
        if sym.parent[s] >= 0:
            children[sym.parent[s]].append(s)
    pos = np.full(n, -1, dtype=np.int64)
    for s in range(ns):
        c0, c1 = int(sym.super_ptr[s]), int(sym.super_ptr[s + 1])
        w = c1 - c0
        R = sym.rows(s)
        r = R.size
        front_rows = np.concatenate([np.arange(c0, c1), R])
        pos[front_rows] = np.arange(w + r)
        F = np.zeros((w + r, w + r))
        # entries of A in the columns of s (lower triangle, rows >= c0)
        lo, hi = Acsc.indptr[c0], Acsc.indptr[c1]
        rows = Acsc.indices[lo:hi]
        cols = np.repeat(np.arange(c0, c1), np.diff(Acsc.indptr[c0:c1 + 1]))
        vals = Acsc.data[lo:hi]
        pr = pos[rows]
        if np.any(pr < 0):
            raise RuntimeError("symbolic structure misses an entry of A")
        F[pr, cols - c0] += vals
        offdiag = pr >= w
        F[cols[offdiag] - c0, pr[offdiag]] += vals[offdiag]
        F[:w, :w] = np.tril(F[:w, :w]) + np.tril(F[:w, :w], -1).T
        for c in children[s]:
            U = updates.pop(c)
            idx = pos[sym.rows(c)]
            F[np.ix_(idx, idx)] += U
        Rc = np.linalg.cholesky(F[:w, :w])          # F11 = Rc Rc^T, Rc lower
        d = np.diag(Rc) ** 2
        if np.any(~np.isfinite(d)) or np.any(d <= 0):
            raise np.linalg.LinAlgError("matrix is not SPD")
        S21 = sla.solve_triangular(Rc, F[w:, :w].T, lower=True).T if r else np.zeros((0, w))
        sq = np.sqrt(d)
        panel = np.empty((w + r, w))
        panel[:w] = Rc / sq[None, :]
        panel[w:] = S21 / sq[None, :]
        Lpanels[val_ptr[s]:val_ptr[s + 1]] = panel.T.ravel()       # column-major
        D[c0:c1] = d
        if r:
            updates[s] = F[w:, w:] - S21 @ S21.T
        pos[front_rows] = -1
    return Factor(sym=sym, val_ptr=val_ptr, Lpanels=Lpanels, D=D)
