"""Nested-dissection ordering and the supernodal symbolic structure.

The ordering works on the node graph (three DOFs per node stay together) by
recursive coordinate bisection: the node set is cut at the median of its
widest axis, the nodes of the upper half adjacent to the lower half form the
separator, the halves are ordered first and the separator last.  Every leaf
block and every separator becomes one supernode, so supernode boundaries
always fall on node boundaries (multiples of three DOFs).

The symbolic step computes, for every supernode s with DOF columns
[c0, c1), the sorted list R_s of DOF rows below the diagonal block that the
factor L can touch, and the supernodal elimination-tree parent: the supernode
that owns min(R_s).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


def node_graph(T: np.ndarray, n_nodes: int) -> sp.csr_matrix:
    i = np.repeat(T, 4, axis=1).ravel()
    j = np.tile(T, (1, 4)).ravel()
    G = sp.csr_matrix((np.ones_like(i, dtype=np.int8), (i, j)), shape=(n_nodes, n_nodes))
    G.setdiag(0)
    G.eliminate_zeros()
    return G


def nested_dissection(X: np.ndarray, G: sp.csr_matrix, leaf_nodes: int = 24):
    """Return (node_order, blocks) where blocks lists the node counts of the
    supernodes in elimination order."""
    order: list[np.ndarray] = []
    blocks: list[int] = []

    def rec(nodes: np.ndarray):
        if nodes.size <= leaf_nodes:
            if nodes.size:
                order.append(nodes)
                blocks.append(nodes.size)
            return
        P = X[nodes]
        axis = int(np.argmax(P.max(axis=0) - P.min(axis=0)))
        c = P[:, axis]
        cut = np.median(c)
        low = c < cut
        if low.all() or not low.any():
            low = c < np.sort(c)[c.size // 2]
        if low.all() or not low.any():
            order.append(nodes)
            blocks.append(nodes.size)
            return
        in_low = np.zeros(G.shape[0], dtype=bool)
        in_low[nodes[low]] = True
        high = nodes[~low]
        sub = G[high]
        touches = np.asarray(sub.multiply(in_low[None, :]).sum(axis=1)).ravel() > 0
        sep = high[touches]
        rest = high[~touches]
        rec(nodes[low])
        rec(rest)
        if sep.size:
            order.append(sep)
            blocks.append(sep.size)

    rec(np.arange(X.shape[0]))
    return np.concatenate(order), np.asarray(blocks, dtype=np.int64)


@dataclass
class Symbolic:
    n: int                      # DOFs
    super_ptr: np.ndarray       # (nsuper+1,) DOF column ranges
    rowpat_ptr: np.ndarray      # (nsuper+1,) offsets into rowpat
    rowpat: np.ndarray          # below-diagonal DOF rows of every supernode, sorted
    parent: np.ndarray          # (nsuper,) etree parent, -1 at roots

    @property
    def nsuper(self) -> int:
        return self.super_ptr.size - 1

    def width(self, s: int) -> int:
        return int(self.super_ptr[s + 1] - self.super_ptr[s])

    def rows(self, s: int) -> np.ndarray:
        return self.rowpat[self.rowpat_ptr[s]:self.rowpat_ptr[s + 1]]


def symbolic(A_perm: sp.csr_matrix, node_blocks: np.ndarray) -> Symbolic:
    """Supernodal structure of the LDL^T factor of the permuted matrix."""
    n = A_perm.shape[0]
    super_ptr = np.concatenate([[0], np.cumsum(3 * node_blocks)]).astype(np.int64)
    ns = super_ptr.size - 1
    col_super = np.repeat(np.arange(ns), np.diff(super_ptr))
    Acsc = sp.tril(A_perm, format="csc")
    children: list[list[int]] = [[] for _ in range(ns)]
    rows_of: list[np.ndarray] = []
    parent = np.full(ns, -1, dtype=np.int64)
    for s in range(ns):
        c0, c1 = super_ptr[s], super_ptr[s + 1]
        a_rows = Acsc.indices[Acsc.indptr[c0]:Acsc.indptr[c1]]
        parts = [a_rows[a_rows >= c1]]
        for c in children[s]:
            r = rows_of[c]
            parts.append(r[r >= c1])
        R = np.unique(np.concatenate(parts)) if parts else np.zeros(0, dtype=np.int64)
        rows_of.append(R.astype(np.int64))
        if R.size:
            p = int(col_super[R[0]])
            parent[s] = p
            children[p].append(s)
    rowpat_ptr = np.concatenate([[0], np.cumsum([r.size for r in rows_of])]).astype(np.int64)
    rowpat = np.concatenate(rows_of).astype(np.int64) if rows_of else np.zeros(0, np.int64)
    return Symbolic(n=n, super_ptr=super_ptr, rowpat_ptr=rowpat_ptr, rowpat=rowpat, parent=parent)
