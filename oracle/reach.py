"""Which supernodes each contact's columns of H^T reach in the elimination tree.

The nonzero structure of x = L^-1 b is the set of elimination-tree ancestors
of the nonzeros of b (the reach of a sparse right-hand side).  Column
3*a + d of H^T is nonzero on DOFs 3*node + d of the four nodes of contact a,
so, on a supernodal factor whose supernodes hold whole nodes, all three
columns of contact a reach the same supernodes: the ancestors (inclusive) of
the supernodes owning its nodes.  This is the structure of
X = L^-1 H^T that W_H = X^T D^-1 X is built from (Eq. "schur complemnt
reformulated" with A = L D L^T).
"""
from __future__ import annotations

import numpy as np


def supernode_of_dof(super_ptr: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(super_ptr.size - 1), np.diff(super_ptr))


def contact_reach(parent: np.ndarray, super_ptr: np.ndarray, nodes: np.ndarray) -> list[list[int]]:
    """For every supernode s, the ascending list of contacts whose columns reach s."""
    sod = supernode_of_dof(super_ptr)
    ns = parent.size
    reached: list[set] = [set() for _ in range(ns)]
    for a in range(nodes.shape[0]):
        for node in nodes[a]:
            s = int(sod[3 * int(node)])
            while s >= 0:
                reached[s].add(a)
                s = int(parent[s])
    return [sorted(r) for r in reached]
