"""Structured tetrahedral meshes: beams and voxelised ellipsoids.

Every cube of a regular grid is split into five tetrahedra (one central tet
plus four corner tets).  The split alternates with the parity of the cube
index so that the face diagonals of neighbouring cubes coincide and the mesh
is conforming.
"""
from __future__ import annotations

import numpy as np

# Cube corners are numbered c = i + 2 j + 4 k for (i, j, k) in {0, 1}^3.
_EVEN_SPLIT = np.array([[1, 2, 4, 7],   # central tet on the odd-parity corners
                        [0, 1, 2, 4],
                        [3, 1, 2, 7],
                        [5, 1, 4, 7],
                        [6, 2, 4, 7]], dtype=np.int64)
_ODD_SPLIT = np.array([[0, 3, 5, 6],    # central tet on the even-parity corners
                       [1, 0, 3, 5],
                       [2, 0, 3, 6],
                       [4, 0, 5, 6],
                       [7, 3, 5, 6]], dtype=np.int64)


def _orient(X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Swap two vertices of every negatively oriented tet."""
    d = X[T[:, 1:]] - X[T[:, :1]]
    vol6 = np.einsum("ij,ij->i", d[:, 0], np.cross(d[:, 1], d[:, 2]))
    T = T.copy()
    neg = vol6 < 0
    T[neg, 1], T[neg, 2] = T[neg, 2].copy(), T[neg, 1].copy()
    return T


def grid_tets(mask_cubes: np.ndarray, spacing: float, origin) -> tuple[np.ndarray, np.ndarray]:
    """Tet mesh of the cubes flagged in ``mask_cubes`` (shape (nx, ny, nz)).

    Returns node coordinates (N, 3) and tets (T, 4) over the nodes that at
    least one kept cube uses, numbered in lexicographic (i, j, k) order.
    """
    nx, ny, nz = mask_cubes.shape
    ci, cj, ck = np.nonzero(mask_cubes)
    corner = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=np.int64)
    # grid node id of corner c of cube (ci, cj, ck) on an (nx+1, ny+1, nz+1) lattice
    gi = ci[:, None] + corner[None, :, 0]
    gj = cj[:, None] + corner[None, :, 1]
    gk = ck[:, None] + corner[None, :, 2]
    gid = (gk * (ny + 1) + gj) * (nx + 1) + gi            # (ncubes, 8)
    parity = (ci + cj + ck) % 2
    split = np.where(parity[:, None, None] == 0, _EVEN_SPLIT[None], _ODD_SPLIT[None])
    tets_g = np.take_along_axis(gid[:, None, :].repeat(5, axis=1), split, axis=2).reshape(-1, 4)
    used, inv = np.unique(tets_g, return_inverse=True)
    T = inv.reshape(-1, 4).astype(np.int64)
    gk_u = used // ((nx + 1) * (ny + 1))
    rem = used % ((nx + 1) * (ny + 1))
    gj_u = rem // (nx + 1)
    gi_u = rem % (nx + 1)
    X = np.stack([gi_u, gj_u, gk_u], axis=1).astype(np.float64) * spacing + np.asarray(origin, dtype=np.float64)
    return X, _orient(X, T)


def beam(nodes_xyz=(4, 4, 20), spacing=0.01) -> tuple[np.ndarray, np.ndarray]:
    """Box beam with ``nodes_xyz`` nodes per axis, z = 0 at the bottom face."""
    nx, ny, nz = (n - 1 for n in nodes_xyz)
    mask = np.ones((nx, ny, nz), dtype=bool)
    return grid_tets(mask, spacing, (0.0, 0.0, 0.0))


def _ellipsoid_mask(semi, spacing):
    a, b, c = semi
    n = [int(np.ceil(2 * s / spacing)) + 2 for s in semi]
    origin = -0.5 * spacing * np.array(n, dtype=np.float64)
    # cube (i, j, k) is kept when all 8 corners lie inside the ellipsoid
    xs = origin[0] + spacing * np.arange(n[0] + 1)
    ys = origin[1] + spacing * np.arange(n[1] + 1)
    zs = origin[2] + spacing * np.arange(n[2] + 1)
    inside = ((xs[:, None, None] / a) ** 2 + (ys[None, :, None] / b) ** 2
              + (zs[None, None, :] / c) ** 2) <= 1.0
    keep = np.ones(n, dtype=bool)
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                keep &= inside[di:di + n[0], dj:dj + n[1], dk:dk + n[2]]
    return keep, origin


def _largest_component(X, T):
    """Keep the connected component (through shared nodes) with most tets."""
    n = X.shape[0]
    parent = np.arange(n)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for t in T:
        r0 = find(t[0])
        for v in t[1:]:
            r = find(v)
            if r != r0:
                parent[r] = r0
    roots = np.array([find(v) for v in range(n)])
    troot = roots[T[:, 0]]
    vals, counts = np.unique(troot, return_counts=True)
    keep_t = troot == vals[np.argmax(counts)]
    T = T[keep_t]
    used, inv = np.unique(T, return_inverse=True)
    return X[used], inv.reshape(-1, 4)


def ellipsoid(semi=(0.15, 0.1, 0.08), target_nodes=3000) -> tuple[np.ndarray, np.ndarray, float]:
    """Voxelised ellipsoid whose node count is as close as possible to ``target_nodes``.

    The grid spacing is searched on a fine geometric scan followed by
    bisection; cubes are kept when all their corners are inside.
    Returns (X, T, spacing).
    """
    vol = 4.0 / 3.0 * np.pi * semi[0] * semi[1] * semi[2]
    h0 = (vol / target_nodes) ** (1.0 / 3.0)
    best = None
    for h in h0 * np.geomspace(0.75, 1.25, 161):
        keep, _ = _ellipsoid_mask(semi, h)
        # node count of the kept cubes without building the mesh
        nxyz = keep.shape
        used = np.zeros((nxyz[0] + 1, nxyz[1] + 1, nxyz[2] + 1), dtype=bool)
        for di in (0, 1):
            for dj in (0, 1):
                for dk in (0, 1):
                    used[di:di + nxyz[0], dj:dj + nxyz[1], dk:dk + nxyz[2]] |= keep
        cnt = int(used.sum())
        if best is None or abs(cnt - target_nodes) < abs(best[0] - target_nodes):
            best = (cnt, h)
    h = best[1]
    keep, origin = _ellipsoid_mask(semi, h)
    X, T = grid_tets(keep, h, origin)
    X, T = _largest_component(X, T)
    return X, T, h


def boundary_faces(T: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Faces used by exactly one tet.

    Returns (face_nodes (F, 3), tet_index (F,), opposite_local (F,)) where
    ``opposite_local`` is the local index (0..3) of the tet vertex not on
    the face.
    """
    local = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    faces = T[:, local].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    once = cnt[inv.ravel()] == 1
    idx = np.nonzero(once)[0]
    return faces[idx], idx // 4, idx % 4
