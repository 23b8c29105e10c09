"""Contact points, obstacles and the per-Newton-iteration constraint linearisation.

This is the collision-detection / linearisation layer that sits above the
constraint solver (Sec. 3.2, Alg. 3 step 1): given the current proximity
positions p it produces the direction blocks C_k (one 3x3 block per contact
with rows n, t1, t2, Eq. "jacobian directions") and the gaps delta_k that the
solver starts from.

Readings used here (the paper leaves them open):
  * tangent frame: e_a is the coordinate axis with the smallest |n_a| (lowest
    index on ties), t1 = normalize(n x e_a), t2 = n x t1;
  * gaps: the normal gap is the signed distance to the obstacle, the two
    tangential gaps are the displacement of p from the contact's anchor on the
    obstacle projected on t1 and t2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def tangent_frame(n: np.ndarray) -> np.ndarray:
    """Direction blocks (m, 3, 3) with rows n, t1, t2 for unit normals n (m, 3)."""
    n = np.asarray(n, dtype=np.float64)
    a = np.argmin(np.abs(n), axis=1)
    e = np.zeros_like(n)
    e[np.arange(n.shape[0]), a] = 1.0
    t1 = np.cross(n, e)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(n, t1)
    return np.stack([n, t1, t2], axis=1)


def dirichlet(rng: np.random.Generator, m: int, k: int) -> np.ndarray:
    """m points uniform on the (k-1)-simplex: normalised -log(u)."""
    e = -np.log(rng.random((m, k)))
    return e / e.sum(axis=1, keepdims=True)


@dataclass
class PlaneObstacle:
    """Plane contacts whose normals are redrawn for every Newton iteration.

    normals[k] (m, 3) is the normal used at iteration k; anchors (m, 3) are
    the obstacle points the gaps are measured from.
    """
    normals: np.ndarray
    anchors: np.ndarray
    kind: str = field(default="plane", init=False)

    def linearize(self, p: np.ndarray, k: int):
        C = tangent_frame(self.normals[k])
        delta = np.einsum("mij,mj->mi", C, p - self.anchors).reshape(-1)
        return C, delta


@dataclass
class SphereObstacle:
    """Rigid sphere tools (centres at the end of the step, radii), each
    translating with its own velocity; ``tool`` names the tool each contact
    touches and the anchors are the tool-surface points each contact started
    from, already moved with its tool to the end of the step."""
    centers: np.ndarray      # (tools, 3)
    radii: np.ndarray        # (tools,)
    tool: np.ndarray         # (m,) int
    anchors: np.ndarray      # (m, 3)
    kind: str = field(default="sphere", init=False)

    def linearize(self, p: np.ndarray, k: int):
        c = self.centers[self.tool]
        d = p - c
        dist = np.linalg.norm(d, axis=1)
        n = d / dist[:, None]
        C = tangent_frame(n)
        rel = p - self.anchors
        delta = np.stack([dist - self.radii[self.tool],
                          np.einsum("mj,mj->m", C[:, 1], rel),
                          np.einsum("mj,mj->m", C[:, 2], rel)], axis=1).reshape(-1)
        return C, delta


def plane_contacts(rng, X, T, m, n_newton, tilt_sigma=0.05, gap_mm=0.5, slip_mm=0.05, gap_range_mm=None):
    """Contacts inside tets that have a face on z = min z (the beam's bottom).

    Normal gaps are uniform in (-gap_mm, gap_mm) mm, or in gap_range_mm =
    (lo, hi) mm when given; tangential free slips uniform in (-slip_mm,
    slip_mm) mm per axis."""
    zmin = X[:, 2].min()
    on = np.isclose(X[T, 2], zmin)
    cand = np.nonzero(on.sum(axis=1) >= 3)[0]
    tets = rng.choice(cand, size=m, replace=cand.size < m)
    nodes = T[tets].astype(np.int64)
    bary = dirichlet(rng, m, 4)
    p0 = np.einsum("mi,mij->mj", bary, X[nodes])
    theta = rng.normal(0.0, tilt_sigma, size=(n_newton, m))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(n_newton, m))
    normals = np.stack([np.sin(theta) * np.sin(phi), -np.sin(theta) * np.cos(phi), np.cos(theta)], axis=2)
    lo, hi = (-gap_mm, gap_mm) if gap_range_mm is None else gap_range_mm
    g = rng.uniform(lo, hi, size=m) * 1e-3
    s = rng.uniform(-slip_mm, slip_mm, size=(m, 2)) * 1e-3
    anchors = p0 - np.stack([s[:, 0], s[:, 1], g], axis=1)
    return nodes, bary, p0, PlaneObstacle(normals=normals, anchors=anchors)


def sphere_contacts(rng, X, T, faces, face_tet, m, radius=0.02, indent=3e-3,
                    velocity=(0.05, 0.0, 0.0), h=0.01, tools=((0.0, 0.0, 1.0),)):
    """Contacts inside the boundary tets nearest sphere tools pressed
    ``indent`` into the body.

    Tool i presses along -tools[i] at the extreme point of the body in the
    direction tools[i] (the first tool on the top, +z); the m contacts are split
    evenly between the tools (the first tools take the remainder).  Tool i moves
    with ``velocity`` turned from +z onto tools[i] (the same vector for the
    +z tool).  The proximity point of each contact is uniform in its tet
    (barycentric weights on all four nodes); tets are taken nearest first and
    each must bring a node that no earlier contact uses, so H has full row rank.
    """
    nt = len(tools)
    dirs = [np.asarray(t, dtype=np.float64) / np.linalg.norm(t) for t in tools]
    v0 = np.asarray(velocity, dtype=np.float64)
    centers, vels = [], []
    for d in dirs:
        centers.append(d * (float((X @ d).max()) + radius - indent))
        vels.append(_turn_z_onto(d) @ v0)
    cen = X[faces].mean(axis=1)
    used = np.zeros(X.shape[0], dtype=bool)
    seen = set()
    tets, tool = [], []
    counts = [m // nt + (1 if i < m % nt else 0) for i in range(nt)]
    for i in range(nt):
        dist = np.linalg.norm(cen - centers[i][None, :], axis=1)
        order = np.argsort(dist, kind="stable")
        got = 0
        # nearest first; a tet is kept only if it brings a node no kept tet
        # uses, which makes the barycentric rows (and H) full row rank
        for f in order:
            if got == counts[i]:
                break
            t = int(face_tet[f])
            if t in seen:
                continue
            seen.add(t)
            if not used[T[t]].all():
                used[T[t]] = True
                tets.append(t)
                tool.append(i)
                got += 1
        if got < counts[i]:
            raise ValueError("not enough boundary tets for the requested contact count")
    nodes = T[np.asarray(tets, dtype=np.int64)].astype(np.int64)
    tool = np.asarray(tool, dtype=np.int64)
    bary = dirichlet(rng, m, 4)
    p0 = np.einsum("mi,mij->mj", bary, X[nodes])
    C = np.asarray(centers)
    V = np.asarray(vels)
    c_start = C[tool] - V[tool] * h
    d0 = p0 - c_start
    anchors = c_start + radius * d0 / np.linalg.norm(d0, axis=1, keepdims=True) + V[tool] * h
    return nodes, bary, p0, SphereObstacle(centers=C, radii=np.full(nt, float(radius)), tool=tool, anchors=anchors)


def _turn_z_onto(d):
    """Rotation taking +z onto the unit vector d (identity for d = +z)."""
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, d)
    c = float(z @ d)
    if np.linalg.norm(v) < 1e-15:
        return np.eye(3) if c > 0 else np.diag([1.0, -1.0, -1.0])
    K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + K + K @ K / (1.0 + c)
