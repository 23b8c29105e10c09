"""Seeded synthetic contact scenes.

A scene bundles everything both sides of a parity check consume: the
permuted system matrix A, its supernodal LDL^T factor (the input of
``set_system``), the contact mapping (4 node ids and barycentric weights per
contact, the input of ``set_mapping``), friction coefficients, the obstacle
that turns proximity positions into direction blocks and gaps, and the
solver schedule.  All arrays are in the factor's (nested-dissection) node
order: DOF = 3 * node + axis.

Named workloads:
  beam_c0   tetrahedral beam on a 4x4x20 node grid (long axis along x), 0.01 m,
            40 contacts on its bottom face (z = 0) against a plane, seed 0
  liver_c1  ellipsoid of 0.15 x 0.1 x 0.08 m overall extent (semi-axes 0.075,
            0.05, 0.04) with ~3,000 nodes, its lowest 20 % of nodes held by
            1e4 N/m grounding springs, and 300 contacts against a 0.02 m sphere
            tool pressed 6 mm into its top and sliding at 0.05 m/s, seed 1
  tissue_c3 the same ellipsoid meshed to ~20,000 nodes (~60k DOF) with 1,500
            contacts split between two 0.02 m sphere tools, one pressed into
            its top (+z) and one into its +x end, seed 3
  press_c1  contact-dense scene of the C1 size: a 60 x 10 x 5-node beam
            (9,000 DOF, 0.01 m) held at its top face by 1e4 N/m grounding
            springs and pressed 0.2-0.3 mm into a plane along its bottom face,
            300 contacts with mu uniform in 0.1-0.6, 5 Newton x 50 sweeps, seed 5
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import contacts as ct
from .factor import Factor, multifrontal_ldlt
from .fem import assemble
from .mesh import beam, boundary_faces, ellipsoid
from .ordering import nested_dissection, node_graph, symbolic


@dataclass
class Scene:
    name: str
    X: np.ndarray            # (N, 3) node positions, permuted order
    T: np.ndarray            # (nt, 4) tets over permuted node ids
    A: sp.csr_matrix         # (n, n) SPD system matrix, permuted
    factor: Factor
    nodes: np.ndarray        # (m, 4) int64 permuted node ids
    bary: np.ndarray         # (m, 4) barycentric weights
    mu: np.ndarray           # (m,) friction coefficients
    p0: np.ndarray           # (m, 3) proximity positions after the free motion
    obstacle: object         # PlaneObstacle | SphereObstacle
    n_newton: int
    n_sweeps: int
    h: float

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def m(self) -> int:
        return self.nodes.shape[0]

    def linearize(self, p: np.ndarray, k: int):
        """(C_k (m,3,3), delta_k (3m,)) at proximity positions p (m,3)."""
        return self.obstacle.linearize(np.asarray(p, dtype=np.float64).reshape(-1, 3), k)


def _permute(X, T, leaf_nodes):
    G = node_graph(T, X.shape[0])
    order, blocks = nested_dissection(X, G, leaf_nodes=leaf_nodes)
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    return X[order], inv[T], blocks


def _system(X, T, blocks, **fe):
    A, _, _ = assemble(X, T, **fe)
    sym = symbolic(A, blocks)
    return A, multifrontal_ldlt(A, sym)


def beam_scene(nodes_xyz=(20, 4, 4), spacing=0.01, m=40, seed=0, n_newton=3, n_sweeps=50,
               mu=0.3, leaf_nodes=24, h=0.01, name=None) -> Scene:
    rng = np.random.default_rng(seed)
    X, T = beam(nodes_xyz, spacing)
    X, T, blocks = _permute(X, T, leaf_nodes)
    A, F = _system(X, T, blocks, h=h)
    nodes, bary, p0, obst = ct.plane_contacts(rng, X, T, m, n_newton)
    return Scene(name or f"beam{nodes_xyz}", X, T, A, F, nodes, bary, np.full(m, float(mu)), p0, obst,
                 n_newton, n_sweeps, h)


def press_scene(nodes_xyz=(60, 10, 5), spacing=0.01, m=300, seed=5, n_newton=5, n_sweeps=50,
                mu_range=(0.1, 0.6), gap_range_mm=(-0.3, -0.2), slip_mm=0.05, ground_k=1e4, leaf_nodes=24,
                h=0.01, name=None) -> Scene:
    """A beam held at its top face by grounding springs and pressed into a
    plane along its bottom face: normal gaps all negative, so most contacts
    carry load, with sticking and slipping ones mixed (mu per contact)."""
    rng = np.random.default_rng(seed)
    X, T = beam(nodes_xyz, spacing)
    X, T, blocks = _permute(X, T, leaf_nodes)
    top = np.nonzero(np.isclose(X[:, 2], X[:, 2].max()))[0]
    A, F = _system(X, T, blocks, h=h, anchor_nodes=top, anchor_k=ground_k)
    nodes, bary, p0, obst = ct.plane_contacts(rng, X, T, m, n_newton, slip_mm=slip_mm, gap_range_mm=gap_range_mm)
    mu = rng.uniform(mu_range[0], mu_range[1], size=m)
    return Scene(name or f"press{nodes_xyz}", X, T, A, F, nodes, bary, mu, p0, obst, n_newton, n_sweeps, h)


def ellipsoid_scene(semi=(0.075, 0.05, 0.04), target_nodes=3000, m=300, seed=1, n_newton=5,
                    n_sweeps=50, mu=0.3, leaf_nodes=24, h=0.01, indent=6e-3, anchor_frac=0.2,
                    anchor_k=1e4, tools=((0.0, 0.0, 1.0),), name=None) -> Scene:
    rng = np.random.default_rng(seed)
    X, T, _ = ellipsoid(semi, target_nodes)
    X, T, blocks = _permute(X, T, leaf_nodes)
    z = X[:, 2]
    anchored = np.nonzero(z <= z.min() + anchor_frac * (z.max() - z.min()))[0]
    A, F = _system(X, T, blocks, h=h, anchor_nodes=anchored, anchor_k=anchor_k)
    faces, ftet, _ = boundary_faces(T)
    nodes, bary, p0, obst = ct.sphere_contacts(rng, X, T, faces, ftet, m, indent=indent, h=h, tools=tools)
    return Scene(name or f"ellipsoid{target_nodes}", X, T, A, F, nodes, bary, np.full(m, float(mu)), p0,
                 obst, n_newton, n_sweeps, h)


def _batch_member(args):
    """One scene of the batched workload (kept at module level for process pools)."""
    i, nodes, m, mu_seed = args
    rng = np.random.default_rng(mu_seed)
    if i % 2 == 0:
        sc = ellipsoid_scene(target_nodes=nodes, m=m, seed=1000 + i, name=f"batch{i}_ellipsoid")
    else:
        length = max(4, int(round(nodes / 16)))
        cand = 2 * 3 * (length - 1)   # tets with a face on the bottom (z = 0)
        sc = beam_scene(nodes_xyz=(length, 4, 4), m=min(m, cand), seed=1000 + i, n_newton=5,
                        name=f"batch{i}_beam")
    sc.mu = rng.uniform(0.1, 0.6, size=sc.m)
    return sc


def batch_specs(n_scenes=64, seed=2, min_nodes=500, max_nodes=8000, min_m=20, max_m=600):
    """Sizes of the batched workload: node counts log-uniform in [min_nodes,
    max_nodes], contact counts uniform in [min_m, max_m] (beams are capped at
    their number of bottom tets), scenes alternate ellipsoid and beam."""
    rng = np.random.default_rng(seed)
    nodes = np.exp(rng.uniform(np.log(min_nodes), np.log(max_nodes), size=n_scenes)).round().astype(int)
    ms = rng.integers(min_m, max_m + 1, size=n_scenes)
    return [(i, int(nodes[i]), int(min(ms[i], nodes[i] // 3)), seed * 1000 + i) for i in range(n_scenes)]


def batch_scenes(n_scenes=64, seed=2, processes=None, **kw) -> list[Scene]:
    """The batched workload (64 independent scenes by default), generated in a
    spawn-started process pool."""
    import multiprocessing as mp
    import os
    specs = batch_specs(n_scenes, seed, **kw)
    procs = processes or min(len(specs), os.cpu_count() or 1)
    if procs <= 1:
        return [_batch_member(a) for a in specs]
    # one BLAS thread per worker: the pool already fills the cores
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            return pool.map(_batch_member, specs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def beam_c0() -> Scene:
    return beam_scene(name="beam_c0")


def liver_c1() -> Scene:
    return ellipsoid_scene(name="liver_c1")


def tissue_c3() -> Scene:
    return ellipsoid_scene(target_nodes=20000, m=1500, seed=3, tools=((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)),
                           name="tissue_c3")


def press_c1() -> Scene:
    return press_scene(name="press_c1")


NAMED = {"beam_c0": beam_c0, "liver_c1": liver_c1, "tissue_c3": tissue_c3, "press_c1": press_c1}
