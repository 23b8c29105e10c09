"""One time step of the fast recursive scheme (Alg. 3) through libicr.

Helpers that hand a factor, a contact mapping and an obstacle to a
``icr.Scene`` and run the calls of one step in the order the C ABI expects:
set_mapping -> build_WH -> n_newton x (directions -> update_W ->
solve_friction -> update_proximity) -> correct_motion.  Inputs are plain
arrays or objects exposing them by attribute; nothing here computes any part
of the path.
"""
from __future__ import annotations

import numpy as np

from . import icr


def load_system(sc: icr.Scene, factor) -> None:
    """``factor`` exposes sym.{n, super_ptr, rowpat_ptr, rowpat, parent},
    val_ptr, Lpanels and D (the panel layout of icr_set_system)."""
    sym = factor.sym
    sc.set_system(sym.n, sym.super_ptr, sym.rowpat_ptr, sym.rowpat, factor.val_ptr, factor.Lpanels, factor.D,
                  sym.parent)


def load_contacts(sc: icr.Scene, nodes, bary, p0) -> None:
    sc.set_mapping(nodes, bary)
    sc.set_proximity(np.asarray(p0, dtype=np.float64).reshape(-1))


def load_obstacle(sc: icr.Scene, obstacle) -> None:
    """Plane obstacles expose ``normals`` (iters x m x 3) and ``anchors``;
    sphere obstacles ``centers`` (tools x 3), ``radii`` (tools), ``tool``
    (each contact's tool) and ``anchors``."""
    if obstacle.kind == "plane":
        sc.set_obstacle_plane(obstacle.normals, obstacle.anchors)
    elif obstacle.kind == "sphere":
        spheres = np.concatenate([np.asarray(obstacle.centers, dtype=np.float64).reshape(-1, 3),
                                  np.asarray(obstacle.radii, dtype=np.float64).reshape(-1, 1)], axis=1)
        sc.set_obstacle_spheres(spheres, obstacle.tool, obstacle.anchors)
    else:
        raise ValueError(f"unknown obstacle kind {obstacle.kind!r}")


def newton_step(sc: icr.Scene, n_newton: int, mu=None, linearize=None, warm_start: bool = False,
                want_dq: bool = True, stats: bool = False):
    """Run build_WH, the Newton iterations and the corrective motion.

    With ``linearize`` = None the directions come from the scene's obstacle on
    the device (icr_linearize); otherwise ``linearize(p, k) -> (C, delta)`` is
    called on the host with the proximity positions read back each iteration.
    Returns (dq or None, list of per-iteration stats or None).
    """
    sc.build_WH()
    hist = []
    for k in range(n_newton):
        if linearize is None:
            sc.linearize(k)
            if mu is not None and k == 0:
                sc.set_field("MU", mu)
        else:
            C, delta = linearize(sc.get("P"), k)
            sc.update_directions(C, delta, mu)
        sc.update_W()
        hist.append(sc.solve_friction(warm_start=warm_start and k == 0, stats=stats))
        sc.update_proximity()
    dq = sc.correct_motion(want_dq=want_dq, reset=True)
    return dq, (hist if stats else None)
