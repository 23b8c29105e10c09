"""Shared set-up of the GPU parity tests: load scenegen scenes into libicr and
compute the oracle's reference once per scene."""
from __future__ import annotations

import functools

import numpy as np

import scenegen
from oracle import delassus as dl
from oracle import newton as nw
from oracle import pgs as pg
from oracle import reach as rc


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@functools.lru_cache(maxsize=None)
def scene(name: str):
    if name == "beam_c0":
        return scenegen.NAMED["beam_c0"]()
    if name == "liver_c1":
        return scenegen.NAMED["liver_c1"]()
    if name == "beam_mid":      # several tiles, ragged tail: 77 contacts, 2,160 DOF
        return scenegen.beam_scene(nodes_xyz=(24, 6, 5), m=77, seed=7, n_newton=3, n_sweeps=40, name="beam_mid")
    if name == "tools2":        # two sphere tools (top and +x end), 90 contacts on a 900-node ellipsoid
        return scenegen.ellipsoid_scene(target_nodes=900, m=90, seed=11, tools=((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)),
                                        name="tools2")
    if name == "beam_one":      # a single contact
        return scenegen.beam_scene(nodes_xyz=(6, 3, 3), m=1, seed=2, n_newton=2, n_sweeps=10, name="beam_one")
    if name in ("press_c1", "tissue_c3"):
        return scenegen.NAMED[name]()
    if name == "press_wide":    # 640 contacts, 20 PGS blocks of 32 carrying load in every Newton iteration
        return scenegen.press_scene(nodes_xyz=(80, 10, 5), m=640, seed=6, name="press_wide")
    if name == "prox_wide":     # 4,200 contacts: C^T lambda~ exceeds the default shared memory in FP32 and FP64
        return scenegen.press_scene(nodes_xyz=(100, 45, 3), m=4200, seed=9, n_newton=1, name="prox_wide")
    raise KeyError(name)


# scenes whose system is factored in its own (nested-dissection) order by the
# oracle's sparse LU, and whose W_H is formed by column blocks in parallel
LARGE = {"tissue_c3", "press_wide", "prox_wide"}


@functools.lru_cache(maxsize=None)
def oracle_solver(name: str):
    return dl.SystemSolver(scene(name).A, "NATURAL" if name in LARGE else "COLAMD")


def _columns_job(args):
    A, nodes, bary, cols = args
    return dl.compliance_columns(A, nodes, bary, cols, "NATURAL")


@functools.lru_cache(maxsize=None)
def oracle_WH(name: str):
    s = scene(name)
    if name not in LARGE:
        return dl.compliance_mapping(oracle_solver(name), dl.mapping_matrix(s.nodes, s.bary, s.n))
    # column blocks of W_H in spawned processes (one BLAS thread each)
    import multiprocessing as mp
    import os
    procs = max(1, min(16, os.cpu_count() or 1))
    chunks = np.array_split(np.arange(3 * s.m), procs)
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            blocks = pool.map(_columns_job, [(s.A, s.nodes, s.bary, c) for c in chunks], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return np.hstack(blocks)


@functools.lru_cache(maxsize=None)
def oracle_fast(name: str):
    s = scene(name)
    return nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, s.n_sweeps,
                          solver=oracle_solver(name), WH=oracle_WH(name))


@functools.lru_cache(maxsize=None)
def oracle_reach(name: str):
    s = scene(name)
    sym = s.factor.sym
    return rc.contact_reach(sym.parent, sym.super_ptr, s.nodes)


def make_scene(ctx, name: str, precision: int, n_sweeps=None, tol=0.0, obstacle=True):
    from paper_2306_06946_gb300 import driver, icr
    s = scene(name)
    sc = icr.Scene(ctx, precision=precision, n_sweeps=s.n_sweeps if n_sweeps is None else n_sweeps, tol=tol)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    if obstacle:
        driver.load_obstacle(sc, s.obstacle)
    return sc


def classify(lam, mu, rel_=1e-9):
    return pg.classify(np.asarray(lam), np.asarray(mu), rel_)


def margin_mask(lam, mu, margin=1e-3):
    """Contacts whose oracle state is more than ``margin`` (relative) away from
    a classification boundary."""
    L = np.asarray(lam).reshape(-1, 3)
    ln = L[:, 0]
    nt = np.linalg.norm(L[:, 1:], axis=1)
    lim = mu * ln
    big = ln.max(initial=0.0)
    sep_ok = (ln == 0) | (ln > margin * big)
    cone_ok = (ln == 0) | (np.abs(nt - lim) > margin * lim) | (nt >= lim * (1 - 1e-9))
    return sep_ok & cone_ok


def per_contact_error(lam, ref, mu, margin=1e-3):
    """Largest change of one contact's lambda~ (max over its three entries)
    among the contacts more than ``margin`` away from a state boundary,
    relative to the largest entry of the reference."""
    L = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    R = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
    ok = margin_mask(ref, mu, margin)
    if not ok.any():
        return 0.0
    return float(np.abs(L - R)[ok].max() / max(np.abs(R).max(), 1e-300))


def as_stored(x, precision):
    """Values as a scene of the given precision stores them (FP32: rounded)."""
    x = np.asarray(x, dtype=np.float64)
    return x if precision == 1 else x.astype(np.float32).astype(np.float64)
