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
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def oracle_solver(name: str):
    return dl.SystemSolver(scene(name).A)


@functools.lru_cache(maxsize=None)
def oracle_WH(name: str):
    s = scene(name)
    return dl.compliance_mapping(oracle_solver(name), dl.mapping_matrix(s.nodes, s.bary, s.n))


@functools.lru_cache(maxsize=None)
def oracle_fast(name: str):
    s = scene(name)
    return nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, s.n_sweeps,
                          solver=oracle_solver(name))


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
