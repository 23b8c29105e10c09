"""PGS sweeps over the contacts that may change (S-only sweeps) against the
FP64 oracle's plain sweeps.

A contact with lambda~ = 0 and a non-negative normal residual keeps
lambda~ = 0 under the local rule (Eq. "PGS"), so the library sweeps only the
blocks that may change while the sum of |changes| since the last complete
residual stays below min r_n / max |W[n, j]| over the other contacts (j over the
columns of S's blocks), and folds those changes into the others' residuals
later, in one pass, or lets the blocks of contacts about to change join S.  The
iterate is that of plain sweeps; these cases drive both the S-only sweeps and
their ends (the bound running out, |S| above the block limit, the last block
in S, an exact fixed point) and compare with the oracle on the same W.

The instances are those of tests/pgs_cases.py.
"""
import numpy as np
import pytest

from oracle import pgs as pg

from gpu_helpers import rel, scene
from pgs_cases import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_06946_gb300 import build, icr
    build.build()
    return icr.Context(0)


def pgs_scene(ctx, prec, m, sweeps):
    """A scene with m contacts (the mapping only sizes the buffers: W, delta
    and mu are set directly)."""
    from paper_2306_06946_gb300 import driver, icr
    s = scene("beam_mid")
    sc = icr.Scene(ctx, precision=prec, n_sweeps=sweeps)
    driver.load_system(sc, s.factor)
    rng = np.random.default_rng(m)
    nodes = rng.integers(0, s.n // 3, size=(m, 4))
    driver.load_contacts(sc, nodes, np.full((m, 4), 0.25), np.zeros((m, 3)))
    return sc


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [1, 0])
def test_s_only_sweeps_match_the_oracle(ctx, name, prec):
    make, expect = CASES[name]
    W, delta, mu = make()
    m = mu.size
    sweeps = 50
    lam_ref, sw_ref, eps_ref = pg.pgs(W, delta, mu, sweeps=sweeps)
    sc = pgs_scene(ctx, prec, m, sweeps)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", mu)
    st = sc.solve_friction(stats=True)
    lam = sc.get("LAMBDA")
    if prec == 1:
        # where the oracle's last sweeps change lambda~ by rounding only (eps
        # near 1e-16 or 0: a fixed point, or a limit cycle of one-ulp changes
        # that runs to the cap), where the iteration stops depends on that
        # rounding; lambda~ itself must agree
        if eps_ref > 1e-13:
            assert st["sweeps"] == sw_ref
        elif sw_ref < sweeps:   # both stop at an exact fixed point, a few sweeps apart
            assert abs(st["sweeps"] - sw_ref) <= 5
        else:                   # the oracle's one-ulp cycle runs to the cap
            assert st["sweeps"] <= sweeps
        assert rel(lam, lam_ref) < 1e-9
    else:
        assert rel(lam, lam_ref) < 1e-4
    if expect == "off":
        assert st["sweeps_s_only"] == 0 and st["deferred_folds"] == 0
    elif expect == "fixed":
        assert sw_ref < sweeps and st["sweeps"] < sweeps
    elif expect == "leave":   # the bound ran out with a 17th block about to change: a fold
        assert st["deferred_folds"] > 0
    else:
        assert st["sweeps_s_only"] > 0
        if expect == "join":   # a contact outside S started to change: its block joined S
            assert st["joins"] > 0
    # a warm start from the result continues from it: same lambda~ again after
    # the sweeps a fixed point or the cap allows
    if prec == 1 and expect == "fixed":
        sc.solve_friction(warm_start=True)
        assert rel(sc.get("LAMBDA"), lam_ref) < 1e-12


@pytest.mark.parametrize("prec", [1, 0])
def test_coupling_bound_of_a_given_W(ctx, prec):
    """W formed on the device (C W_H C^T) and the same W set directly give the
    same coupling bound, hence bit-identical solves; a second solve on the
    same W repeats the first."""
    from gpu_helpers import make_scene
    s = scene("beam_mid")
    sc = make_scene(ctx, "beam_mid", prec)
    sc.build_WH()
    C, delta = s.linearize(s.p0, 0)
    sc.update_directions(C, delta, s.mu)
    sc.update_W()
    st = sc.solve_friction(stats=True)
    a = sc.get("LAMBDA")
    sc.solve_friction()
    assert np.array_equal(sc.get("LAMBDA"), a)
    sc2 = pgs_scene(ctx, prec, s.m, s.n_sweeps)
    sc2.set_field("W", sc.get("W"))
    sc2.set_field("DELTA", sc.get("DELTA"))
    sc2.set_field("MU", s.mu)
    st2 = sc2.solve_friction(stats=True)
    assert np.array_equal(sc2.get("LAMBDA"), a)
    assert (st2["sweeps"], st2["sweeps_s_only"], st2["deferred_folds"], st2["joins"]) == \
        (st["sweeps"], st["sweeps_s_only"], st["deferred_folds"], st["joins"])
