"""Parity at full size and on the paths only large or contact-dense scenes take.

  * tissue_c3: the 60k-DOF, 1,500-contact two-tool scene, in FP64 call by
    call, and in FP32 in the configuration the bench times (autotuned
    forward-solve plan, 3xTF32 tensor-core contraction, the captured step
    graph); every entry of W_H, W of Newton iteration 1, lambda~ of every
    Newton iteration, the proximity positions and dq against the FP64 oracle
    (W_H formed by column blocks in parallel processes).  At this size every
    tensor-core unit runs unsplit (one persistent pass per tile).
  * press_wide: 640 contacts of which 20 blocks of 32 carry load in every
    Newton iteration, so the PGS runs full sweeps throughout (more blocks may
    change than it sweeps alone).
  * prox_wide: 4,200 contacts, beyond the shared memory of the one-launch
    proximity update in FP32 and FP64 (the two-launch path).

Tolerances as in test_gpu_parity: FP64 W_H and W 1e-12, lambda~ 1e-9, states
identical; FP32 W_H and W 1e-5, lambda~ 1e-4, dq 1e-4, states identical on
contacts more than 1e-3 from a state boundary.
"""
import numpy as np
import pytest

from oracle import delassus as dl
from oracle import pgs as pg

from gpu_helpers import (classify, make_scene, margin_mask, oracle_fast, oracle_solver, oracle_WH, rel, scene)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_06946_gb300 import build, icr
    build.build()
    return icr.Context(0)


def _eager_step(sc, n_newton):
    """One time step call by call; lambda~ and the PGS statistics of every
    Newton iteration, W of the first."""
    sc.reset_proximity()
    sc.build_WH()
    lams, stats, W1 = [], [], None
    for k in range(n_newton):
        sc.linearize(k)
        sc.update_W()
        if k == 0:
            W1 = sc.get("W")
        stats.append(sc.solve_friction(stats=True))
        lams.append(sc.get("LAMBDA"))
        sc.update_proximity()
    P = sc.get("P")
    dq = sc.correct_motion(want_dq=True, reset=True)
    return {"WH": sc.get("WH"), "W1": W1, "lams": lams, "stats": stats, "P": P, "dq": dq}


def _check_iterates(s, ref, got, prec):
    lam_tol = 1e-9 if prec == 1 else 1e-4
    big = max(np.abs(it["lam"]).max() for it in ref["iters"])
    scale = max(np.linalg.norm(it["lam"]) for it in ref["iters"])
    for k, (it, lam) in enumerate(zip(ref["iters"], got["lams"])):
        assert np.linalg.norm(lam - it["lam"]) <= lam_tol * scale, f"iteration {k}"
        ok = margin_mask(it["lam"], s.mu)
        if prec == 1:
            assert np.array_equal(classify(lam, s.mu), classify(it["lam"], s.mu)), f"iteration {k}"
        else:
            assert np.array_equal(classify(lam, s.mu, 1e-5)[ok], classify(it["lam"], s.mu)[ok]), f"iteration {k}"
        if ok.any():
            assert np.abs(lam - it["lam"]).reshape(-1, 3)[ok].max() <= lam_tol * big, f"iteration {k}"
    disp_ref = ref["p"].reshape(-1) - s.p0.reshape(-1)
    assert rel(got["P"].reshape(-1) - s.p0.reshape(-1), disp_ref) < lam_tol
    assert rel(got["dq"], ref["dq"]) < (1e-9 if prec == 1 else 1e-4)


# ---------------------------------------------------------------- tissue_c3
def test_tissue_c3_fp64_matches_oracle(ctx):
    from paper_2306_06946_gb300 import icr
    s = scene("tissue_c3")
    ref = oracle_fast("tissue_c3")
    sc = make_scene(ctx, "tissue_c3", icr.FP64)
    sc.set_field("MU", s.mu)
    got = _eager_step(sc, s.n_newton)
    assert rel(got["WH"], ref["WH"]) < 1e-12
    assert rel(got["W1"], ref["iters"][0]["W"]) < 1e-12
    _check_iterates(s, ref, got, 1)
    # the FP64 residual check of every solve equals the oracle's on the same
    # iterate (the oracle's W and gaps agree with the device's to ~1e-12, so
    # the residuals agree to ~1e-12 of the gap scale)
    for k, (st, it) in enumerate(zip(got["stats"], ref["iters"])):
        r = pg.residuals(it["W"], it["delta"], got["lams"][k], s.mu)
        gap = np.abs(it["delta"]).max()
        for key in ("normal", "cone", "stick", "slip"):
            assert abs(st["res_" + key] - r[key]) <= 1e-9 * gap, (k, key)
        cls = pg.classify(got["lams"][k], s.mu)
        assert (st["n_separated"], st["n_stick"], st["n_slip"]) == tuple(int((cls == c).sum()) for c in range(3))
    assert got["stats"][0]["n_slip"] + got["stats"][0]["n_stick"] > 0


def test_tissue_c3_fp32_bench_configuration_matches_oracle(ctx):
    torch = pytest.importorskip("torch")
    from paper_2306_06946_gb300 import driver, icr
    s = scene("tissue_c3")
    ref = oracle_fast("tissue_c3")
    stream = torch.cuda.Stream()              # a graph is captured on a stream of its own
    sctx = icr.Context(0, stream.cuda_stream)
    sc = make_scene(sctx, "tissue_c3", icr.FP32)
    sc.set_field("MU", s.mu)
    # the bench's launch configuration: autotuned plan, 3xTF32, captured step graph
    tc_levels = sc.autotune()
    sc.step_capture(s.n_newton)
    for _ in range(2):        # replays read the scene's buffers and repeat exactly
        sc.step_launch()
        sc.sync()
        WH, P, dq, lam = sc.get("WH"), sc.get("P"), sc.get("DQ"), sc.get("LAMBDA")
        assert rel(WH, ref["WH"]) < 1e-5
        assert rel(P.reshape(-1) - s.p0.reshape(-1), ref["p"].reshape(-1) - s.p0.reshape(-1)) < 1e-4
        assert rel(dq, ref["dq"]) < 1e-4
        scale = max(np.linalg.norm(it["lam"]) for it in ref["iters"])
        assert np.linalg.norm(lam - ref["iters"][-1]["lam"]) <= 1e-4 * scale
    info = sc.build_info()
    assert tc_levels >= 1 and info["tc_levels"] == tc_levels
    assert info["gemm_tc_units"] > 0 and info["contract_tc_units"] > 0
    # at this size every tensor-core unit is a whole tile (no K split)
    assert info["gemm_tc_split_max"] == 1 and info["contract_tc_split"] == 1
    # the same kernels call by call: W of iteration 1 and every iteration's lambda~
    got = _eager_step(sc, s.n_newton)
    assert rel(got["W1"], ref["iters"][0]["W"]) < 1e-5
    _check_iterates(s, ref, got, 0)
    dq2, _ = driver.newton_step(make_scene(ctx, "tissue_c3", icr.FP32), s.n_newton, mu=s.mu)
    assert rel(dq2, ref["dq"]) < 1e-4


# ---------------------------------------------------------------- press_wide (PGS: more than 16 blocks change)
@pytest.mark.parametrize("prec", [1, 0])
def test_press_wide_full_sweeps_match_oracle(ctx, prec):
    s = scene("press_wide")
    ref = oracle_fast("press_wide")
    for it in ref["iters"]:
        act = np.nonzero(it["lam"].reshape(-1, 3)[:, 0] > 0)[0]
        assert len(set((act // 32).tolist())) > 16
    sc = make_scene(ctx, "press_wide", prec)
    sc.set_field("MU", s.mu)
    got = _eager_step(sc, s.n_newton)
    assert rel(got["WH"], ref["WH"]) < (1e-12 if prec == 1 else 1e-5)
    assert rel(got["W1"], ref["iters"][0]["W"]) < (1e-12 if prec == 1 else 1e-5)
    _check_iterates(s, ref, got, prec)
    # more blocks may change than the PGS sweeps on their own: full sweeps only
    assert all(st["sweeps_s_only"] == 0 for st in got["stats"])
    if prec == 1:
        # the sweep count is exact unless the oracle's last sweeps change lambda~
        # by rounding only (then where an exact fixed point falls depends on it)
        for k, (st, it) in enumerate(zip(got["stats"], ref["iters"])):
            if it["eps"] > 1e-13:
                assert st["sweeps"] == it["sweeps"], (k, st["sweeps"], it["sweeps"], it["eps"])
            else:
                assert st["sweeps"] <= s.n_sweeps


# ---------------------------------------------------------------- prox_wide (two-launch proximity update)
@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 2e-5)])
def test_prox_wide_two_launch_update_matches_oracle(ctx, prec, tol):
    s = scene("prox_wide")
    sc = make_scene(ctx, "prox_wide", prec)
    sc.build_WH()
    assert sc.build_info()["prox_split"] == 1
    rng = np.random.default_rng(12)
    lam = np.abs(rng.normal(size=3 * s.m))
    C, delta = s.linearize(s.p0, 0)
    sc.update_directions(C, delta, s.mu)
    sc.set_field("LAMBDA", lam)
    dp = sc.update_proximity(want_dp=True)
    uk = np.einsum("aji,aj->ai", C, lam.reshape(-1, 3)).reshape(-1)
    # W_H u = H (A^-1 (H^T u)): the oracle's corrective motion mapped back by H
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    dq_ref = dl.correct_motion(oracle_solver("prox_wide"), H, uk)
    assert rel(dp, H @ dq_ref) < tol
    assert rel(sc.get("U"), uk) < (1e-15 if prec == 1 else 1e-7)
    dq = sc.correct_motion()
    assert rel(dq, dq_ref) < (1e-12 if prec == 1 else 1e-4)
