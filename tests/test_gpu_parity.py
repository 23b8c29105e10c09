"""GPU path (through the C ABI) against the FP64 oracle.

Tolerances: FP32 path, W_H and W within 1e-5 relative Frobenius error and
lambda~ within 1e-4; FP64 path, W_H within 1e-12, lambda~ within 1e-9 and the
contact classification identical.  Integer work (the etree reach) is bit-exact.
"""
import numpy as np
import pytest

from oracle import delassus as dl
from oracle import pgs as pg

from gpu_helpers import (as_stored, classify, make_scene, margin_mask, oracle_fast, oracle_reach, oracle_WH,
                         per_contact_error, rel, scene)

pytestmark = pytest.mark.gpu

SCENES = ["beam_c0", "beam_mid", "liver_c1", "beam_one"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_06946_gb300 import build, icr
    build.build()
    return icr.Context(0)


# ---------------------------------------------------------------- a1 reach (bit-exact)
@pytest.mark.parametrize("name", SCENES)
def test_reach_is_bitexact(ctx, name):
    from paper_2306_06946_gb300 import icr
    sc = make_scene(ctx, name, icr.FP32)
    sc.build_WH()
    ptr = sc.get("REACH_PTR")
    idx = sc.get("REACH_IDX")
    ref = oracle_reach(name)
    assert ptr.size == len(ref) + 1
    for s, lst in enumerate(ref):
        assert idx[ptr[s]:ptr[s + 1]].tolist() == lst


# ---------------------------------------------------------------- a2-a4 W_H
@pytest.mark.parametrize("name", SCENES)
@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)])
def test_WH_matches_oracle(ctx, name, prec, tol):
    sc = make_scene(ctx, name, prec)
    sc.build_WH()
    WH = sc.get("WH")
    ref = oracle_WH(name)
    assert rel(WH, ref) < tol
    assert np.array_equal(WH, WH.T)


def test_WH_rebuild_is_repeatable(ctx):
    from paper_2306_06946_gb300 import icr
    sc = make_scene(ctx, "beam_mid", icr.FP64)
    sc.build_WH()
    a = sc.get("WH")
    sc.build_WH()
    b = sc.get("WH")
    assert rel(a, b) < 1e-14


# ---------------------------------------------------------------- a5 device linearisation
@pytest.mark.parametrize("name", ["beam_c0", "liver_c1", "tools2"])
def test_device_linearize_matches_scene_rule(ctx, name):
    from paper_2306_06946_gb300 import icr
    s = scene(name)
    sc = make_scene(ctx, name, icr.FP64)
    for k in range(min(2, s.n_newton)):
        sc.linearize(k)
        C, delta = s.linearize(s.p0, k)
        assert np.abs(sc.get("C") - C).max() < 1e-14
        assert np.abs(sc.get("DELTA") - delta).max() < 1e-15


# ---------------------------------------------------------------- a6 W = C W_H C^T
@pytest.mark.parametrize("name", SCENES)
@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)])
def test_W_matches_oracle(ctx, name, prec, tol):
    s = scene(name)
    sc = make_scene(ctx, name, prec)
    sc.build_WH()
    C, delta = s.linearize(s.p0, 0)
    sc.update_directions(C, delta, s.mu)
    sc.update_W()
    W = sc.get("W")
    ref = dl.delassus_fast(C, oracle_WH(name))
    assert rel(W, ref) < tol
    assert np.array_equal(W, W.T)


# ---------------------------------------------------------------- a7 PGS on a given W
@pytest.mark.parametrize("name", ["beam_c0", "beam_mid", "liver_c1", "press_c1"])
def test_pgs_fp64_matches_oracle_exactly_in_classification(ctx, name):
    from paper_2306_06946_gb300 import icr
    s = scene(name)
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_fast(C, oracle_WH(name))
    lam_ref, sweeps, eps_ref = pg.pgs(W, delta, s.mu, sweeps=s.n_sweeps)
    sc = make_scene(ctx, name, icr.FP64)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    st = sc.solve_friction(stats=True)
    lam = sc.get("LAMBDA")
    assert st["sweeps"] == sweeps
    assert rel(lam, lam_ref) < 1e-9
    assert np.array_equal(classify(lam, s.mu), classify(lam_ref, s.mu))
    assert abs(st["eps"] - eps_ref) <= 1e-6 * max(eps_ref, 1e-12) + 1e-12 or (st["eps"] < 1e-15 and eps_ref < 1e-15)
    cls = classify(lam_ref, s.mu)
    assert st["n_separated"] == int((cls == 0).sum())
    assert st["n_stick"] == int((cls == 1).sum())
    assert st["n_slip"] == int((cls == 2).sum())
    assert per_contact_error(lam, lam_ref, s.mu) < 1e-9


@pytest.mark.parametrize("name", ["beam_c0", "beam_mid", "liver_c1", "press_c1"])
def test_pgs_fp32_matches_oracle(ctx, name):
    from paper_2306_06946_gb300 import icr
    s = scene(name)
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_fast(C, oracle_WH(name))
    lam_ref, _, _ = pg.pgs(W, delta, s.mu, sweeps=s.n_sweeps)
    sc = make_scene(ctx, name, icr.FP32)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    sc.solve_friction()
    lam = sc.get("LAMBDA")
    assert rel(lam, lam_ref) < 1e-4
    ok = margin_mask(lam_ref, s.mu)
    assert np.array_equal(classify(lam, s.mu, 1e-5)[ok], classify(lam_ref, s.mu)[ok])
    assert per_contact_error(lam, lam_ref, s.mu) < 1e-4


# ---------------------------------------------------------------- a7 FP64 residual check
@pytest.mark.parametrize("name", ["beam_c0", "beam_mid", "liver_c1", "press_c1"])
@pytest.mark.parametrize("prec", [1, 0])
def test_pgs_residual_stats_match_oracle(ctx, name, prec):
    """The device's FP64 residuals and per-state counts equal the oracle's
    residuals() and classify() evaluated on the same stored W, gaps, mu and
    the solve's lambda~, each one separately."""
    s = scene(name)
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_fast(C, oracle_WH(name))
    sc = make_scene(ctx, name, prec)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    st = sc.solve_friction(stats=True)
    lam = sc.get("LAMBDA")
    rel_ = 1e-9 if prec == 1 else 1e-5
    Ws, ds, mus = as_stored(W, prec), as_stored(delta, prec), as_stored(s.mu, prec)
    ref = pg.residuals(Ws, ds, lam, mus, rel_)
    scale = max(np.abs(ds).max(), 1e-300)
    for key in ("normal", "cone", "stick", "slip"):
        assert abs(st["res_" + key] - ref[key]) <= 1e-9 * max(ref[key], 1e-6 * scale), key
    cls = pg.classify(lam, mus, rel_)
    assert st["n_separated"] == int((cls == pg.SEPARATED).sum())
    assert st["n_stick"] == int((cls == pg.STICK).sum())
    assert st["n_slip"] == int((cls == pg.SLIP).sum())
    if name == "press_c1":     # contact-dense: most contacts carry load, sticking and slipping mixed
        assert st["n_stick"] + st["n_slip"] >= 150 and st["n_stick"] >= 10 and st["n_slip"] >= 10


def test_pgs_tol_stops_at_the_oracle_sweep(ctx):
    from paper_2306_06946_gb300 import icr
    s = scene("beam_c0")
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_fast(C, oracle_WH("beam_c0"))
    lam_ref, sweeps, eps = pg.pgs(W, delta, s.mu, sweeps=2000, tol=1e-8)
    assert sweeps < 2000
    sc = make_scene(ctx, "beam_c0", icr.FP64, n_sweeps=2000, tol=1e-8)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    st = sc.solve_friction(stats=True)
    assert st["converged"] and st["sweeps"] == sweeps
    assert rel(sc.get("LAMBDA"), lam_ref) < 1e-9


def test_pgs_reports_noconv(ctx):
    from paper_2306_06946_gb300 import icr
    s = scene("beam_c0")
    C, delta = s.linearize(s.p0, 0)
    sc = make_scene(ctx, "beam_c0", icr.FP64, n_sweeps=2, tol=1e-14)
    sc.set_field("W", dl.delassus_fast(C, oracle_WH("beam_c0")))
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    st = sc.solve_friction(stats=True)
    assert not st["converged"] and st["sweeps"] == 2


def test_pgs_stops_at_a_fixed_point(ctx):
    # every contact separated: the first sweep changes nothing and ends the solve
    from paper_2306_06946_gb300 import icr
    s = scene("beam_mid")
    C, _ = s.linearize(s.p0, 0)
    W = dl.delassus_fast(C, oracle_WH("beam_mid"))
    delta = np.zeros(3 * s.m)
    delta[0::3] = 1e-3
    lam_ref, sweeps, _ = pg.pgs(W, delta, s.mu, sweeps=50)
    assert sweeps == 1 and not lam_ref.any()
    sc = make_scene(ctx, "beam_mid", icr.FP32)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    st = sc.solve_friction(stats=True)
    assert st["sweeps"] == 1 and not sc.get("LAMBDA").any()


def test_pgs_warm_start_continues(ctx):
    # 20 sweeps, then 30 more warm-started, equal 50 sweeps from zero
    from paper_2306_06946_gb300 import icr
    s = scene("beam_mid")
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_fast(C, oracle_WH("beam_mid"))
    lam_ref, _, _ = pg.pgs(W, delta, s.mu, sweeps=50)
    sc = make_scene(ctx, "beam_mid", icr.FP64, n_sweeps=20)
    sc.set_field("W", W)
    sc.set_field("DELTA", delta)
    sc.set_field("MU", s.mu)
    sc.solve_friction()
    sc.set_params(n_sweeps=30)
    sc.solve_friction(warm_start=True)
    assert rel(sc.get("LAMBDA"), lam_ref) < 1e-10


# ---------------------------------------------------------------- a8 + a9
@pytest.mark.parametrize("name", ["beam_c0", "liver_c1"])
@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 2e-5)])
def test_proximity_and_correction_match_oracle(ctx, name, prec, tol):
    s = scene(name)
    sc = make_scene(ctx, name, prec)
    sc.build_WH()
    rng = np.random.default_rng(5)
    lam = np.abs(rng.normal(size=3 * s.m))
    C, delta = s.linearize(s.p0, 0)
    sc.update_directions(C, delta, s.mu)
    sc.set_field("LAMBDA", lam)
    dp = sc.update_proximity(want_dp=True)
    uk = np.einsum("aji,aj->ai", C, lam.reshape(-1, 3)).reshape(-1)
    WH = oracle_WH(name)
    assert rel(dp, WH @ uk) < tol
    assert rel(sc.get("P").reshape(-1) - s.p0.reshape(-1), WH @ uk) < tol
    assert rel(sc.get("U"), uk) < (1e-15 if prec == 1 else 1e-7)
    dq = sc.correct_motion()
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    ref = dl.correct_motion(dl.SystemSolver(s.A), H, uk)
    assert rel(dq, ref) < (1e-12 if prec == 1 else 1e-4)
    assert np.abs(sc.get("U")).max() == 0.0        # reset


# ---------------------------------------------------------------- full step (Alg. 3)
@pytest.mark.parametrize("name,prec", [("beam_c0", 1), ("beam_c0", 0), ("beam_mid", 0), ("liver_c1", 1),
                                       ("liver_c1", 0), ("tools2", 1), ("tools2", 0), ("press_c1", 1),
                                       ("press_c1", 0)])
def test_newton_step_matches_oracle(ctx, name, prec):
    from paper_2306_06946_gb300 import driver
    s = scene(name)
    ref = oracle_fast(name)
    sc = make_scene(ctx, name, prec)
    sc.build_WH()
    lam_scale = max(np.linalg.norm(it["lam"]) for it in ref["iters"])
    lam_big = max(np.abs(it["lam"]).max() for it in ref["iters"])
    disp_ref = ref["p"].reshape(-1) - s.p0.reshape(-1)
    lam_tol = 1e-9 if prec == 1 else 1e-4
    for k, it in enumerate(ref["iters"]):
        sc.linearize(k)
        if k == 0:
            sc.set_field("MU", s.mu)
        sc.update_W()
        sc.solve_friction()
        lam = sc.get("LAMBDA")
        assert np.linalg.norm(lam - it["lam"]) <= lam_tol * lam_scale, f"iteration {k}"
        # per contact, away from state boundaries, against the step's largest entry
        ok = margin_mask(it["lam"], s.mu)
        if ok.any():
            assert np.abs(lam - it["lam"]).reshape(-1, 3)[ok].max() <= lam_tol * lam_big, f"iteration {k}"
        if prec == 1:
            assert np.array_equal(classify(lam, s.mu), classify(it["lam"], s.mu))
        sc.update_proximity()
    disp = sc.get("P").reshape(-1) - s.p0.reshape(-1)
    assert rel(disp, disp_ref) < lam_tol
    dq = sc.correct_motion()
    assert rel(dq, ref["dq"]) < (1e-9 if prec == 1 else 1e-4)
    # the driver's call sequence gives the same step
    sc2 = make_scene(ctx, name, prec)
    dq2, _ = driver.newton_step(sc2, s.n_newton, mu=s.mu)
    assert rel(dq2, dq) < (1e-12 if prec == 1 else 1e-5)


def test_host_directions_match_device_directions(ctx):
    from paper_2306_06946_gb300 import driver, icr
    s = scene("liver_c1")
    a = make_scene(ctx, "liver_c1", icr.FP64)
    dq_dev, _ = driver.newton_step(a, s.n_newton, mu=s.mu)
    b = make_scene(ctx, "liver_c1", icr.FP64)
    dq_host, _ = driver.newton_step(b, s.n_newton, mu=s.mu, linearize=s.linearize)
    assert rel(dq_host, dq_dev) < 1e-12


# ---------------------------------------------------------------- edge cases and errors
def test_no_contacts(ctx):
    from paper_2306_06946_gb300 import icr
    s = scene("beam_c0")
    sc = icr.Scene(ctx, precision=icr.FP32)
    from paper_2306_06946_gb300 import driver
    driver.load_system(sc, s.factor)
    sc.set_mapping(np.zeros((0, 4), np.int32), np.zeros((0, 4)))
    sc.build_WH()
    sc.update_directions(np.zeros((0, 3, 3)), np.zeros(0))
    sc.update_W()
    st = sc.solve_friction(stats=True)
    assert st["sweeps"] == 0 or st["n_separated"] == 0
    sc.update_proximity()
    assert np.all(sc.correct_motion() == 0)


def test_call_order_and_argument_errors(ctx):
    from paper_2306_06946_gb300 import driver, icr
    s = scene("beam_c0")
    sc = icr.Scene(ctx, precision=icr.FP32)
    with pytest.raises(icr.IcrError) as e:
        sc.build_WH()
    assert e.value.code == icr.ESTATE
    driver.load_system(sc, s.factor)
    bad = s.bary.copy()
    bad[0, 0] += 1e-6
    with pytest.raises(icr.IcrError) as e:
        sc.set_mapping(s.nodes, bad)
    assert e.value.code == icr.EINVAL
    with pytest.raises(icr.IcrError) as e:
        sc.set_mapping(s.nodes + 10 ** 6, s.bary)
    assert e.value.code == icr.EINVAL
    sc.set_mapping(s.nodes, s.bary)
    with pytest.raises(icr.IcrError) as e:
        sc.update_W()
    assert e.value.code == icr.ESTATE
    C, delta = s.linearize(s.p0, 0)
    C2 = C.copy()
    C2[0, 0] *= 1.01
    with pytest.raises(icr.IcrError) as e:
        sc.update_directions(C2, delta)
    assert e.value.code == icr.EINVAL
    D = s.factor.D.copy()
    D[5] = -1.0
    sym = s.factor.sym
    with pytest.raises(icr.IcrError) as e:
        sc.set_system(sym.n, sym.super_ptr, sym.rowpat_ptr, sym.rowpat, s.factor.val_ptr, s.factor.Lpanels, D,
                      sym.parent)
    assert e.value.code == icr.ENOTSPD


def test_hbm_budget_is_enforced():
    from paper_2306_06946_gb300 import driver, icr
    s = scene("liver_c1")
    small = icr.Context(0, hbm_budget=1 << 20)
    sc = icr.Scene(small, precision=icr.FP32)
    with pytest.raises(icr.IcrError) as e:
        driver.load_system(sc, s.factor)
    assert e.value.code == icr.ENOMEM


# ---------------------------------------------------------------- contraction variants
@pytest.mark.parametrize("name", ["beam_mid", "liver_c1"])
@pytest.mark.parametrize("mode,tol", [("simt", 1e-5), ("tf32x3", 1e-5), ("tf32", 2e-3), ("bf16", 2e-2)])
def test_WH_contraction_modes(ctx, name, mode, tol):
    from paper_2306_06946_gb300 import driver, icr
    s = scene(name)
    sc = icr.Scene(ctx, precision=icr.FP32, contraction=mode)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    sc.build_WH()
    WH = sc.get("WH")
    err = rel(WH, oracle_WH(name))
    print(f"{name} {mode}: relative Frobenius error of W_H vs FP64 oracle {err:.3e}")
    assert err < tol
    assert np.array_equal(WH, WH.T)


# ---------------------------------------------------------------- forward-solve engine autotuner
def test_autotune_keeps_parity(ctx):
    from paper_2306_06946_gb300 import icr
    s = scene("liver_c1")
    sc = make_scene(ctx, "liver_c1", icr.FP32)
    n = sc.autotune()
    assert 0 <= n <= s.factor.sym.nsuper
    sc.build_WH()
    assert rel(sc.get("WH"), oracle_WH("liver_c1")) < 1e-5
    sc64 = make_scene(ctx, "liver_c1", icr.FP64)
    assert sc64.autotune() == 0          # FP64: CUDA-core tiles only (64 or 32 rows per level)
    sc64.build_WH()
    assert rel(sc64.get("WH"), oracle_WH("liver_c1")) < 1e-12
    n, ms = sc.autotune(level_times=True)
    assert ms.shape == (sc.forward_levels(), 3) and np.all(ms > 0)
    sc.build_WH()   # the tuning builds ran every shape; build_info reads the last build's work lists
    info = sc.build_info()
    assert info["tc_levels"] == n and 0 <= info["short_tile_levels"] <= sc.forward_levels() - n


# ---------------------------------------------------------------- forward-solve plans
@pytest.mark.parametrize("name", ["beam_mid", "liver_c1"])
@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)])
def test_forward_plans_keep_parity(ctx, name, prec, tol):
    """Every plan of the forward solve (tile shape per level: 64-row or 32-row
    CUDA-core tiles, tensor cores; uniform and mixed) forms the same W_H."""
    from paper_2306_06946_gb300 import icr
    sc = make_scene(ctx, name, prec)
    nlev = sc.forward_levels()
    assert nlev >= 2
    plans = [np.zeros(nlev), np.ones(nlev), np.full(nlev, 2), np.arange(nlev) % 2, 1 - np.arange(nlev) % 2,
             np.arange(nlev) % 3, 2 - np.arange(nlev) % 3]
    for plan in plans:
        sc.set_forward_plan(plan.astype(np.uint8))
        sc.build_WH()
        assert rel(sc.get("WH"), oracle_WH(name)) < tol, plan
        assert sc.build_info()["short_tile_levels"] == int(np.sum(plan == 2))
    for bad in [np.zeros(nlev + 1), np.full(nlev, 3)]:
        with pytest.raises(icr.IcrError) as e:
            sc.set_forward_plan(bad.astype(np.uint8))
        assert e.value.code == icr.EINVAL


# ---------------------------------------------------------------- precision of the W update
@pytest.mark.parametrize("name", ["beam_mid", "liver_c1"])
@pytest.mark.parametrize("mode,tol", [("fp32", 1e-5), ("tf32", 2e-3), ("bf16", 2e-2)])
def test_W_update_modes(ctx, name, mode, tol):
    """W = C W_H C^T with TF32 or BF16 operands and FP32 accumulation against
    the FP64 oracle's W (the error is reported, the bound is loose)."""
    from paper_2306_06946_gb300 import icr
    s = scene(name)
    sc = make_scene(ctx, name, icr.FP32)
    sc.set_params(w_update=mode)
    sc.build_WH()
    C, delta = s.linearize(s.p0, 0)
    sc.update_directions(C, delta, s.mu)
    sc.update_W()
    W = sc.get("W")
    err = rel(W, dl.delassus_fast(C, oracle_WH(name)))
    print(f"{name} W update {mode}: relative Frobenius error of W vs FP64 oracle {err:.3e}")
    assert err < tol
    assert np.array_equal(W, W.T)
    if mode != "fp32":
        assert err > 1e-6            # the operands were rounded
    assert rel(sc.get("WH"), oracle_WH(name)) < 1e-5   # W_H itself stays FP32


# ---------------------------------------------------------------- Newton stop from the FP64 residual check
@pytest.mark.parametrize("name,ntol", [("beam_c0", 1e-8), ("liver_c1", 1e-9), ("press_c1", 1e-5)])
@pytest.mark.parametrize("prec", [1, 0])
def test_newton_tol_ends_the_loop_like_the_oracle(ctx, name, ntol, prec):
    torch = pytest.importorskip("torch")
    from oracle import newton as nw
    from paper_2306_06946_gb300 import icr
    from gpu_helpers import oracle_solver
    s = scene(name)
    ref = nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, s.n_sweeps,
                         solver=oracle_solver(name), WH=oracle_WH(name), newton_tol=ntol)
    assert len(ref["iters"]) < s.n_newton
    sctx = icr.Context(0, torch.cuda.Stream().cuda_stream)
    sc = make_scene(sctx, name, prec)
    sc.set_field("MU", s.mu)
    sc.set_params(newton_tol=ntol)
    tol = 1e-9 if prec == 1 else 1e-4
    sc.step(s.n_newton)                       # eager
    assert sc.newton_iterations() == len(ref["iters"])
    assert rel(sc.get("DQ"), ref["dq"]) < tol
    sc.step_capture(s.n_newton)               # the captured step decides on the device as well
    for _ in range(2):
        sc.step_launch()
        assert sc.newton_iterations() == len(ref["iters"])
        assert rel(sc.get("DQ"), ref["dq"]) < tol
    sc.set_params(newton_tol=0.0)
    sc.step(s.n_newton)
    assert sc.newton_iterations() == s.n_newton
