"""Batched time steps (icr_batch): one captured graph whose every kernel launch
covers many scenes of uneven DOF and contact counts.

Each scene of a batch runs Alg. 3 exactly as its own step would, so its
results must equal its alone run (same kernels, same arguments; FP32 sums
with atomics may round in another order) and the FP64 oracle, and the batch
must make far fewer launches than the scenes' steps one by one."""
import numpy as np
import pytest

from oracle import newton as nw

from gpu_helpers import rel, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    return pytest.importorskip("torch")


@pytest.fixture(scope="module")
def members():
    """16 scenes of the batched workload's distribution (ellipsoids and beams,
    log-uniform node counts, uniform contact counts), plus the liver-size scene
    whose wide fronts take the tensor-core forward solve."""
    import scenegen
    return scenegen.batch_scenes(16, seed=7, min_nodes=300, max_nodes=2500, min_m=20, max_m=300) + [scene("liver_c1")]


@pytest.fixture(scope="module")
def oracle_refs(members):
    return [nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, s.n_sweeps) for s in members]


def _load(icr, driver, ctx, s, precision):
    sc = icr.Scene(ctx, precision=precision, n_sweeps=s.n_sweeps)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    driver.load_obstacle(sc, s.obstacle)
    sc.set_field("MU", s.mu)
    return sc


def _results(sc):
    return sc.get("DQ"), sc.get("LAMBDA"), sc.get("P")


# dq and p against the alone run to 1e-5 (FP32) / 1e-12 (FP64); lambda~ of the
# last Newton iteration (an increment, relatively sensitive to the rounding
# order of the atomic sums in W_H) to the stated lambda tolerance
@pytest.mark.parametrize("prec,groups,tol_alone,tol_lam,tol_oracle",
                         [(0, 1, 1e-5, 1e-4, 1e-4), (0, 3, 1e-5, 1e-4, 1e-4), (1, 1, 1e-12, 1e-9, 1e-9)])
def test_batch_equals_alone_and_oracle(members, oracle_refs, torch_mod, prec, groups, tol_alone, tol_lam,
                                       tol_oracle):
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    n_newton = members[0].n_newton
    assert all(s.n_newton == n_newton for s in members)
    stream = torch_mod.cuda.Stream()
    ctx = icr.Context(0, stream.cuda_stream)
    scenes = [_load(icr, driver, ctx, s, prec) for s in members]
    alone = []
    for sc in scenes:   # each scene's own device-resident step, one after another, on the plan the batch keeps
        sc.autotune()
        sc.step(n_newton)
        sc.sync()
        alone.append(_results(sc))
    b = icr.Batch(scenes, n_newton, groups)   # creation runs one batched step
    for _ in range(2):                # and every launch one more: each from p_0, the same result
        for sc in scenes:             # a launch that did not run would leave these
            sc.set_field("LAMBDA", np.zeros(3 * sc.m))
            sc.set_field("P", np.zeros(3 * sc.m))
        b.launch()
        stream.synchronize()
        for i, (sc, s) in enumerate(zip(scenes, members)):
            dq, lam, p = _results(sc)
            assert rel(dq, alone[i][0]) < tol_alone, (i, s.n, s.m)
            assert rel(lam, alone[i][1]) < tol_lam, (i, s.n, s.m)
            assert rel(p, alone[i][2]) < tol_alone, (i, s.n, s.m)
            ref = oracle_refs[i]
            assert rel(dq, ref["dq"]) < tol_oracle, (i, s.n, s.m)
            assert rel(lam, ref["iters"][-1]["lam"]) < tol_oracle, (i, s.n, s.m)
    prof = b.profile()                # one more step, eager, with events around each merged launch
    assert len(prof) == b.info()["launches_per_step"]
    assert all(p["ms"] >= 0 and 0 <= p["group"] < groups and p["slots"] >= 1 for p in prof)
    assert sum(1 for p in prof if p["name"] != "copies/fills") == b.info()["kernel_launches_per_step"]
    stream.synchronize()
    for i, sc in enumerate(scenes):
        assert rel(sc.get("DQ"), alone[i][0]) < tol_alone
    info = b.info()
    assert info["n_scenes"] == len(members) and info["steps"] == 3 and info["n_groups"] == groups
    # the scenes' launches share kernels: far fewer launches than one by one
    assert info["kernel_launches_per_step"] * (4 if groups == 1 else 2) < info["scene_launches_per_step"]
    b.close()
    for sc in scenes:
        sc.close()
    ctx.close()


def test_batch_with_tensor_core_levels_runs_them(members, torch_mod):
    """The liver-size member puts its wide fronts on tcgen05 when stepped alone;
    in the batch the same plan runs (its build info matches its alone run)."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    stream = torch_mod.cuda.Stream()
    ctx = icr.Context(0, stream.cuda_stream)
    s = members[-1]
    sc = _load(icr, driver, ctx, s, icr.FP32)
    sc.autotune()
    sc.set_forward_plan([1] * sc.forward_levels())   # every qualifying level on the tensor cores
    sc.step(s.n_newton)
    sc.sync()
    info_alone = sc.build_info()
    dq_alone = sc.get("DQ")
    others = [_load(icr, driver, ctx, x, icr.FP32) for x in members[:4]]
    b = icr.Batch([sc] + others, s.n_newton)
    stream.synchronize()
    info = sc.build_info()
    assert info_alone["tc_levels"] > 0 and info["gemm_tc_units"] == info_alone["gemm_tc_units"]
    assert info["contract_tc_units"] == info_alone["contract_tc_units"] > 0
    assert rel(sc.get("DQ"), dq_alone) < 1e-5
    b.close()
    for x in [sc] + others:
        x.close()
    ctx.close()


def test_batch_argument_and_state_errors(members, torch_mod):
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    stream = torch_mod.cuda.Stream()
    ctx = icr.Context(0, stream.cuda_stream)
    ctx2 = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    a = _load(icr, driver, ctx, members[0], icr.FP32)
    c = _load(icr, driver, ctx, members[1], icr.FP32)
    other = _load(icr, driver, ctx2, members[2], icr.FP32)
    with pytest.raises(icr.IcrError) as e:
        icr.Batch([a, other], members[0].n_newton)   # two contexts
    assert e.value.code == icr.EINVAL
    with pytest.raises(icr.IcrError) as e:
        icr.Batch([a, a], members[0].n_newton)       # a scene twice
    assert e.value.code == icr.EINVAL
    bare = icr.Scene(ctx)
    with pytest.raises(icr.IcrError) as e:
        icr.Batch([a, bare], members[0].n_newton)    # no system, mapping or obstacle
    assert e.value.code == icr.ESTATE
    b = icr.Batch([a, c], members[0].n_newton)
    with pytest.raises(icr.IcrError) as e:
        a.close()                                    # held by the batch
    assert e.value.code == icr.ESTATE
    # another contact count reallocates the scene's buffers: the batch is stale
    s = members[0]
    keep = s.m - 3
    a.set_mapping(s.nodes[:keep], s.bary[:keep])
    with pytest.raises(icr.IcrError) as e:
        b.launch()
    assert e.value.code == icr.ESTATE
    with pytest.raises(icr.IcrError) as e:
        b.profile()                                  # the eager path refuses a stale batch too
    assert e.value.code == icr.ESTATE
    b.close()
    for x in (a, c, other, bare):
        x.close()
    ctx.close()
    ctx2.close()
