"""Failure handling of the library, made to happen without faulting the GPU.

  * corrupt inputs (NaN / Inf in every host array a set call takes) are
    rejected on the host, and the scene keeps what it had;
  * an injected device-allocation failure part way through loading leaves a
    scene that refuses to run (ICR_ESTATE) instead of running on freed
    buffers, and loads and steps correctly afterwards;
  * a tensor-core pipeline wait that runs out (the context's wait limit set
    to a single non-blocking poll) ends the kernel with ICR_ETIMEOUT on the
    next synchronising call, and the next W_H build matches the oracle.
"""
import numpy as np
import pytest

from gpu_helpers import make_scene, oracle_fast, oracle_WH, rel, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2306_06946_gb300 import build, icr
    build.build()
    return icr.Context(0)


def _raises(code, fn, *args):
    from paper_2306_06946_gb300 import icr
    with pytest.raises(icr.IcrError) as e:
        fn(*args)
    assert e.value.code == code, str(e.value)


def test_non_finite_inputs_are_rejected(ctx):
    from paper_2306_06946_gb300 import driver, icr
    s = scene("beam_c0")
    sc = make_scene(ctx, "beam_c0", icr.FP64)
    sym, F = s.factor.sym, s.factor
    L = F.Lpanels.copy()
    L[len(L) // 2] = np.nan
    _raises(icr.EINVAL, sc.set_system, sym.n, sym.super_ptr, sym.rowpat_ptr, sym.rowpat, F.val_ptr, L, F.D,
            sym.parent)
    D = F.D.copy()
    D[3] = np.inf
    _raises(icr.ENOTSPD, sc.set_system, sym.n, sym.super_ptr, sym.rowpat_ptr, sym.rowpat, F.val_ptr, F.Lpanels, D,
            sym.parent)
    bary = s.bary.copy()
    bary[2, 1] = np.nan
    _raises(icr.EINVAL, sc.set_mapping, s.nodes, bary)
    p = s.p0.reshape(-1).copy()
    p[5] = np.nan
    _raises(icr.EINVAL, sc.set_proximity, p)
    C, delta = s.linearize(s.p0, 0)
    C2 = C.copy()
    C2[1, 2, 0] = np.nan
    _raises(icr.EINVAL, sc.update_directions, C2, delta, s.mu)
    d2 = delta.copy()
    d2[4] = -np.inf
    _raises(icr.EINVAL, sc.update_directions, C, d2, s.mu)
    mu = s.mu.copy()
    mu[0] = np.nan
    _raises(icr.EINVAL, sc.update_directions, C, delta, mu)
    nrm = s.obstacle.normals.copy()
    nrm[0, 3, 1] = np.nan
    _raises(icr.EINVAL, sc.set_obstacle_plane, nrm, s.obstacle.anchors)
    anc = s.obstacle.anchors.copy()
    anc[7, 2] = np.nan
    _raises(icr.EINVAL, sc.set_obstacle_plane, s.obstacle.normals, anc)
    W = np.zeros((3 * s.m, 3 * s.m))
    W[0, 0] = np.inf
    _raises(icr.EINVAL, sc.set_field, "W", W)
    # every rejection happened before anything was replaced: the scene still steps
    dq, _ = driver.newton_step(sc, s.n_newton, mu=s.mu)
    assert rel(dq, oracle_fast("beam_c0")["dq"]) < 1e-9


def test_injected_allocation_failure_leaves_a_usable_scene():
    from paper_2306_06946_gb300 import driver, icr
    s = scene("beam_mid")
    ref = oracle_fast("beam_mid")
    c = icr.Context(0)
    failures = 0
    for after in (0, 3, 11, 26, 40, 55):
        sc = icr.Scene(c, precision=icr.FP32, n_sweeps=s.n_sweeps)
        c.inject_alloc_failure(after)
        stage = "none"
        try:
            driver.load_system(sc, s.factor)
            stage = "system"
            driver.load_contacts(sc, s.nodes, s.bary, s.p0)
            stage = "mapping"
            driver.load_obstacle(sc, s.obstacle)
            stage = "obstacle"
            sc.set_field("MU", s.mu)
        except icr.IcrError as e:
            assert e.code == icr.ENOMEM and "injected" in str(e)
            failures += 1
            # the part that failed is not there: nothing runs on freed buffers
            if stage in ("none", "system"):
                _raises(icr.ESTATE, sc.build_WH)
            _raises(icr.ESTATE, sc.step, s.n_newton)
        c.inject_alloc_failure(-1)
        driver.load_system(sc, s.factor)
        driver.load_contacts(sc, s.nodes, s.bary, s.p0)
        driver.load_obstacle(sc, s.obstacle)
        dq, _ = driver.newton_step(sc, s.n_newton, mu=s.mu)
        assert rel(dq, ref["dq"]) < 1e-4, (after, stage)
        sc.close()
    assert failures >= 4
    assert c.bytes_in_use() == 0
    c.close()


def test_tensor_core_wait_runout_reports_timeout_and_recovers():
    from paper_2306_06946_gb300 import icr
    c = icr.Context(0)
    sc = make_scene(c, "liver_c1", icr.FP32)
    sc.build_WH()
    good = sc.get("WH")
    info = sc.build_info()
    assert info["gemm_tc_units"] > 0 and info["contract_tc_units"] > 0
    c.set_wait_limit(0)             # every pipeline wait: one non-blocking poll
    sc.build_WH()
    _raises(icr.ETIMEOUT, sc.get, "WH")
    c.set_wait_limit(1_000_000_000)
    sc.build_WH()
    again = sc.get("WH")
    assert rel(again, good) < 1e-6
    assert rel(again, oracle_WH("liver_c1")) < 1e-5
    sc.close()
    c.close()
