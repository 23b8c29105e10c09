"""Device-resident steps, captured step graphs, batching and the request loop.

A scene's step must give the same result when it runs alone and when it runs
in the mix with other scenes' steps on other streams (batching and serving),
and the device-resident step must match the host-driven call sequence and the
FP64 oracle."""
import numpy as np
import pytest

from oracle import newton as nw

from gpu_helpers import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    return pytest.importorskip("torch")


@pytest.fixture(scope="module")
def batch():
    import scenegen
    return scenegen.batch_scenes(6, seed=5, min_nodes=200, max_nodes=900, min_m=20, max_m=120)


def _load(icr, driver, ctx, s):
    sc = icr.Scene(ctx, precision=icr.FP32, n_sweeps=s.n_sweeps)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    driver.load_obstacle(sc, s.obstacle)
    sc.set_field("MU", s.mu)
    return sc


@pytest.fixture(scope="module")
def loaded(batch, torch_mod):
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    streams = [torch_mod.cuda.Stream() for _ in batch]
    ctxs = [icr.Context(0, st.cuda_stream) for st in streams]
    scenes = [_load(icr, driver, c, s) for c, s in zip(ctxs, batch)]
    alone = []
    for sc, s in zip(scenes, batch):
        sc.step(s.n_newton)
        sc.sync()
        alone.append(sc.get("DQ"))
    return streams, ctxs, scenes, alone


def test_step_matches_host_sequence_and_oracle(batch, loaded):
    from paper_2306_06946_gb300 import driver, icr
    _, ctxs, scenes, alone = loaded
    for i in (0, 1):
        s = batch[i]
        sc2 = _load(icr, driver, ctxs[i], s)
        dq_host, _ = driver.newton_step(sc2, s.n_newton)
        assert rel(alone[i], dq_host) < 1e-5
        ref = nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, s.n_sweeps)
        assert rel(alone[i], ref["dq"]) < 1e-4


def test_batch_in_mix_equals_alone(batch, loaded):
    from paper_2306_06946_gb300 import icr
    _, _, scenes, alone = loaded
    for sc, s in zip(scenes, batch):
        sc.step_capture(s.n_newton)
    n = len(scenes)
    lat, makespan = icr.serve(scenes, np.arange(n), np.zeros(n), n_slots=n)
    assert np.all(lat > 0) and makespan >= lat.max() * 0.999
    for sc, a in zip(scenes, alone):
        assert rel(sc.get("DQ"), a) < 1e-5


def test_serve_poisson_arrivals(batch, loaded):
    from paper_2306_06946_gb300 import icr
    _, _, scenes, alone = loaded
    for sc, s in zip(scenes, batch):
        sc.step_capture(s.n_newton)
    rng = np.random.default_rng(9)
    nreq = 40
    arrivals = np.cumsum(rng.exponential(1.0 / 2000.0, size=nreq))
    which = rng.integers(0, len(scenes), size=nreq)
    lat, makespan = icr.serve(scenes, which, arrivals, n_slots=4)
    assert lat.shape == (nreq,) and np.all(lat > 0)
    assert makespan >= arrivals[-1]
    for sc, a in zip(scenes, alone):
        assert rel(sc.get("DQ"), a) < 1e-5


def test_serve_argument_and_state_errors(batch, torch_mod):
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    st = torch_mod.cuda.Stream()
    ctx = icr.Context(0, st.cuda_stream)
    sc = _load(icr, driver, ctx, batch[0])
    with pytest.raises(icr.IcrError) as e:
        icr.serve([sc], [0], [0.0], n_slots=1)
    assert e.value.code == icr.ESTATE
    sc.step_capture(batch[0].n_newton)
    with pytest.raises(icr.IcrError) as e:
        icr.serve([sc], [3], [0.0], n_slots=1)
    assert e.value.code == icr.EINVAL
    with pytest.raises(icr.IcrError) as e:
        icr.serve([sc], [0, 0], [0.5, 0.1], n_slots=1)
    assert e.value.code == icr.EINVAL
    default = icr.Context(0)
    sc2 = _load(icr, driver, default, batch[0])
    with pytest.raises(icr.IcrError) as e:
        sc2.step_capture(batch[0].n_newton)
    assert e.value.code == icr.EINVAL


# ---------------------------------------------------------------- warm start (Newton iteration 1)
@pytest.mark.parametrize("prec,tol", [(1, 1e-9), (0, 1e-4)])
def test_warm_started_steps_follow_the_oracle_chain(batch, torch_mod, prec, tol):
    """With warm_start, iteration 1 of each step starts from the previous
    step's iteration-1 lambda~; the oracle run with lam0 chained the same way
    gives the same steps.  Five sweeps keep PGS far from converged, so a warm
    and a cold start differ well above the tolerance."""
    from oracle import delassus as dl
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    s = batch[0]
    sweeps = 5
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    sc = icr.Scene(ctx, precision=prec, n_sweeps=sweeps, warm_start=True)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    driver.load_obstacle(sc, s.obstacle)
    sc.set_field("MU", s.mu)
    solver = dl.SystemSolver(s.A)
    cold = nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, sweeps, solver=solver)
    lam0 = None
    for j in range(3):
        sc.step(s.n_newton)
        ref = nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, sweeps,
                             lam0=lam0, solver=solver)
        lam0 = ref["iters"][0]["lam"]
        assert rel(sc.get("DQ"), ref["dq"]) < tol, f"step {j}"
        scale = max(np.linalg.norm(ref["iters"][-1]["lam"]), 1e-300)
        assert np.linalg.norm(sc.get("LAMBDA") - ref["iters"][-1]["lam"]) <= tol * scale
        if j > 0:
            assert rel(ref["dq"], cold["dq"]) > 100 * tol


def test_warm_started_scenes_alone_equal_the_mix(batch, torch_mod):
    """Warm-started scenes carry lambda~ from step to step; a scene served in
    the mix with others ends in the same state as the same number of its
    steps run alone."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    rng = np.random.default_rng(21)
    nreq = 30
    which = rng.integers(0, len(batch), size=nreq)
    arrivals = np.cumsum(rng.exponential(1.0 / 4000.0, size=nreq))

    def fresh():
        out = []
        for s in batch:
            ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
            sc = icr.Scene(ctx, precision=icr.FP32, n_sweeps=s.n_sweeps, warm_start=True)
            driver.load_system(sc, s.factor)
            driver.load_contacts(sc, s.nodes, s.bary, s.p0)
            driver.load_obstacle(sc, s.obstacle)
            sc.set_field("MU", s.mu)
            sc.step_capture(s.n_newton)
            out.append(sc)
        return out

    alone = fresh()
    for i, sc in enumerate(alone):
        for _ in range(int(np.sum(which == i))):
            sc.step_launch()
        sc.sync()
    mixed = fresh()
    icr.serve(mixed, which, arrivals, n_slots=3)
    # the contraction's atomic scatter-add makes W_H reproducible to rounding
    # only, so the comparison is at the FP32 tolerances (dq 1e-5, lambda~ 1e-4
    # of the step's largest lambda~, the first Newton iteration's)
    for a, b in zip(alone, mixed):
        assert rel(b.get("DQ"), a.get("DQ")) < 1e-5
        l0 = a.get("LAMBDA0")
        assert np.linalg.norm(l0) > 0
        assert rel(b.get("LAMBDA0"), l0) < 1e-4
        assert np.linalg.norm(b.get("LAMBDA") - a.get("LAMBDA")) <= 1e-4 * np.linalg.norm(l0)


def test_two_sphere_obstacle_errors(batch, torch_mod):
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    s = batch[0]
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    sc = icr.Scene(ctx, precision=icr.FP32)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    anchors = np.asarray(s.p0, dtype=np.float64)
    two = np.array([[0.0, 0.0, 1.0, 0.02], [1.0, 0.0, 0.0, 0.02]])
    for spheres, tool in [(two, np.full(s.m, 2)), (two, np.full(s.m, -1)),
                          (np.array([[0.0, 0.0, 1.0, 0.0]]), np.zeros(s.m))]:
        with pytest.raises(icr.IcrError) as e:
            sc.set_obstacle_spheres(spheres, tool, anchors)
        assert e.value.code == icr.EINVAL
    import ctypes as ct
    sc.params.warm_start = 2
    assert icr.lib().icr_set_params(sc.h, ct.byref(sc.params)) == icr.EINVAL


def test_captured_step_follows_new_inputs_and_detects_stale_graphs(batch, torch_mod):
    """A captured step reads the scene's buffers: loading the same-shape inputs
    again and relaunching reproduces the step; a different contact count makes
    the graph stale (ICR_ESTATE) until it is captured again."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    s, s2 = batch[0], batch[1]
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    sc = icr.Scene(ctx, precision=icr.FP32, n_sweeps=s.n_sweeps)
    driver.load_system(sc, s.factor)

    def load(x):
        driver.load_contacts(sc, x.nodes, x.bary, x.p0)
        driver.load_obstacle(sc, x.obstacle)
        sc.set_field("MU", x.mu)

    load(s)
    sc.step_capture(s.n_newton)
    sc.sync()
    first = sc.get("DQ")
    load(s)                      # same inputs again, same shape: the graph is still valid
    sc.step_launch()
    sc.sync()
    assert rel(sc.get("DQ"), first) < 1e-5
    sub = scenegen_subset(s, max(1, s.m // 2))
    load(sub)                    # fewer contacts: stale
    with pytest.raises(icr.IcrError) as e:
        sc.step_launch()
    assert e.value.code == icr.ESTATE
    sc.step_capture(sub.n_newton)
    sc.sync()
    assert np.all(np.isfinite(sc.get("DQ")))


def scenegen_subset(s, m):
    """The first m contacts of a scene (same system and obstacle kind)."""
    import copy
    t = copy.copy(s)
    t.nodes, t.bary, t.p0, t.mu = s.nodes[:m], s.bary[:m], s.p0[:m], s.mu[:m]
    ob = copy.copy(s.obstacle)
    ob.anchors = s.obstacle.anchors[:m]
    if ob.kind == "sphere":
        ob.tool = s.obstacle.tool[:m]
    else:
        ob.normals = s.obstacle.normals[:, :m]
    t.obstacle = ob
    return t


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)])
def test_step_inputs_in_one_call_equal_the_single_calls(batch, torch_mod, prec, tol):
    """icr_set_step_inputs (first call: the four single calls; later calls:
    one staged copy) gives the steps the single calls give, and a captured
    step graph stays valid across it."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    a, b = batch[0], batch[2]
    assert a.obstacle.kind == "sphere"

    def spheres(s):
        ob = s.obstacle
        return np.concatenate([np.asarray(ob.centers, dtype=np.float64).reshape(-1, 3),
                               np.asarray(ob.radii, dtype=np.float64).reshape(-1, 1)], axis=1)

    def single(s, inputs):
        ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
        sc = icr.Scene(ctx, precision=prec, n_sweeps=s.n_sweeps)
        driver.load_system(sc, s.factor)
        nodes, bary, p0, mu, sph, tool, anch = inputs
        sc.set_mapping(nodes, bary)
        sc.set_proximity(p0)
        sc.set_obstacle_spheres(sph, tool, anch)
        sc.set_field("MU", mu)
        sc.step(s.n_newton)
        sc.sync()
        return sc.get("DQ")

    ins_a = (a.nodes, a.bary, a.p0, a.mu, spheres(a), a.obstacle.tool, a.obstacle.anchors)
    # the same contacts moved: other proximity positions and friction, same count
    rng = np.random.default_rng(4)
    ins_b = (a.nodes, a.bary, np.asarray(a.p0) + 1e-4 * rng.standard_normal(np.shape(a.p0)), 0.5 * np.asarray(a.mu),
             spheres(a), a.obstacle.tool, a.obstacle.anchors)
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    sc = icr.Scene(ctx, precision=prec, n_sweeps=a.n_sweeps)
    driver.load_system(sc, a.factor)
    sc.set_step_inputs(*ins_a)              # no mapping yet: the single calls
    sc.step_capture(a.n_newton)
    sc.sync()
    assert rel(sc.get("DQ"), single(a, ins_a)) < tol
    for ins in (ins_b, ins_a):              # same count: one staged copy, the graph stays valid
        sc.set_step_inputs(*ins)
        sc.step_launch()
        sc.sync()
        assert rel(sc.get("DQ"), single(a, ins)) < tol
    # checks of the single calls apply on the staged path too
    bad = np.array(a.bary, dtype=np.float64).copy()
    bad[0, 0] += 0.5
    for args in [(a.nodes, bad) + ins_a[2:],
                 ins_a[:3] + (np.full(a.m, np.nan),) + ins_a[4:],
                 ins_a[:5] + (np.full(a.m, 7),) + ins_a[6:]]:
        with pytest.raises(icr.IcrError) as e:
            sc.set_step_inputs(*args)
        assert e.value.code == icr.EINVAL
    # another contact count: the single calls again, then a new capture
    sc.set_step_inputs(b.nodes, b.bary, b.p0, b.mu, spheres(b), b.obstacle.tool, b.obstacle.anchors)
    sc.step(b.n_newton)
    sc.sync()
    assert np.all(np.isfinite(sc.get("DQ")))


# ---------------------------------------------------------------- eviction and admission under a budget
FIELDS_KEPT = ("LAMBDA0", "LAMBDA", "P", "U", "DQ", "C", "DELTA", "MU")


def _warm_scene(icr, driver, ctx, s, prec=None):
    sc = icr.Scene(ctx, precision=icr.FP32 if prec is None else prec, n_sweeps=s.n_sweeps, warm_start=True)
    driver.load_system(sc, s.factor)
    driver.load_contacts(sc, s.nodes, s.bary, s.p0)
    driver.load_obstacle(sc, s.obstacle)
    sc.set_field("MU", s.mu)
    sc.step_capture(s.n_newton)
    return sc


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)])
def test_evict_readmit_restores_the_state_bitwise(batch, torch_mod, prec, tol):
    """An evicted scene gives its device memory back and refuses calls; once
    readmitted it holds the same bytes as before, and its next warm-started
    steps follow those of a twin that was never evicted."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    s = batch[1]
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    twin_ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    sc = _warm_scene(icr, driver, ctx, s, prec)
    twin = _warm_scene(icr, driver, twin_ctx, s, prec)
    for x in (sc, twin):
        for _ in range(2):
            x.step_launch()
        x.sync()
    before = {f: sc.get(f).copy() for f in FIELDS_KEPT}
    used = ctx.bytes_in_use()
    assert sc.residency() == (True, used)
    sc.evict()
    assert ctx.bytes_in_use() == 0 and sc.residency() == (False, used)
    for call in (lambda: sc.get("DQ"), sc.step_launch, sc.build_WH):
        with pytest.raises(icr.IcrError) as e:
            call()
        assert e.value.code == icr.ESTATE
    sc.evict()                               # a second eviction does nothing
    sc.readmit()
    assert ctx.bytes_in_use() == used and sc.residency() == (True, used)
    for f in FIELDS_KEPT:
        assert np.array_equal(sc.get(f), before[f]), f
    for x in (sc, twin):
        x.step_launch()
        x.sync()
    assert rel(sc.get("DQ"), twin.get("DQ")) < tol
    assert rel(sc.get("LAMBDA0"), twin.get("LAMBDA0")) < max(tol, 1e-4 if prec == 0 else tol)


def test_serve_evicts_and_readmits_under_a_budget(batch, torch_mod):
    """Scenes of one context whose budget holds about two of them: the request
    loop readmits each requested scene, evicting the least recently used idle
    ones, and every scene ends where the same steps run alone (never evicted)
    end."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    scenes_ = batch[:4]
    foot = []
    for s in scenes_:
        c = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
        x = _warm_scene(icr, driver, c, s)
        foot.append(x.residency()[1])
        x.close()
        c.close()
    budget = sorted(foot)[-1] + sorted(foot)[-2] + (1 << 20)
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream, hbm_budget=budget)
    served = []
    for s in scenes_:
        x = _warm_scene(icr, driver, ctx, s)
        x.evict()
        served.append(x)
    rng = np.random.default_rng(31)
    nreq = 24
    which = rng.integers(0, len(scenes_), size=nreq)
    which[:4] = np.arange(4)                 # every scene is requested
    arrivals = np.cumsum(rng.exponential(1.0 / 2000.0, size=nreq))
    lat, span, st = icr.serve(served, which, arrivals, n_slots=2, stats=True)
    assert st["rejected"] == 0 and np.all(lat >= 0)
    assert st["evictions"] > 0 and st["readmissions"] >= len(scenes_)
    assert ctx.bytes_in_use() <= budget
    alone = []
    for i, s in enumerate(scenes_):
        c = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
        x = _warm_scene(icr, driver, c, s)
        for _ in range(int(np.sum(which == i))):
            x.step_launch()
        x.sync()
        alone.append((c, x))
    for x in served:                         # read the scenes back one at a time
        x.evict()
    for x, (_, a) in zip(served, alone):
        x.readmit()
        assert rel(x.get("DQ"), a.get("DQ")) < 1e-5
        l0 = a.get("LAMBDA0")
        assert rel(x.get("LAMBDA0"), l0) < 1e-4
        x.evict()


def test_serve_rejects_a_scene_that_cannot_fit(batch, torch_mod):
    """A scene that does not fit next to memory the loop may not evict (a
    resident scene outside the request loop) is rejected, not waited for."""
    from paper_2306_06946_gb300 import build, driver, icr
    build.build()
    s = batch[0]
    c = icr.Context(0, torch_mod.cuda.Stream().cuda_stream)
    probe = _warm_scene(icr, driver, c, s)
    foot = probe.residency()[1]
    probe.close()
    c.close()
    ctx = icr.Context(0, torch_mod.cuda.Stream().cuda_stream, hbm_budget=int(1.5 * foot))
    other = _warm_scene(icr, driver, ctx, s)   # stays resident, not served
    other.evict()                              # room to load y ...
    y = _warm_scene(icr, driver, ctx, s)
    y.evict()
    other.readmit()                            # ... then other takes it back
    lat, _, st = icr.serve([y], np.zeros(3, np.int32), np.zeros(3), n_slots=1, stats=True)
    assert st["rejected"] == 3 and np.all(lat == -1.0)
    assert not y.residency()[0]
