"""The allocation-free reach entry point against the reach icr_build_WH computes.

Callers that cannot allocate device memory (a real-time loop that forbids
allocation after start-up, or a framework that owns all device memory) use
icr_reach_noalloc with buffers they own; its working memory is a fixed static
device array.  This file is collected last so that a failure here leaves every
other test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reach_via_build(ctx, scene):
    from paper_2306_06946_gb300 import driver, icr
    sc = icr.Scene(ctx, precision=icr.FP32)
    driver.load_system(sc, scene.factor)
    driver.load_contacts(sc, scene.nodes, scene.bary, scene.p0)
    sc.build_WH()
    return sc.get("REACH_PTR"), sc.get("REACH_IDX")


@pytest.mark.parametrize("name", ["beam_c0", "liver_c1"])
def test_reach_noalloc_matches_build(name):
    torch = pytest.importorskip("torch")
    import scenegen
    from paper_2306_06946_gb300 import build, icr
    build.build()
    scene = scenegen.NAMED[name]()
    sym = scene.factor.sym
    ns, m, n_nodes = sym.nsuper, scene.m, scene.n // 3
    node_super = np.repeat(np.arange(ns), np.diff(sym.super_ptr))[0::3].astype(np.int32)
    dev = torch.device("cuda", 0)
    d_nodes = torch.from_numpy(scene.nodes.astype(np.int32)).to(dev)
    d_ns = torch.from_numpy(node_super).to(dev)
    d_par = torch.from_numpy(sym.parent.astype(np.int32)).to(dev)
    ctx = icr.Context(0)
    ptr_ref, idx_ref = _reach_via_build(ctx, scene)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):          # two calls in a row share the static scratch
        d_cnt = torch.full((ns,), -7, dtype=torch.int32, device=dev)
        d_idx = torch.full((ns * m,), -7, dtype=torch.int32, device=dev)
        icr.reach_noalloc(m, ns, n_nodes, d_nodes.data_ptr(), d_ns.data_ptr(), d_par.data_ptr(),
                          d_cnt.data_ptr(), d_idx.data_ptr(), stream)
        cnt = d_cnt.cpu().numpy()
        idx = d_idx.cpu().numpy().reshape(ns, m)
        assert np.array_equal(np.concatenate([[0], np.cumsum(cnt)]), ptr_ref)
        got = np.concatenate([idx[s, :cnt[s]] for s in range(ns)])
        assert np.array_equal(got, idx_ref)


def test_reach_noalloc_rejects_oversized_problems():
    torch = pytest.importorskip("torch")
    from paper_2306_06946_gb300 import build, icr
    build.build()
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(16, dtype=torch.int32, device=dev)
    nsuper = icr.NOALLOC_SCRATCH_WORDS // 1000 + 1      # x ceil(32000/32) words > the scratch
    with pytest.raises(icr.IcrError) as e:
        icr.reach_noalloc(32000, nsuper, 4, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                          dummy.data_ptr(), dummy.data_ptr(), 0)
    assert e.value.code == icr.EINVAL
    assert "static scratch" in str(e.value)


def test_reach_noalloc_rejects_bad_ids():
    """Ids out of range and a parent below its child give ICR_EINVAL (the
    kernel checks every id before it indexes with it); a good call afterwards
    still matches the build."""
    torch = pytest.importorskip("torch")
    import scenegen
    from paper_2306_06946_gb300 import build, icr
    build.build()
    scene = scenegen.NAMED["beam_c0"]()
    sym = scene.factor.sym
    ns, m, n_nodes = sym.nsuper, scene.m, scene.n // 3
    node_super = np.repeat(np.arange(ns), np.diff(sym.super_ptr))[0::3].astype(np.int32)
    parent = sym.parent.astype(np.int32)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(dev)
    d_cnt = torch.zeros(ns, dtype=torch.int32, device=dev)
    d_idx = torch.zeros(ns * m, dtype=torch.int32, device=dev)

    def call(nodes, nsup, par):
        dn, ds, dp = t(nodes), t(nsup), t(par)
        icr.reach_noalloc(m, ns, n_nodes, dn.data_ptr(), ds.data_ptr(), dp.data_ptr(), d_cnt.data_ptr(),
                          d_idx.data_ptr(), 0)

    bad_node = scene.nodes.astype(np.int32).copy()
    bad_node[3, 1] = n_nodes                      # one node id past the end
    neg_super = node_super.copy()
    neg_super[scene.nodes[0, 0]] = -2             # a negative supernode id
    bad_parent = parent.copy()
    leaf = int(node_super[scene.nodes[0, 0]])
    bad_parent[leaf] = 0 if leaf > 0 else leaf    # a parent not above its child
    for args in [(bad_node, node_super, parent), (scene.nodes, neg_super, parent),
                 (scene.nodes, node_super, bad_parent)]:
        with pytest.raises(icr.IcrError) as e:
            call(*args)
        assert e.value.code == icr.EINVAL
    call(scene.nodes, node_super, parent)
    ctx = icr.Context(0)
    ptr_ref, idx_ref = _reach_via_build(ctx, scene)
    cnt = d_cnt.cpu().numpy()
    assert np.array_equal(np.concatenate([[0], np.cumsum(cnt)]), ptr_ref)


def test_reach_noalloc_refuses_a_capturing_stream():
    torch = pytest.importorskip("torch")
    from paper_2306_06946_gb300 import build, icr
    build.build()
    dev = torch.device("cuda", 0)
    buf = torch.zeros(64, dtype=torch.int32, device=dev)
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        g.capture_begin()
        try:
            with pytest.raises(icr.IcrError) as e:
                icr.reach_noalloc(1, 1, 4, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                  buf.data_ptr(), st.cuda_stream)
        finally:
            g.capture_end()
    assert e.value.code == icr.ESTATE
