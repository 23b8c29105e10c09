"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: a
dense inverse, closed forms, brute-force enumeration, the exactness of the
reformulation, invariants (symmetry, PSD, complementarity) and the paper's
own printed table.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import delassus as dl
from oracle import newton as nw
from oracle import pgs as pg
from oracle import reach as rc
import scenegen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    # 4x3x3-node beam, 8 contacts: small enough for dense inverses everywhere
    return scenegen.beam_scene(nodes_xyz=(4, 3, 3), m=8, seed=3, n_newton=3, n_sweeps=40, leaf_nodes=6)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- fixture pins
def test_factor_reconstructs_A(beam_c0):
    F = beam_c0.factor
    L = F.to_sparse_L()
    R = (L @ sp.diags(F.D) @ L.T - beam_c0.A)
    assert abs(R).max() <= 1e-13 * abs(beam_c0.A).max()
    assert np.all(F.D > 0)


def test_factor_reconstructs_A_liver(liver_c1):
    F = liver_c1.factor
    L = F.to_sparse_L()
    R = (L @ sp.diags(F.D) @ L.T - liver_c1.A)
    assert abs(R).max() <= 1e-13 * abs(liver_c1.A).max()


def test_supernodes_hold_whole_nodes(beam_c0, liver_c1):
    for s in (beam_c0, liver_c1):
        assert np.all(s.factor.sym.super_ptr % 3 == 0)
        par = s.factor.sym.parent
        assert np.all((par == -1) | (par > np.arange(par.size)))


def test_material_matrix_special_values():
    # C0 reading: A = (1 + h a_M) M + (h a_K + h^2) K = 1.001 M + 0.0011 K
    from scenegen.fem import assemble
    from scenegen.mesh import beam
    X, T = beam((2, 2, 2), 0.01)
    A, mdiag, K = assemble(X, T)
    ref = 1.001 * sp.diags(mdiag) + 0.0011 * K
    assert abs(A - ref).max() <= 1e-12 * abs(A).max()
    # rigid translations are in the null space of K; total mass = rho * volume
    t = np.tile([1.0, 0.0, 0.0], X.shape[0])
    assert np.abs(K @ t).max() <= 1e-9 * abs(K).max()
    assert np.isclose(mdiag[0::3].sum(), 1000.0 * 0.01 ** 3)


# ---------------------------------------------------------------- H, C, J, W
def test_mapping_matrix_reproduces_barycentric_points(beam_c0):
    s = beam_c0
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    q = s.X.reshape(-1)                       # positions as the DOF vector 3*node + axis
    assert np.allclose(H @ q, s.p0.reshape(-1), atol=1e-15)
    assert H.shape == (3 * s.m, s.n)


def test_W_matches_dense_inverse(tiny):
    s = tiny
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    C, _ = s.linearize(s.p0, 0)
    J = dl.jacobian(C, H)
    W = dl.delassus_standard(dl.SystemSolver(s.A), J)
    Ainv = np.linalg.inv(s.A.toarray())
    Jd = np.zeros((3 * s.m, s.n))
    for a in range(s.m):                      # J written out entry by entry
        for r in range(3):
            for i in range(4):
                for d in range(3):
                    Jd[3 * a + r, 3 * s.nodes[a, i] + d] += C[a, r, d] * s.bary[a, i]
    assert _rel(W, Jd @ Ainv @ Jd.T) < 1e-12


def test_reformulation_is_exact(beam_c0):
    s = beam_c0
    solver = dl.SystemSolver(s.A)
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    C, _ = s.linearize(s.p0, 1)
    W_std = dl.delassus_standard(solver, dl.jacobian(C, H))
    W_fast = dl.delassus_fast(C, dl.compliance_mapping(solver, H))
    assert _rel(W_fast, W_std) < 1e-12
    assert np.linalg.norm(W_std - W_std.T) <= 1e-13 * np.linalg.norm(W_std)
    # PD: 3m <= n and the contact points are distinct
    np.linalg.cholesky(W_std + 1e-14 * np.trace(W_std) * np.eye(W_std.shape[0]))


def test_WH_identity_system_closed_form():
    # A = I gives W_H = H H^T; one contact gives sum_i w_i^2 on the 3x3 diagonal
    nodes = np.array([[0, 1, 2, 3], [2, 3, 4, 5]])
    bary = np.array([[0.1, 0.2, 0.3, 0.4], [0.25, 0.25, 0.25, 0.25]])
    n = 18
    H = dl.mapping_matrix(nodes, bary, n)
    WH = dl.compliance_mapping(dl.SystemSolver(sp.identity(n, format="csc")), H)
    assert np.allclose(WH[:3, :3], 0.30 * np.eye(3), atol=1e-15)
    assert np.allclose(WH[3:, 3:], 0.25 * np.eye(3), atol=1e-15)
    # shared nodes 2 and 3: w_2 w'_0 + w_3 w'_1 = 0.3*0.25 + 0.4*0.25
    assert np.allclose(WH[:3, 3:], 0.175 * np.eye(3), atol=1e-15)


def test_WH_lumped_mass_closed_form():
    # single tet, K = 0, diagonal lumped mass m_i per node: W_H = sum_i w_i^2 / m_i
    w = np.array([0.4, 0.3, 0.2, 0.1])
    mass = np.array([1.0, 2.0, 4.0, 8.0])
    A = sp.diags(np.repeat(mass, 3)).tocsc()
    H = dl.mapping_matrix(np.array([[0, 1, 2, 3]]), w[None, :], 12)
    WH = dl.compliance_mapping(dl.SystemSolver(A), H)
    assert np.allclose(WH, np.sum(w ** 2 / mass) * np.eye(3), rtol=1e-14)


def test_direction_matrix_is_block_transpose_sensitive():
    # C has rows n, t1, t2: J = C H maps q to (n.p, t1.p, t2.p)
    from scenegen.contacts import tangent_frame
    n = np.array([[0.0, 0.6, 0.8]])
    C = tangent_frame(n)
    H = dl.mapping_matrix(np.array([[0, 1, 2, 3]]), np.array([[1.0, 0, 0, 0]]), 12)
    q = np.zeros(12)
    q[:3] = [1.0, 2.0, 3.0]
    assert np.allclose(dl.jacobian(C, H) @ q, C[0] @ q[:3])
    assert np.isclose((dl.jacobian(C, H) @ q)[0], 0.6 * 2 + 0.8 * 3)


def test_tangent_frame_reading():
    from scenegen.contacts import tangent_frame
    C = tangent_frame(np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.6, 0.0, 0.8]]))
    # n = +z: smallest |n_a| ties between x and y -> x; t1 = z x x = +y, t2 = z x y = -x
    assert np.allclose(C[0], [[0, 0, 1], [0, 1, 0], [-1, 0, 0]])
    for blk in C:
        assert np.allclose(blk @ blk.T, np.eye(3), atol=1e-15)
        assert np.isclose(np.linalg.det(blk), 1.0)


# ---------------------------------------------------------------- PGS
def test_pgs_single_contact_closed_form():
    W = np.diag([2.0, 3.0, 3.0])
    mu = np.array([0.5])
    # frictionless-looking: small tangential gap stays inside the cone
    lam, _, _ = pg.pgs(W, np.array([-1.0, 0.1, -0.2]), mu, sweeps=3)
    assert np.allclose(lam, [0.5, -0.1 / 3, 0.2 / 3])
    # large slip: tangential force saturates on the cone, opposite to the slip
    lam, _, _ = pg.pgs(W, np.array([-1.0, 3.0, 4.0]), mu, sweeps=3)
    assert np.allclose(lam, [0.5, -0.15, -0.2])
    # separated: positive normal gap gives no force at all
    lam, _, _ = pg.pgs(W, np.array([0.3, 3.0, 4.0]), mu, sweeps=3)
    assert np.allclose(lam, 0.0)


def _lcp_bruteforce(Wn, dn):
    m = dn.size
    for k in range(m + 1):
        for S in itertools.combinations(range(m), k):
            S = list(S)
            lam = np.zeros(m)
            if S:
                lam[S] = np.linalg.solve(Wn[np.ix_(S, S)], -dn[S])
            w = dn + Wn @ lam
            if np.all(lam >= -1e-12) and np.all(w >= -1e-12):
                return lam
    raise AssertionError("no LCP solution")


def test_pgs_frictionless_matches_enumerated_lcp(tiny):
    s = tiny
    solver = dl.SystemSolver(s.A)
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_standard(solver, dl.jacobian(C, H))
    mu = np.zeros(s.m)
    lam, _, _ = pg.pgs(W, delta, mu, sweeps=4000)
    ref = _lcp_bruteforce(W[0::3, 0::3], delta[0::3])
    assert 0 < np.count_nonzero(ref) < s.m
    assert np.allclose(lam[0::3], ref, rtol=1e-7, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(lam[1::3], 0) and np.allclose(lam[2::3], 0)


def test_pgs_full_stick_is_linear_solve():
    # gaps built as delta = -W lambda* with lambda* strictly inside every cone:
    # with mu -> infinity every contact sticks and PGS must return lambda*
    m = 12
    rng = np.random.default_rng(11)
    G = rng.normal(size=(3 * m, 3 * m))
    W = G @ G.T / (3 * m) + np.eye(3 * m)
    ref = np.zeros(3 * m)
    ref[0::3] = rng.uniform(0.5, 1.5, m)
    ref[1::3] = rng.uniform(-0.2, 0.2, m)
    ref[2::3] = rng.uniform(-0.2, 0.2, m)
    lam, _, _ = pg.pgs(W, -W @ ref, np.full(m, 1e6), sweeps=4000)
    assert _rel(lam, ref) < 1e-10
    assert np.array_equal(pg.classify(lam, np.full(m, 1e6)), np.full(m, pg.STICK))


def test_pgs_friction_residuals_vanish(beam_c0):
    s = beam_c0
    solver = dl.SystemSolver(s.A)
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_standard(solver, dl.jacobian(C, H))
    lam, _, eps = pg.pgs(W, delta, s.mu, sweeps=3000)
    res = pg.residuals(W, delta, lam, s.mu)
    scale = np.abs(delta).max()
    assert res["normal"] < 1e-8 * scale and res["stick"] < 1e-8 * scale and res["slip"] < 1e-8 * scale
    assert res["cone"] < 1e-12 * np.abs(lam).max()
    cls = pg.classify(lam, s.mu)
    assert {0, 1, 2} <= set(cls.tolist())     # the C0 mix has all three states


def test_pgs_tol_stops_early(beam_c0):
    s = beam_c0
    solver = dl.SystemSolver(s.A)
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    C, delta = s.linearize(s.p0, 0)
    W = dl.delassus_standard(solver, dl.jacobian(C, H))
    lam, done, eps = pg.pgs(W, delta, s.mu, sweeps=5000, tol=1e-6)
    assert done < 5000 and eps <= 1e-6
    lam2, _, _ = pg.pgs(W, delta, s.mu, sweeps=done)
    assert np.array_equal(lam, lam2)


# ---------------------------------------------------------------- Newton loops
def test_standard_and_fast_schemes_agree(beam_c0):
    s = beam_c0
    kw = dict(A=s.A, nodes=s.nodes, bary=s.bary, mu=s.mu, p0=s.p0, linearize=s.linearize,
              n_newton=s.n_newton, sweeps=s.n_sweeps)
    std = nw.standard_scheme(**kw)
    fast = nw.fast_scheme(**kw)
    for a, b in zip(std["iters"], fast["iters"]):
        assert _rel(b["W"], a["W"]) < 1e-11
        assert _rel(b["lam"], a["lam"]) < 1e-10
        assert _rel(b["p"], a["p"]) < 1e-12
    assert _rel(fast["dq"], std["dq"]) < 1e-10


def test_corrective_motion_residual(beam_c0):
    s = beam_c0
    fast = nw.fast_scheme(s.A, s.nodes, s.bary, s.mu, s.p0, s.linearize, s.n_newton, s.n_sweeps)
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    rhs = H.T @ fast["u"]
    assert np.linalg.norm(s.A @ fast["dq"] - rhs) <= 1e-12 * np.linalg.norm(rhs)
    assert np.linalg.norm(fast["u"]) > 0


def test_newton_fixed_directions_accumulate(tiny):
    # with C_k fixed and every contact resolved in iteration 1, iteration 2 has
    # nothing left to correct: the total dq equals the one-iteration dq
    s = tiny
    C0, d0 = s.linearize(s.p0, 0)
    anchors = s.p0 + 1e-4 * C0[:, 0, :]       # every normal gap -0.1 mm, no slip

    def lin(p, k):
        return C0, np.einsum("mij,mj->mi", C0, p - anchors).reshape(-1)

    one = nw.fast_scheme(s.A, s.nodes, s.bary, np.zeros(s.m), s.p0, lin, 1, 6000)
    two = nw.fast_scheme(s.A, s.nodes, s.bary, np.zeros(s.m), s.p0, lin, 2, 6000)
    assert np.abs(two["iters"][1]["lam"]).max() <= 1e-9 * np.abs(one["iters"][0]["lam"]).max()
    assert _rel(two["dq"], one["dq"]) < 1e-8


# ---------------------------------------------------------------- reach
def _reach_mismatches(reach, scene) -> int:
    """Supernodes whose contact list differs from the contacts with a non-zero
    in the supernode's rows of X = L^-1 H^T, formed densely by forward
    substitution on the fixture's unit lower factor (exact zeros stay zero:
    every product of a structural zero is an exact zero)."""
    import scipy.linalg as sla
    sym = scene.factor.sym
    L = scene.factor.to_sparse_L().toarray()
    H = dl.mapping_matrix(scene.nodes, scene.bary, scene.n).toarray()
    X = sla.solve_triangular(L, H.T, lower=True, unit_diagonal=True)
    sod = rc.supernode_of_dof(sym.super_ptr)
    bad = 0
    for sn in range(sym.nsuper):
        rows = sod == sn
        hit = [a for a in range(scene.m) if np.any(X[rows, 3 * a:3 * a + 3] != 0)]
        bad += hit != list(reach[sn])
    return bad


@pytest.fixture(scope="module")
def reach_scenes():
    # random barycentric weights: no cancellation in L^-1 H^T
    return [scenegen.beam_scene(nodes_xyz=(6, 3, 3), m=10, seed=5, leaf_nodes=4),
            scenegen.ellipsoid_scene(target_nodes=500, m=60, seed=4, leaf_nodes=8)]


def test_reach_equals_nonzero_structure(reach_scenes):
    for s in reach_scenes:
        sym = s.factor.sym
        reach = rc.contact_reach(sym.parent, sym.super_ptr, s.nodes)
        assert _reach_mismatches(reach, s) == 0, s.name
        assert sum(len(r) for r in reach) < sym.nsuper * s.m      # not every contact everywhere


def test_reach_pin_catches_planted_mistakes(reach_scenes):
    s = reach_scenes[1]
    sym = s.factor.sym
    reach = rc.contact_reach(sym.parent, sym.super_ptr, s.nodes)
    # over-reach: every contact reaches every supernode
    assert _reach_mismatches([list(range(s.m))] * sym.nsuper, s) > 0
    # over-reach by one: contact 0 added to one supernode off its etree paths
    off = next(sn for sn in range(sym.nsuper) if 0 not in reach[sn])
    planted = [list(r) for r in reach]
    planted[off] = sorted(planted[off] + [0])
    assert _reach_mismatches(planted, s) == 1
    # under-reach: the walk stops below the root
    roots = set(np.nonzero(sym.parent < 0)[0].tolist())
    planted = [[] if sn in roots else list(r) for sn, r in enumerate(reach)]
    assert _reach_mismatches(planted, s) == len(roots)


# ---------------------------------------------------------------- PGS residuals and states
# Single contacts with a chosen lambda~, the gaps d = delta + W lambda~ it
# leaves and mu; each with its residuals and state written down by hand from
# Eqs. "signorini's law" and "coulomb's law" (disc reading) and maximal
# dissipation.  W is a random non-symmetric 3x3 block, so delta = d - W lambda~
# is only right if the residual is formed with W lambda~ (not W^T lambda~).
RES_CASES = [
    # name, lambda~, d, mu, {normal, cone, stick, slip}, state
    ("stick", (1.0, 0.1, 0.0), (0.0, 0.3, -0.4), 0.5, dict(stick=0.5), pg.STICK),
    ("slip_aligned", (1.0, 0.3, 0.4), (0.0, -1.2, -1.6), 0.5, dict(), pg.SLIP),
    ("slip_misaligned", (1.0, 0.3, 0.4), (0.0, -1.4, -1.45), 0.5, dict(slip=0.25), pg.SLIP),
    ("slip_with_force", (1.0, 0.3, 0.4), (0.0, 0.06, 0.08), 0.5, dict(slip=0.1), pg.SLIP),
    ("cone_violated", (1.0, 0.6, 0.8), (0.0, -0.6, -0.8), 0.5, dict(cone=0.5), pg.SLIP),
    ("separated_open", (0.0, 0.0, 0.0), (0.2, 5.0, 5.0), 0.5, dict(), pg.SEPARATED),
    ("separated_penetrating", (0.0, 0.0, 0.0), (-0.2, 0.0, 0.0), 0.5, dict(normal=0.2), pg.SEPARATED),
    ("loaded_open", (0.3, 0.0, 0.0), (0.1, 0.0, 0.0), 0.5, dict(normal=0.1), pg.STICK),
    ("frictionless_sliding", (1.0, 0.0, 0.0), (0.0, 0.7, 0.0), 0.0, dict(), pg.SLIP),
]


def _res_case(lam, d, mu, residuals=pg.residuals):
    W = np.random.default_rng(7).normal(size=(3, 3)) + 3 * np.eye(3)
    lam = np.asarray(lam, dtype=np.float64)
    delta = np.asarray(d, dtype=np.float64) - W @ lam
    return residuals(W, delta, lam, np.array([mu]))


def _residual_pin_failures(residuals=pg.residuals, classify=pg.classify):
    bad = []
    for name, lam, d, mu, want, state in RES_CASES:
        got = _res_case(lam, d, mu, residuals)
        for key in ("normal", "cone", "stick", "slip"):
            if abs(got[key] - want.get(key, 0.0)) > 1e-12:
                bad.append((name, key, got[key]))
        if classify(np.asarray(lam, dtype=np.float64), np.array([mu]))[0] != state:
            bad.append((name, "state"))
    return bad


def test_residuals_and_states_on_hand_built_contacts():
    assert _residual_pin_failures() == []
    # several contacts at once: the maxima over contacts, W block-diagonal
    k = len(RES_CASES)
    W = np.zeros((3 * k, 3 * k))
    lam = np.zeros(3 * k)
    d = np.zeros(3 * k)
    for i, (_, l, dd, _, _, _) in enumerate(RES_CASES):
        W[3 * i:3 * i + 3, 3 * i:3 * i + 3] = np.random.default_rng(i).normal(size=(3, 3)) + 3 * np.eye(3)
        lam[3 * i:3 * i + 3] = l
        d[3 * i:3 * i + 3] = dd
    mu = np.array([c[3] for c in RES_CASES])
    got = pg.residuals(W, d - W @ lam, lam, mu)
    assert got == pytest.approx({"normal": 0.2, "cone": 0.5, "stick": 0.5, "slip": 0.25}, abs=1e-12)
    assert pg.classify(lam, mu).tolist() == [c[5] for c in RES_CASES]


def test_residual_pins_catch_planted_mistakes():
    swapped = lambda lam, mu, rel=1e-9: np.choose(pg.classify(lam, mu, rel), [0, 2, 1])   # stick <-> slip
    assert _residual_pin_failures(classify=swapped)
    transposed = lambda W, delta, lam, mu, rel=1e-9: pg.residuals(W.T, delta, lam, mu, rel)
    assert _residual_pin_failures(residuals=transposed)

    def no_dissipation(W, delta, lam, mu, rel=1e-9):      # slip residual without the along term
        r = pg.residuals(W, delta, lam, mu, rel)
        d = (delta + W @ lam).reshape(-1, 3)
        if lam[0] > 0 and np.linalg.norm(lam[1:]) > 0:
            t = lam[1:] / np.linalg.norm(lam[1:])
            r["slip"] = float(np.linalg.norm(d[0, 1:] - (d[0, 1:] @ t) * t))
        return r
    assert _residual_pin_failures(residuals=no_dissipation)


def test_classification_margin():
    lam = np.array([1.0, 0.3, 0.4 * (1 - 1e-7)])      # ||lambda_t|| just inside mu lambda_n = 0.5
    assert pg.classify(lam, np.array([0.5]))[0] == pg.STICK
    assert pg.classify(lam, np.array([0.5]), rel=1e-5)[0] == pg.SLIP


# ---------------------------------------------------------------- paper table
def test_paper_table_arithmetic():
    t = json.load(open(os.path.join(GOLD, "table_fast_vs_standard.json")))
    k = t["newton_iterations"]
    rn, rt = [], []
    for row in t["rows"]:
        st, fa = row["standard"], row["fast"]
        assert abs(st["rebuild_W"] + st["pgs"] + st["corr"] - st["newton"]) < 0.015
        assert abs(fa["rebuild_W"] + fa["pgs"] + fa["corr"] - fa["newton"]) < 0.015
        assert abs(fa["build_WH"] + k * fa["newton"] - fa["total"]) < 0.05
        assert abs(k * st["newton"] - st["total"]) < 0.05
        # "Update" is the share of rebuilding W plus the correction in one Newton iteration
        for v in (st, fa):
            assert abs(100 * (v["rebuild_W"] + v["corr"]) / v["newton"] - v["update_pct"]) < 0.1
        rn.append(st["newton"] / fa["newton"])
        rt.append(st["total"] / fa["total"])
    assert abs(np.mean(rn) - t["speedup_newton"]) < 0.01
    assert abs(np.mean(rt) - t["speedup_total"]) < 0.02


def test_solver_orderings_agree(beam_c0):
    # the column ordering of the sparse LU changes rounding only
    s = beam_c0
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    a = dl.compliance_mapping(dl.SystemSolver(s.A), H)
    b = dl.compliance_mapping(dl.SystemSolver(s.A, ordering="NATURAL"), H)
    Ainv = np.linalg.inv(s.A.toarray())
    ref = H.toarray() @ Ainv @ H.T.toarray()
    assert _rel(a, ref) < 1e-12 and _rel(b, ref) < 1e-12


def test_column_blocks_form_WH(beam_c0):
    # W_H assembled from column blocks equals W_H formed at once, and the
    # fast scheme given it repeats the fast scheme that forms it
    s = beam_c0
    H = dl.mapping_matrix(s.nodes, s.bary, s.n)
    whole = dl.compliance_mapping(dl.SystemSolver(s.A), H)
    cols = np.array_split(np.arange(3 * s.m), 3)
    blocks = np.hstack([dl.compliance_columns(s.A, s.nodes, s.bary, c, "NATURAL") for c in cols])
    assert _rel(blocks, whole) < 1e-12
    kw = dict(A=s.A, nodes=s.nodes, bary=s.bary, mu=s.mu, p0=s.p0, linearize=s.linearize,
              n_newton=s.n_newton, sweeps=s.n_sweeps)
    a = nw.fast_scheme(**kw)
    b = nw.fast_scheme(**kw, WH=blocks)
    assert _rel(b["dq"], a["dq"]) < 1e-11


# ---------------------------------------------------------------- Newton stop (newton_tol)
def test_newton_stop_rule(beam_c0, liver_c1):
    # sphere tool: after iteration 1 every gap is open, so the skipped
    # iterations would solve to lambda~ = 0 and move nothing: the same dq
    s = liver_c1
    kw = dict(A=s.A, nodes=s.nodes, bary=s.bary, mu=s.mu, p0=s.p0, linearize=s.linearize, sweeps=s.n_sweeps)
    full = nw.fast_scheme(**kw, n_newton=s.n_newton)
    cut = nw.fast_scheme(**kw, n_newton=s.n_newton, newton_tol=1e-12)
    assert len(cut["iters"]) == 1 and len(full["iters"]) == s.n_newton
    assert all(not it["lam"].any() for it in full["iters"][1:])
    assert _rel(cut["dq"], full["dq"]) < 1e-13
    # plane with new normals every iteration: the residual of a zero increment
    # after iteration 1 is above 1e-8, after iteration 2 below: two iterations,
    # the same as a two-iteration run
    b = beam_c0
    kw = dict(A=b.A, nodes=b.nodes, bary=b.bary, mu=b.mu, p0=b.p0, linearize=b.linearize, sweeps=b.n_sweeps)
    cut = nw.fast_scheme(**kw, n_newton=b.n_newton, newton_tol=1e-8)
    two = nw.fast_scheme(**kw, n_newton=2)
    assert len(cut["iters"]) == 2 < b.n_newton
    assert np.array_equal(cut["dq"], two["dq"])
    C, d = b.linearize(cut["iters"][-1]["p"].reshape(-1, 3), 2)
    assert nw.zero_increment_residual(d) <= 1e-8
    C, d = b.linearize(cut["iters"][0]["p"].reshape(-1, 3), 1)
    assert nw.zero_increment_residual(d) > 1e-8
    # the residual is the Signorini residual of lambda~ = 0 (oracle residuals())
    W = np.eye(3 * b.m)
    assert nw.zero_increment_residual(d) == pytest.approx(pg.residuals(W, d, np.zeros(3 * b.m), b.mu)["normal"],
                                                          rel=0, abs=0)
