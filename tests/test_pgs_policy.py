"""The S-only sweep policy of the PGS kernel, restated on the CPU, keeps the
iterate of plain sweeps (Eq. "PGS", contacts in ascending order).

A contact with lambda~ = 0 and a non-negative normal residual keeps
lambda~ = 0 under the local rule, so sweeps may pass over it.  The kernel, once
every residual is complete, visits only the blocks S that may change, while
the changes D of S since the bound's base stay within min beta / ws over the
other contacts (beta: a lower bound on its normal residual at the base, ws: its
largest coupling to the columns of S's blocks), checked after each visited
block.  When the bound runs out before a round of S, one fold and back to
full sweeps; after one, the other contacts' residuals decide: all
positive -> new base; some not -> their blocks join S when S stays within the
block limit, else one fold and back to full sweeps.
This restatement takes the same decisions with residuals formed from scratch,
so its iterate equals the oracle's exactly iff the contacts it passes over
would indeed not have changed."""
import numpy as np
import pytest

from oracle.pgs import local_solve, pgs

from pgs_cases import CASES, pulled_in


def s_only_pgs(W, delta, mu, BC=32, sweeps=50, max_blocks=16):
    """Returns (lambda~, sweeps, S-only sweeps, leaves, joins)."""
    m = mu.size
    nblk = (m + BC - 1) // BC
    lam = np.zeros(3 * m)
    # per contact and block: the largest |W[3a, j]| over the block's columns, a's own excluded
    wn = np.abs(W[0::3, :]).copy()
    for a in range(m):
        wn[a, 3 * a:3 * a + 3] = 0
    wblk = np.zeros((m, nblk))
    for B in range(nblk):
        wblk[:, B] = wn[:, 3 * B * BC:3 * min(m, (B + 1) * BC)].max(axis=1)
    margin = 1.0 / 1024.0

    def res():
        return delta + W @ lam

    def may_change(bb, r):
        return any(np.any(lam[3 * a:3 * a + 3] != 0) or r[3 * a] < 0 for a in range(bb * BC, min(m, (bb + 1) * BC)))

    def visit(bb):
        c = np.zeros(3 * m)
        for a in range(bb * BC, min(m, (bb + 1) * BC)):
            sl = slice(3 * a, 3 * a + 3)
            new = local_solve(lam[sl], delta[sl] + W[sl, :] @ lam, W[sl, sl], float(mu[a]))
            c[sl] = new - lam[sl]
            lam[sl] = new
        return c

    def others(S):
        return [a for a in range(m) if a // BC not in S]

    def theta(S, beta, ws):
        th = np.inf
        for a in others(S):
            v, w = beta[a], ws[a]
            th = min(th, (v / w if v > 0 else 0.0) if w > 0 else (np.inf if v > 0 else 0.0))
        return th * (1 - margin)

    def enter():
        """S, and for the other contacts the residual at the base (beta) and
        the coupling to S (ws); S empty when the S-only sweeps do not start."""
        r = res()
        S = [bb for bb in range(nblk) if may_change(bb, r)]
        beta, ws = r[0::3].copy(), np.zeros(m)
        if S:
            ws = wblk[:, S].max(axis=1)
        ok = len(S) <= max_blocks and len(S) < nblk and theta(S, beta, ws) > 0
        return (S if ok else []), beta, ws

    b, pb, known, chg_prev, chg_sweep = 0, -1, False, True, False
    S, th, D, D0, kpos, tryd, flag, pend = [], 0.0, None, None, 0, True, False, False
    since = 0   # visits of S's blocks since the bound's base
    beta = ws = None
    done = s_only = leaves = joins = 0

    def end_sweep():
        nonlocal chg_sweep, done, s_only, tryd
        brk = not chg_sweep
        chg_sweep = False
        s_only += bool(S)
        done += 1
        tryd = True
        return brk

    while done < sweeps:
        if S and flag:
            # the bound ran out: when it lasted a round of S, each other
            # contact's normal residual with the changes of S decides; else
            # one fold
            flag = False
            r = res()
            J = set(range(nblk)) if since < len(S) else set()
            for a in (others(S) if since >= len(S) else []):
                v = r[3 * a]
                beta[a] = v
                if not v > 0:
                    J.add(a // BC)
            if not J:
                th, D0, since = theta(S, beta, ws), D.copy(), 0
                if pend:
                    pend = False
                    if end_sweep():
                        break
                continue
            if since >= len(S) and len(S) + len(J) <= max_blocks:
                # the blocks of the contacts that may change join S; the sweep
                # goes on after pb in order, through them
                joins += 1
                S = sorted(set(S) | J)
                ws = np.maximum(ws, wblk[:, sorted(J)].max(axis=1))
                th, D0, since = theta(S, beta, ws), D.copy(), 0
                kpos = (S.index(pb) + 1) % len(S)
                pend, nxt = False, S[kpos]
                wrap = nxt <= pb
                b, pb = nxt, -1
                if wrap and end_sweep():
                    break
                continue
            pend = False
            leaves += 1
            S, tryd, b, pb, known, chg_prev = [], True, pb + 1, -1, False, False
            continue
        if not S and not known and not chg_prev:
            r = res()
            nb_ = next((bb for bb in range(b, nblk) if may_change(bb, r)), nblk)
            nw_ = next((bb for bb in range(nblk) if may_change(bb, r)), nblk)
            b = nb_
            if tryd and b < nblk:
                tryd = False
                S, beta, ws = enter()
                if S:
                    th, D, kpos, since = theta(S, beta, ws), np.zeros(3 * m), S.index(b), 0
                    D0 = D.copy()
            if b == nblk:
                brk = not chg_sweep
                chg_sweep = False
                done += 1
                if not brk and nw_ == nblk and done < sweeps:
                    done += 1
                    brk = True
                tryd = True
                if not brk and nw_ < nblk and done < sweeps:
                    tryd = False
                    S, beta, ws = enter()
                    if S:
                        th, D, kpos, since = theta(S, beta, ws), np.zeros(3 * m), 0, 0
                        D0 = D.copy()
                b, known = nw_, True
                if brk:
                    break
                continue
        known = False
        bn = S[(kpos + 1) % len(S)] if S else (b + 1) % nblk
        c = visit(b)
        chg_prev = bool(np.any(c != 0))
        chg_sweep = chg_sweep or chg_prev
        if S:
            D += c
            since += 1
            flag = not (np.abs(D - D0).sum() <= th)
        pb = b
        leave = bool(S) and flag
        pend = leave and bn <= b
        if bn <= b and not leave and end_sweep():
            break
        b = bn
        if S:
            kpos = (kpos + 1) % len(S)
    return lam, done, s_only, leaves, joins


@pytest.mark.parametrize("name", ["one_block", "three_blocks", "small_gaps", "last_block", "fixed_point",
                                  "joined_late", "folds"])
@pytest.mark.parametrize("BC", [32, 16])
def test_s_only_policy_keeps_the_plain_iterate(name, BC):
    make, expect = CASES[name]
    W, delta, mu = make()
    lam, done, s_only, leaves, joins = s_only_pgs(W, delta, mu, BC=BC)
    ref, sw, _ = pgs(W, delta, mu, None, 50)
    assert np.array_equal(lam, ref) and done == sw
    assert s_only > 0 or expect == "leave"
    if expect == "leave":
        assert leaves > 0
    if expect == "join":
        assert joins > 0


def test_s_only_policy_off_above_the_block_limit():
    W, delta, mu = CASES["many_blocks"][0]()
    W, delta, mu = W[:1200, :1200], delta[:1200], mu[:400]     # 13 blocks of 32 with 2 active contacts each
    lam, done, s_only, _, _ = s_only_pgs(W, delta, mu, BC=32, max_blocks=12)
    ref, sw, _ = pgs(W, delta, mu, None, 50)
    assert np.array_equal(lam, ref) and done == sw and s_only == 0


def test_passing_over_a_contact_that_would_change_breaks_the_iterate():
    """Planted mistake: sweeping only the block that starts in contact, with
    no bound, never visits the contacts it pulls in, and the iterate departs
    from plain sweeps; the policy (bound, recheck) keeps it."""
    W, delta, mu = pulled_in()
    m = mu.size
    ref, sw, _ = pgs(W, delta, mu, None, 50)
    assert np.all(ref.reshape(-1, 3)[[70, 80], 0] > 0)   # pulled into contact
    lam, done, s_only, _, _ = s_only_pgs(W, delta, mu)
    assert np.array_equal(lam, ref) and done == sw and s_only > 0
    bad = np.zeros(3 * m)
    for _ in range(50):
        for a in range(32):
            sl = slice(3 * a, 3 * a + 3)
            bad[sl] = local_solve(bad[sl], delta[sl] + W[sl, :] @ bad, W[sl, sl], float(mu[a]))
    assert np.all(bad.reshape(-1, 3)[[70, 80], 0] == 0)
    assert not np.allclose(bad, ref)
