"""Synthetic PGS instances shared by the S-only sweep tests (CPU and GPU).

W is a dense SPD matrix kron(K, M): K an exponential kernel over random
contact positions on a line (coupling that decays with distance, as between
contacts on a body), M a fixed 3x3 SPD block; negative normal gaps make the
chosen contacts active, the others have positive gaps drawn log-uniformly.
pulled_in is a random dense SPD W (couplings of both signs) where the pressed
contacts pull two far contacts into contact.
"""
import numpy as np


def synth(m, active, gaps, seed, ell=0.05):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(0.0, 1.0, m))
    K = np.exp(-np.abs(x[:, None] - x[None, :]) / ell)
    M = np.array([[1.0, 0.3, -0.2], [0.3, 0.8, 0.1], [-0.2, 0.1, 0.7]])
    W = np.kron(K, M)
    delta = np.zeros(3 * m)
    lo, hi = gaps
    delta[0::3] = np.exp(rng.uniform(np.log(lo), np.log(hi), m))
    delta[3 * np.asarray(active)] = -rng.uniform(0.01, 0.03, len(active))
    delta[1::3] = 0.01 * rng.standard_normal(m)
    delta[2::3] = 0.01 * rng.standard_normal(m)
    mu = rng.uniform(0.2, 0.5, m)
    return W, delta, mu


def many_active():
    act = sorted([32 * k + 3 for k in range(20)] + [32 * k + 10 for k in range(20)])
    W, d, mu = synth(700, act, (0.05, 0.1), 7)
    d[3 * np.asarray(act)] = -0.05
    return W, d, mu


def pulled_in(seed=1, m=96):
    """Random dense SPD W (couplings of both signs); contacts 3, 5, 8 (block 0)
    pressed in, 70 and 80 (block 2) almost touching: the pressed contacts'
    impulses pull those two into contact."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3 * m, 3 * m // 2)) / np.sqrt(3 * m)
    W = A @ A.T + 0.5 * np.eye(3 * m)
    d = np.zeros(3 * m)
    d[0::3] = rng.uniform(5e-2, 1e-1, m)
    d[1::3] = 0.01 * rng.standard_normal(m)
    d[2::3] = 0.01 * rng.standard_normal(m)
    d[3 * np.array([3, 5, 8])] = -0.2
    d[3 * np.array([70, 80])] = 2e-4
    return W, d, rng.uniform(0.2, 0.5, m)


def _random_spd(seed, m, pressed):
    """Random dense SPD W (couplings of both signs), positive gaps, the
    pressed contacts' normal gaps -0.2."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3 * m, 3 * m // 2)) / np.sqrt(3 * m)
    W = A @ A.T + 0.5 * np.eye(3 * m)
    d = np.zeros(3 * m)
    d[0::3] = rng.uniform(5e-2, 1e-1, m)
    d[1::3] = 0.01 * rng.standard_normal(m)
    d[2::3] = 0.01 * rng.standard_normal(m)
    d[3 * np.asarray(pressed)] = -0.2
    return W, d, rng.uniform(0.2, 0.5, m)


def joined_late():
    """Contacts 3, 5, 8 (block 0) pressed in; contact 67 (block 2, 32 contacts
    a block; block 4 with 16) has a gap just under the pull the pressed
    contacts' impulses reach by the end, so it first goes negative in sweep 3,
    after the S-only sweeps over block 0 have started: its block joins S."""
    W, d, mu = _random_spd(1, 96, [3, 5, 8])
    d[3 * 67] = 5.5e-3
    return W, d, mu


def folds():
    """One pressed contact in each of the first 16 blocks of 32 (544
    contacts): S holds 16 blocks; contact 515 goes negative in sweep 3, and a
    17th block cannot join: the deferred changes are folded into every row."""
    W, d, mu = _random_spd(4, 544, [32 * k + 3 for k in range(16)])
    d[3 * 515] = 3.4753e-3
    return W, d, mu


# name -> (W, delta, mu) and what the S-only sweeps must do: "run" (S-only
# sweeps), "join" (S-only sweeps, contacts that start to change join S),
# "leave" (deferred folds back to full sweeps), "off" (|S| > 16 blocks),
# "fixed" (an exact fixed point before the sweep cap)
CASES = {
    "one_block": (lambda: synth(100, [0, 3, 5, 9, 14, 20], (0.05, 0.1), 7), "run"),
    "three_blocks": (lambda: synth(200, [1, 4, 70, 75, 170, 180], (0.05, 0.1), 7), "run"),
    "small_gaps": (lambda: synth(200, [1, 4, 70, 75, 170, 180], (1e-4, 0.1), 11), "run"),
    "joined_late": (joined_late, "join"),
    "folds": (folds, "leave"),
    "last_block": (lambda: synth(150, [2, 130, 140, 149], (0.02, 0.1), 7), "run"),
    "fixed_point": (lambda: synth(64, [5], (0.05, 0.1), 3), "fixed"),
    "many_blocks": (many_active, "off"),
    "pulled_in": (pulled_in, "run"),
}
