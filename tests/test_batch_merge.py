"""The merge rule of batched steps (icr_batch_merge_plan), on the host.

A batch merges the launch sequences of its scenes into one common
supersequence: every merged launch covers scenes whose launch of that key it
takes over, each scene's launches are covered in their own order, one per
merged launch.  For two sequences the merge is a shortest common
supersequence (checked against brute force); when every scene's sequence is a
subsequence of one common step-shaped sequence (the scenes' steps differ only
by levels and optional kernels), the merged sequence is no longer than it."""
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def icr_mod():
    from paper_2306_06946_gb300 import build, icr
    build.build()
    return icr


def check_valid(seqs, plan):
    pos = [0] * len(seqs)
    for key, cover in plan:
        assert cover == sorted(set(cover)) and cover
        for s in cover:
            assert pos[s] < len(seqs[s]) and seqs[s][pos[s]] == key
            pos[s] += 1
    assert pos == [len(q) for q in seqs]


def test_identical_sequences_merge_into_one(icr_mod):
    base = [0, 1, 2, 1, 2, 3, 4, 5]
    plan = icr_mod.batch_merge_plan([base] * 5)
    check_valid([base] * 5, plan)
    assert len(plan) == len(base) and all(c == [0, 1, 2, 3, 4] for _, c in plan)


def step_like(levels, tc, newton, prox_split):
    """A step-shaped key sequence: copies and reach kernels, per level an
    assembly and a product (plus packing and a tensor-core product where tc[l]),
    the contraction, per Newton iteration five kernels (one more where the
    proximity update is split), the backward sweep per level."""
    q = [10, 11, 12, 13]
    for l in range(levels):
        q += [20, 21] + ([22, 23] if tc[l] else [])
    q += [30, 31, 32]
    for _ in range(newton):
        q += [40, 41, 42, 43] + ([44, 45] if prox_split else [46])
    return q + [50] + [51] * levels + [52]


def test_subsequences_of_a_common_step(icr_mod):
    """Steps with fewer levels, fewer tensor-core levels and either proximity
    update are all subsequences of the step with every level and kernel; they
    merge into at most its length (and never fewer launches than the longest)."""
    rng = np.random.default_rng(3)
    top = 9
    for trial in range(20):
        seqs = []
        for _ in range(int(rng.integers(2, 12))):
            lv = int(rng.integers(1, top + 1))
            seqs.append(step_like(lv, rng.random(lv) < 0.4, 5, False))
        plan = icr_mod.batch_merge_plan(seqs)
        check_valid(seqs, plan)
        assert max(len(q) for q in seqs) <= len(plan) <= len(step_like(top, [True] * top, 5, False))


def test_mixed_proximity_paths_cover_in_order(icr_mod):
    seqs = [step_like(4, [False] * 4, 3, False), step_like(6, [True] * 6, 3, True), step_like(2, [True] * 2, 3, False)]
    plan = icr_mod.batch_merge_plan(seqs)
    check_valid(seqs, plan)
    assert len(plan) < sum(len(q) for q in seqs) / 2


def test_two_sequences_merge_into_a_shortest_common_supersequence(icr_mod):
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.integers(0, 3, size=int(rng.integers(0, 7))).tolist()
        b = rng.integers(0, 3, size=int(rng.integers(0, 7))).tolist()
        plan = icr_mod.batch_merge_plan([a, b])
        check_valid([a, b], plan)
        # brute force: the shortest sequence having both as subsequences
        best = None
        for n in range(max(len(a), len(b)), len(a) + len(b) + 1):
            for cand in itertools.product(range(3), repeat=n):
                if is_subseq(a, cand) and is_subseq(b, cand):
                    best = n
                    break
            if best is not None:
                break
        assert len(plan) == best


def is_subseq(q, seq):
    it = iter(seq)
    return all(any(x == y for y in it) for x in q)


def test_extra_kernels_of_one_scene_join_the_common_launches(icr_mod):
    # scene 0 has an extra kernel (7) before the common tail
    seqs = [[1, 7, 2, 3], [1, 2, 3]]
    plan = icr_mod.batch_merge_plan(seqs)
    check_valid(seqs, plan)
    assert plan == [(1, [0, 1]), (7, [0]), (2, [0, 1]), (3, [0, 1])]


def test_empty_and_single_sequences(icr_mod):
    assert icr_mod.batch_merge_plan([[]]) == []
    plan = icr_mod.batch_merge_plan([[4, 4, 5], []])
    check_valid([[4, 4, 5], []], plan)
    assert [k for k, _ in plan] == [4, 4, 5]


def test_invalid_arguments(icr_mod):
    with pytest.raises(icr_mod.IcrError):
        icr_mod.batch_merge_plan([])
    with pytest.raises(icr_mod.IcrError):
        icr_mod.batch_merge_plan([[1, -2]])
