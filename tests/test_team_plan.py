"""The batched eigensolver's team split (sky_tri_team_plan, host code of the
library; no GPU): for a batch of more than 8 problems the cooperative
Householder reduction's blocks split into teams, each reducing its own
problems between its own barriers.  Invariants checked on the 64-box batch
of the twist-averaged form and on random batches: every problem belongs to
one team; the teams' blocks are contiguous, disjoint and within the grid; a
team of several blocks serves one problem; the problems sharing a one-block
team fit its shared memory together; larger single problems never get fewer
blocks than smaller ones; the split uses the grid.
"""
import random

import pytest

from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

SMEM_DOUBLE2 = 200 * 1024 // 16 - 64     # the reduction's shared-memory budget, double2


def vec(n):
    return 3 * n + (n + 1) // 2 + 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    try:
        B.lib()
    except OSError as e:
        pytest.skip(f"library not built: {e}")


def check(n, blocks):
    got = B.sky_tri_team_plan(n, blocks)
    assert got is not None
    team, tb = got
    nteam = len(tb)
    assert sorted(set(team)) == list(range(nteam))            # every team used, every problem placed
    nxt = 0
    for first, count in tb:                                  # contiguous, disjoint, in the grid
        assert first == nxt and count >= 1
        nxt += count
    assert nxt <= blocks
    members = [[b for b in range(len(n)) if team[b] == t] for t in range(nteam)]
    for t, (first, count) in enumerate(tb):
        if count > 1:
            assert len(members[t]) == 1
        else:
            assert sum(vec(n[b]) for b in members[t]) <= SMEM_DOUBLE2
    single = sorted((n[m[0]], tb[t][1]) for t, m in enumerate(members) if len(m) == 1)
    for (n1, c1), (n2, c2) in zip(single, single[1:]):
        assert n1 > n2 or c1 <= c2 or n1 == n2
    return team, tb, members


def test_the_64_box_batch():
    n = []
    for w in IN.batched_workloads(64):
        n += [w.N, w.Z]
    team, tb, members = check(n, 152)
    assert sum(c for _, c in tb) == 152                      # the spare blocks are handed out
    big = [t for t, m in enumerate(members) if any(n[b] == 290 for b in m)]
    assert all(tb[t][1] >= 5 and len(members[t]) == 1 for t in big)   # one team per 290-state problem
    assert len(tb) < len(n)                                  # small problems share blocks


@pytest.mark.parametrize("seed", range(8))
def test_random_batches(seed):
    rng = random.Random(seed)
    np_ = rng.randint(9, 128)
    n = [rng.choice([rng.randint(1, 40), rng.randint(40, 400), rng.randint(400, 1500)])
         for _ in range(np_)]
    check(n, rng.choice([16, 76, 152, 304]))


def test_degenerate_and_invalid_batches():
    team, tb, _ = check([300], 152)                          # one problem: one team
    assert len(tb) == 1 and team == [0]
    team, tb, _ = check([1] * 128, 152)                      # 128 one-state problems
    assert sum(c for _, c in tb) <= 152
    assert B.sky_tri_team_plan([], 152) is None
    assert B.sky_tri_team_plan([10, 0, 5], 152) is None
    assert B.sky_tri_team_plan([10] * 129, 152) is None
    assert B.sky_tri_team_plan([10, 20], 0) is None
    assert B.sky_tri_team_plan([5000, 10], 152) is None      # work vectors beyond shared memory
