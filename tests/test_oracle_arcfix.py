"""Pins of the oracle's arc fixing (Sect. 5.2): after every phase but the
last, arcs whose reduced cost exceeds 2 n eps are deleted for good.

The paper states the rule without its argument; the one the oracle relies
on is that no optimal assignment uses a deleted arc (an alternating cycle
through such an arc would have negative cost in the optimum's residual
graph). These tests check exactly that by enumeration: on small matrices,
heavy ties included, every optimal permutation avoids every deleted arc,
and the cost with fixing equals the enumerated optimum. Larger instances
must still give the Hungarian optimum while most arcs are deleted, so the
pins are not vacuous.
"""

import itertools

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth


def _optimal_perms(C):
    n = C.shape[0]
    best, perms = None, []
    for p in itertools.permutations(range(n)):
        s = sum(int(C[x, p[x]]) for x in range(n))
        if best is None or s < best:
            best, perms = s, [p]
        elif s == best:
            perms.append(p)
    return best, perms


def test_no_optimal_assignment_loses_an_arc():
    rng = np.random.default_rng(41)
    deleted_total, arcs_total, with_deletions = 0, 0, 0
    for t in range(300):
        n = int(rng.integers(2, 8))
        lo, hi = [(0, 4), (0, 30), (-50, 50), (0, 1000)][t % 4]
        C = rng.integers(lo, hi, size=(n, n)).astype(np.int32)
        alpha = [2, 3, 4, 10][(t // 4) % 4]
        best, perms = _optimal_perms(C)
        cost, match, prices, fixed, st = oracle.cost_scaling_arcfix(C, alpha=alpha)
        assert cost == best, (t, n, alpha)
        assert sum(int(C[x, match[x]]) for x in range(n)) == cost
        assert not fixed[np.arange(n), match].any()
        for p in perms:
            assert not fixed[np.arange(n), np.array(p)].any(), (t, p)
        assert st["deleted"] == int(fixed.sum())
        deleted_total += st["deleted"]
        arcs_total += n * n
        with_deletions += st["deleted"] > 0
    # the rule does delete arcs on most of these instances
    assert with_deletions > 150 and deleted_total > arcs_total // 4


@pytest.mark.parametrize("make", [lambda s: synth.uniform_costs(200, 0, 1000, s),
                                  lambda s: synth.uniform_costs(150, 0, (1 << 20) - 1, s),
                                  lambda s: synth.geometric_costs(180, s)],
                         ids=["uniform-n200-c1000", "uniform-n150-c2^20", "geometric-n180"])
def test_arc_fixing_keeps_the_hungarian_optimum(make):
    for seed in range(3):
        C = make(seed)
        n = C.shape[0]
        ref, hm, u, v = oracle.hungarian(C)
        for alpha in (4, 10, 64):
            cost, match, prices, fixed, st = oracle.cost_scaling_arcfix(C, alpha=alpha)
            assert cost == ref
            assert oracle.check_matching(C, match, cost) == 0
            # the Hungarian optimum avoids every deleted arc as well
            assert not fixed[np.arange(n), hm].any()
            plain = oracle.cost_scaling(C, alpha=alpha)
            assert plain[0] == ref
        # at the paper's alpha most arcs are gone before the last phase
        cost, match, prices, fixed, st = oracle.cost_scaling_arcfix(C, alpha=10)
        assert st["deleted"] > n * n // 2


def test_arc_fixing_with_start_prices_and_eps0():
    # any start prices and eps0 give the same optimum (Alg. 5.2's
    # initialisation makes them eps-optimal); fixing must not change that
    rng = np.random.default_rng(3)
    for seed in range(20):
        C = synth.uniform_costs(40, 0, 500, 100 + seed)
        ref = oracle.hungarian(C)[0]
        p0 = rng.integers(-41 * 500, 1, size=40).astype(np.int64)
        for eps0 in (0, 7, 41 * 50):
            assert oracle.cost_scaling_arcfix(C, alpha=5, eps0=eps0, init_prices=p0)[0] == ref


def test_single_arc_rows_and_degenerate_sizes():
    assert oracle.cost_scaling_arcfix(np.array([[7]], np.int32))[0] == 7
    assert oracle.cost_scaling_arcfix(np.zeros((0, 0), np.int32))[0] == 0
    # one cheap column per row, everything else far away: after the first
    # phases each row keeps a single arc, whose bids lower the price by eps
    n = 12
    C = np.full((n, n), 10**6, np.int32)
    perm = np.random.default_rng(0).permutation(n)
    C[np.arange(n), perm] = np.arange(n, dtype=np.int32)
    cost, match, prices, fixed, st = oracle.cost_scaling_arcfix(C, alpha=10)
    assert cost == int(np.arange(n).sum()) and list(match) == list(perm)
    assert (fixed.sum(axis=1) == n - 1).sum() >= n // 2   # rows bidding on a single arc
