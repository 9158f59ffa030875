"""The bound behind the sparse solver's infeasibility test, checked on the CPU.

Before its cost phases, the sparse solver runs one refine phase at eps = 1
with every arc cost taken as 0, from zero prices, and reports that no
perfect matching exists as soon as a bid would lower a column price by more
than 4n + 4. The reading behind that threshold (the path argument of cost
scaling that Lemma 5.6 rests on, Sect. 5): when a perfect matching exists it
is 0-optimal on zero costs, so no price ever drops by more than
(eps + 0)(2n - 1) = 2n - 1; when none exists, the rows of a Hall-violating
set outbid one another for ever and the prices fall without bound.

Here that phase is restated as plain sequential double pushes (best and
second best over the row's own arcs, ties to the lowest column, a row with
one arc bidding as on a tie, parallel arcs kept), with the free row to bid
next drawn at random so that many schedules are tried. Whether a graph has
a perfect matching is the oracle's call (successive shortest paths). Nothing
here touches a GPU or shares code with the CUDA path."""

import random

import numpy as np

import oracle


def _zero_cost_phase(n, rows, rng, limit=10**6):
    """Returns ("ok" | "infeasible", the largest price drop seen)."""
    q = [0] * n           # q = -p: the drop of each column's price
    holder = [-1] * n
    free = list(range(n))
    qmax = steps = 0
    while free:
        steps += 1
        assert steps <= limit, "the phase neither ended nor passed the threshold"
        x = free.pop(rng.randrange(len(free)))
        b1 = b2 = w = None
        for y in rows[x]:
            v = q[y]          # zero costs: the value is the price drop itself
            if b1 is None or v < b1 or (v == b1 and y < w):
                b2, b1, w = b1, v, y
            elif b2 is None or v < b2:
                b2 = v
        if b2 is None:        # a single arc: bid as on a tie
            b2 = b1
        nq = b2 + 1           # q(w) + (b2 - b1) + eps with b1 = q(w)
        if nq > 4 * n + 4:
            return "infeasible", qmax
        q[w] = nq
        qmax = max(qmax, nq)
        if holder[w] >= 0:
            free.append(holder[w])
        holder[w] = x
    return "ok", qmax


def _random_graph(rng, n, degree):
    arcs = [(x, rng.randrange(n)) for x in range(n) for _ in range(rng.randint(1, degree))]
    covered = {y for _, y in arcs}
    arcs += [(rng.randrange(n), y) for y in range(n) if y not in covered]   # no empty column
    rows = [[] for _ in range(n)]
    for x, y in arcs:
        rows[x].append(y)
    return rows


def _feasible(n, rows):
    row_ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    cols = np.array([y for r in rows for y in r], dtype=np.int32)
    try:
        oracle.sparse_ssp(row_ptr, cols, np.zeros_like(cols))
        return True
    except oracle.Infeasible:
        return False


def test_threshold_separates_feasible_from_infeasible_graphs():
    rng = random.Random(1)
    worst = {}
    counts = {True: 0, False: 0}
    for trial in range(1500):
        n = rng.randint(1, 10)
        rows = _random_graph(rng, n, rng.randint(1, 4))
        feasible = _feasible(n, rows)
        counts[feasible] += 1
        for schedule in range(4):
            result, qmax = _zero_cost_phase(n, rows, random.Random(1000 * trial + schedule))
            if feasible:
                assert result == "ok", (n, rows, qmax)
                assert qmax <= 2 * n - 1, (n, rows, qmax)
                worst[n] = max(worst.get(n, 0), qmax)
            else:
                assert result == "infeasible", (n, rows)
    assert counts[True] > 300 and counts[False] > 300
    # the bound 2n - 1 is reached: the margin up to 4n + 4 is not slack
    assert any(worst.get(n) == 2 * n - 1 for n in (2, 3, 4))


def test_a_chain_stays_within_the_bound():
    """Row i has arcs to columns i and i + 1 (the last row only to its own
    column): the perfect matching is unique and every other choice is
    displaced along the chain, yet no price drops by more than 2n - 1."""
    for n in range(1, 9):
        rows = [[i, i + 1] if i + 1 < n else [i] for i in range(n)]
        assert _feasible(n, rows)
        for s in range(8):
            result, qmax = _zero_cost_phase(n, rows, random.Random(s))
            assert result == "ok" and qmax <= 2 * n - 1


def test_hall_violations_pass_the_threshold():
    """Two rows whose only arcs go to one column, beside an otherwise
    complete graph: no row or column is empty, yet no perfect matching
    exists, and the two rows outbid each other past 4n + 4."""
    for n in range(3, 9):
        rows = [[0], [0]] + [list(range(n)) for _ in range(n - 2)]
        assert all(any(y in r for r in rows) for y in range(n))
        assert not _feasible(n, rows)
        for s in range(4):
            assert _zero_cost_phase(n, rows, random.Random(s))[0] == "infeasible"
