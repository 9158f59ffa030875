"""The global price update (Sect. 5.2, Algorithm 5.3): the oracle's Dial
bucket restatement (``oracle/price_update.py``) pinned, and the GPU's form
restated beside it, to pin the readings the GPU kernel rests on. Nothing
here touches a GPU or shares code with the CUDA path.

State: inside a refine phase at scale eps, with column values
v(x, y) = (n + 1)(C[x][y] - min C) + q(y) (q = -p), a partial matching in
which every matched row x (column M(x)) is eps-optimal in the version-2
sense of Sect. 5.1, v(x, M(x)) <= min_y v(x, y) + eps, and some free rows.

Labels are distances, in units of eps, to the nearest free column over the
residual graph. With the row price of a matched row fixed by its arc, the
reduced cost c_p(x, y) of an arc x -> y is v(x, y) - v(x, M(x)) + eps and the
reverse arc M(x) -> x costs -eps, so the lengths floor(c_p / eps) on X -> Y
arcs and floor(c_p / eps) + 1 = 0 on Y -> X arcs are all >= 0. A free row's
arcs are measured from its own best value. Then every column's price falls
by eps * label, labels truncated at one more than the largest label of a
free row.

1. The GPU computes exact labels by Bellman-Ford sweeps and truncates them;
   Algorithm 5.3 scans Dial buckets (the label of a node reached from bucket
   i over an arc of length l is i + l) and gives the unscanned nodes the
   last bucket + 1. The two must agree when the bucket holding the last free
   row is finished, and the update must keep every matched row eps-optimal.
2. Stopping as soon as the last free row is scanned leaves nodes of its
   bucket unscanned; their label (last + 1) then overstates the distance and
   must break eps-optimality on some states.
3. On candidate lists the GPU relaxes only the listed arcs and caps a
   matched row's label by its bound theta (clamped at 0). That must keep
   eps-optimality over every arc, listed or not; without the cap, or with
   a cap that may go negative, it must break on some states.
"""

import random

import numpy as np
import pytest

from oracle.price_update import INF, arc_length as _arc_length, dial_labels as _labels_buckets, \
    eps_optimal as _eps_optimal, mid_phase_state as _mid_phase_state


def _labels_bellman_ford(cs, q, holder, free, e):
    n = len(q)
    row_col, length = _arc_length(cs, q, holder, e)
    lab = [0 if holder[y] < 0 else INF for y in range(n)]
    for _ in range(2 * n + 2):
        changed = False
        for x, w in row_col.items():
            b = min((lab[y] + length(x, y) for y in range(n) if y != w), default=INF)
            if b < lab[w]:
                lab[w], changed = b, True
        if not changed:
            break
    K = max(min(lab[y] + length(x, y) for y in range(n)) for x in free) + 1
    return [min(v, K) for v in lab]


def _states(count, seed):
    rng = random.Random(seed)
    out = []
    for t in range(count):
        n = rng.randint(2, 9)
        hi = (20, 3, 1000)[t % 3]
        C = np.random.default_rng(seed * 7919 + t).integers(0, hi, size=(n, n))
        st = _mid_phase_state(C, rng.choice([2, 4, 10]), rng)
        if st is not None and st[3]:
            out.append(st)
    return out


def test_update_keeps_eps_optimality_and_matches_the_buckets():
    states = _states(600, 3)
    assert len(states) > 100
    moved = 0
    for cs, q, holder, free, e in states:
        assert _eps_optimal(cs, q, holder, e)
        lab = _labels_bellman_ford(cs, q, holder, free, e)
        assert lab == _labels_buckets(cs, q, holder, free, e)
        q2 = [a + e * b for a, b in zip(q, lab)]
        assert _eps_optimal(cs, q2, holder, e)
        moved += any(lab)
    assert moved > len(states) // 4   # the update moves prices in many states


def test_stopping_inside_the_last_bucket_breaks_eps_optimality():
    broken = 0
    for cs, q, holder, free, e in _states(600, 3):
        lab = _labels_buckets(cs, q, holder, free, e, finish_bucket=False)
        broken += not _eps_optimal(cs, [a + e * b for a, b in zip(q, lab)], holder, e)
    assert broken > 0


def _labels_with_lists(cs, q, holder, free, e, lists, theta, cap_rows=True, clamp=True):
    """The GPU's form on candidate lists: only a row's listed arcs are
    relaxed; every unlisted column y of row x has v(x, y) >= theta[x], so a
    matched row's label is capped at floor((theta + eps - v(x, M(x))) / eps),
    which keeps label(M(x)) <= label(y) + length(x, y) for those columns."""
    n = len(q)
    row_col = {holder[w]: w for w in range(n) if holder[w] >= 0}
    lab = [0 if holder[y] < 0 else INF for y in range(n)]
    cap = {}
    for x, w in row_col.items():
        vr = cs[x][w] + q[w]
        # a bound below v(x, M(x)) - eps allows no drop at all: the cap is 0
        c = (theta[x] + e - vr) // e
        cap[x] = (max(0, c) if clamp else c) if cap_rows else INF
        lab[w] = min(lab[w], cap[x])
    for _ in range(2 * n + 2):
        changed = False
        for x, w in row_col.items():
            vr = cs[x][w] + q[w]
            b = cap[x]
            for y in lists[x]:
                if y != w:
                    b = min(b, lab[y] + (cs[x][y] + q[y] + e - vr) // e)
            if b < lab[w]:
                lab[w], changed = b, True
        if not changed:
            break
    K = 0
    for x in free:   # a lower bound of the row's best value measures its arcs
        vr = min(min(cs[x][y] + q[y] for y in lists[x]), theta[x])
        b = (theta[x] - vr) // e
        for y in lists[x]:
            b = min(b, lab[y] + (cs[x][y] + q[y] - vr) // e)
        K = max(K, b)
    return [min(v, K + 1) for v in lab]


def _random_lists(cs, q, rng):
    """Each row lists some of its best columns at the current prices, plus a
    random extra one; theta is the least unlisted value less a random slack
    (a list built earlier, at lower prices, has a lower bound)."""
    n = len(q)
    lists, theta = [], []
    for x in range(n):
        order = sorted(range(n), key=lambda y: (cs[x][y] + q[y], y))
        k = rng.randint(1, n - 1)
        chosen = set(order[:k])
        if rng.random() < 0.5:
            chosen.add(rng.randrange(n))
        unlisted = [cs[x][y] + q[y] for y in range(n) if y not in chosen]
        t = min(unlisted) if unlisted else INF
        lists.append(sorted(chosen))
        theta.append(t - rng.randint(0, 3 * max(1, t // 8)) if unlisted else INF)
    return lists, theta


def test_update_on_candidate_lists_keeps_eps_optimality_over_every_arc():
    rng = random.Random(11)
    states = _states(600, 5)
    assert len(states) > 100
    for cs, q, holder, free, e in states:
        lists, theta = _random_lists(cs, q, rng)
        lab = _labels_with_lists(cs, q, holder, free, e, lists, theta)
        assert _eps_optimal(cs, [a + e * b for a, b in zip(q, lab)], holder, e)


@pytest.mark.parametrize("mistake", ["no cap", "cap not clamped at 0"])
def test_lists_without_the_theta_cap_break_eps_optimality(mistake):
    """Without the cap, a row's label ignores its unlisted columns; a cap
    that may go negative would raise a matched column's price. Both break
    eps-optimality on some states."""
    rng = random.Random(11)
    broken = 0
    for cs, q, holder, free, e in _states(600, 5):
        lists, theta = _random_lists(cs, q, rng)
        lab = _labels_with_lists(cs, q, holder, free, e, lists, theta, cap_rows=mistake != "no cap",
                                 clamp=mistake != "cap not clamped at 0")
        broken += not _eps_optimal(cs, [a + e * b for a, b in zip(q, lab)], holder, e)
    assert broken > 0
