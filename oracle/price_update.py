"""The global price update of Sect. 5.2 (Algorithm 5.3), plain and
sequential, for checking the GPU's update on frozen mid-phase states.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone. It shares no code
with the CUDA path.

State: inside a refine phase at scale eps, with column values
v(x, y) = (n + 1)(C[x][y] - min C) + q(y) (q = -p, the paper's price with
its sign flipped), a partial matching ``holder`` (the row holding each
column, -1 if none) in which every matched row x with column M(x) is
eps-optimal in the version-2 sense of Sect. 5.1,
v(x, M(x)) <= min_y v(x, y) + eps, and the free rows ``free``.

Algorithm 5.3 labels every node with its distance, in units of eps, to the
nearest node with negative excess (a free column) over the residual graph,
scanning nodes bucket by bucket as Dial's implementation of Dijkstra's
method does: a node popped from bucket i gets label i, and an unscanned node
reached from it over an arc of length l moves to bucket i + l if that is
lower. It stops once every node with positive excess (every free row) is
scanned; every node not scanned gets label last + 1. Then every price falls
by eps times the label.

Readings (the paper's listing writes the new bucket as floor(c_p / eps) + 1
with no "+ i", and leaves the row prices implicit):
* the label of a node reached from bucket i over an arc of length l is
  i + l (the text defines a label as the distance from bucket 0);
* a matched row's price is fixed by its own arc, so the reduced cost of an
  arc x -> y is c_p(x, y) = v(x, y) - v(x, M(x)) + eps and that of the
  reverse arc M(x) -> x is -eps; the arc lengths floor(c_p / eps) on X -> Y
  arcs and floor(c_p / eps) + 1 = 0 on Y -> X arcs are then all >= 0, and
  subtracting eps * label keeps every matched row eps-optimal; a free row's
  arcs are measured from its own best value;
* the bucket that holds the last free row is finished before the loop
  stops (stopping inside it gives nodes of that bucket the label last + 1,
  which can break eps-optimality).
"""

from __future__ import annotations

import random

INF = 1 << 62


def mid_phase_state(C, alpha, rng: random.Random):
    """The paper's sequential cost scaling (Alg. 5.0's eps loop, Alg. 5.2's
    initialisation, Alg. 5.4's push/relabel as a double push, the free row
    drawn at random) stopped after a random number of bids inside a random
    phase. Returns (scaled costs cs, q, holder, free rows, eps), or None if
    the chosen phase ended first."""
    n = len(C)
    cmin = min(int(v) for row in C for v in row)
    cmax = max(int(v) for row in C for v in row)
    Ct = (n + 1) * (cmax - cmin)
    cs = [[(int(C[x][y]) - cmin) * (n + 1) for y in range(n)] for x in range(n)]
    sched, e = [], Ct
    while True:
        e = max(1, e // alpha)
        sched.append(e)
        if e == 1:
            break
    stop_phase = rng.randrange(len(sched))
    q = [0] * n
    for ph, e in enumerate(sched):
        m = min(q)
        q = [v - m for v in q]
        holder = [-1] * n
        free = list(range(n))
        stop_after = rng.randrange(1, 4 * n) if ph == stop_phase else None
        bids = 0
        while free:
            if stop_after is not None and bids >= stop_after:
                return cs, q, holder, free, e
            x = free.pop(rng.randrange(len(free)))
            b1 = b2 = w = None
            for y in range(n):
                v = cs[x][y] + q[y]
                if b1 is None or v < b1:
                    b2, b1, w = b1, v, y
                elif b2 is None or v < b2:
                    b2 = v
            if b2 is None:
                b2 = b1
            q[w] += (b2 - b1) + e
            if holder[w] >= 0:
                free.append(holder[w])
            holder[w] = x
            bids += 1
    return None


def eps_optimal(cs, q, holder, e) -> bool:
    """Every matched row is eps-optimal (version 2, Sect. 5.1)."""
    n = len(q)
    for w in range(n):
        x = holder[w]
        if x >= 0 and any(cs[x][w] + q[w] > cs[x][y] + q[y] + e for y in range(n)):
            return False
    return True


def arc_length(cs, q, holder, e):
    """(row -> its column, length(x, y) of the arc x -> y in units of eps)."""
    n = len(q)
    row_col = {holder[w]: w for w in range(n) if holder[w] >= 0}

    def length(x, y):
        if x in row_col:
            w = row_col[x]
            return (cs[x][y] + q[y] + e - (cs[x][w] + q[w])) // e
        best = min(cs[x][z] + q[z] for z in range(n))
        return (cs[x][y] + q[y] - best) // e

    return row_col, length


def dial_labels(cs, q, holder, free, e, finish_bucket=True):
    """Algorithm 5.3 by buckets: the label of every column (matched columns
    carry their row's label over the zero-length reverse arc)."""
    n = len(q)
    row_col, length = arc_length(cs, q, holder, e)
    lab = {("col", y): 0 for y in range(n) if holder[y] < 0}
    buckets = {}
    for node in lab:
        buckets.setdefault(0, []).append(node)
    scanned, waiting = set(), set(free)
    last = i = None
    while buckets:
        i = min(buckets)
        if last is not None and i > last:
            break
        node = buckets[i].pop()
        if not buckets[i]:
            del buckets[i]
        if node in scanned or lab[node] != i:
            continue
        scanned.add(node)
        if node[0] == "row":
            waiting.discard(node[1])
            if not waiting:
                last = i
                if not finish_bucket:
                    break
            continue
        y = node[1]
        for x in range(n):          # the residual arcs entering column y
            if row_col.get(x) == y:
                continue
            target = ("col", row_col[x]) if x in row_col else ("row", x)
            d = i + length(x, y)
            if target not in scanned and d < lab.get(target, INF):
                lab[target] = d
                buckets.setdefault(d, []).append(target)
    K = (last if last is not None else i) + 1
    return [lab[("col", y)] if ("col", y) in scanned else K for y in range(n)]


def apply(q, labels, e):
    """New q after the update: every price falls by eps * label."""
    return [a + e * b for a, b in zip(q, labels)]
