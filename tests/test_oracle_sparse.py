"""Pins for the sparse-graph oracle (no GPU).

The oracle's sparse solver (successive shortest paths with integer duals) is
checked against facts that do not come from itself: hand-worked fixtures
under ``tests/golden/sparse/`` (a forced matching, a greedy trap, a Hall
violation), a pure-Python enumeration, the dense Hungarian method on
complete graphs, scipy's ``min_weight_full_bipartite_matching`` and the LP
duality certificate; its checkers must reject planted bad claims.
"""

import glob
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sparse")


def load_sparse_fixture(path):
    lines = [l for l in open(path) if l.strip() and not l.startswith("#")]
    c = lines[0].split()[1]
    cost = None if c == "infeasible" else int(c)
    m = lines[1].split()[1:]
    match = None if m == ["any"] else np.array([int(t) for t in m], dtype=np.int32)
    n = int(lines[2].split()[1])
    assert lines[3].strip() == "arcs"
    arcs = [tuple(int(t) for t in l.split()) for l in lines[4:]]
    return to_csr(n, arcs), cost, match


def to_csr(n, arcs):
    """CSR arrays of a list of (row, column, cost) arcs (row order kept)."""
    arcs = sorted(arcs, key=lambda a: a[0])
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for r, _, _ in arcs:
        row_ptr[r + 1] += 1
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    cols = np.array([a[1] for a in arcs], dtype=np.int32)
    costs = np.array([a[2] for a in arcs], dtype=np.int32)
    return row_ptr, cols, costs


def python_enumeration(n, arcs):
    """Min cost over permutations made of arcs (cheapest parallel arc), or None."""
    w = {}
    for r, c, x in arcs:
        w[(r, c)] = min(x, w.get((r, c), x))
    best = None
    for p in itertools.permutations(range(n)):
        if all((x, p[x]) in w for x in range(n)):
            s = sum(w[(x, p[x])] for x in range(n))
            best = s if best is None or s < best else best
    return best


def random_sparse(rng, n, density, lo, hi, dup=False):
    arcs = [(x, y, int(rng.integers(lo, hi + 1))) for x in range(n) for y in range(n) if rng.random() < density]
    if dup and arcs:
        arcs += [(a[0], a[1], int(rng.integers(lo, hi + 1))) for a in arcs[: max(1, len(arcs) // 4)]]
    return arcs


FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


@pytest.mark.parametrize("path", FIXTURES, ids=os.path.basename)
def test_sparse_fixtures(path):
    (rp, cols, costs), cost, match = load_sparse_fixture(path)
    for solve in (oracle.sparse_brute_force, lambda *a: oracle.sparse_ssp(*a)[:2]):
        if cost is None:
            with pytest.raises(oracle.Infeasible):
                solve(rp, cols, costs)
            continue
        got_cost, got_match = solve(rp, cols, costs)
        assert got_cost == cost
        assert oracle.sparse_check_matching(rp, cols, costs, got_match, cost) == 0
        if match is not None:
            np.testing.assert_array_equal(got_match, match)


def test_sparse_brute_force_matches_python_enumeration():
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(1, 7))
        arcs = random_sparse(rng, n, float(rng.uniform(0.2, 0.9)), -20, 20, dup=trial % 3 == 0)
        want = python_enumeration(n, arcs)
        rp, cols, costs = to_csr(n, arcs)
        if want is None:
            with pytest.raises(oracle.Infeasible):
                oracle.sparse_brute_force(rp, cols, costs)
        else:
            assert oracle.sparse_brute_force(rp, cols, costs)[0] == want


def test_sparse_ssp_matches_brute_force_with_ties_and_duplicates():
    rng = np.random.default_rng(12)
    feasible = infeasible = 0
    for trial in range(600):
        n = int(rng.integers(1, 9))
        lo, hi = [(0, 2), (-50, 50), (0, 1000), (-(1 << 31), (1 << 31) - 1)][trial % 4]
        arcs = random_sparse(rng, n, float(rng.uniform(0.15, 1.0)), lo, hi, dup=trial % 5 == 0)
        rp, cols, costs = to_csr(n, arcs)
        try:
            want, _ = oracle.sparse_brute_force(rp, cols, costs)
        except oracle.Infeasible:
            infeasible += 1
            with pytest.raises(oracle.Infeasible):
                oracle.sparse_ssp(rp, cols, costs)
            continue
        feasible += 1
        cost, match, u, v = oracle.sparse_ssp(rp, cols, costs)
        assert cost == want
        assert oracle.sparse_check_matching(rp, cols, costs, match, cost) == 0
        assert oracle.sparse_check_duals(rp, cols, costs, match, u, v) == 0
        assert int(u.sum() + v.sum()) == cost
    assert feasible > 100 and infeasible > 100


@pytest.mark.parametrize("n", [1, 2, 17, 64, 150])
def test_sparse_ssp_on_complete_graph_equals_dense_hungarian(n):
    C = synth.uniform_costs(n, -100, 1000, n)
    rp = (np.arange(n + 1) * n).astype(np.int32)
    cols = np.tile(np.arange(n, dtype=np.int32), n)
    cost, match, u, v = oracle.sparse_ssp(rp, cols, C.ravel())
    assert cost == oracle.hungarian(C)[0]
    assert oracle.check_matching(C, match, cost) == 0


@pytest.mark.parametrize("kind", ["uniform", "geometric", "infeasible"])
def test_sparse_ssp_matches_scipy(kind):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    if kind == "uniform":
        rp, cols, costs = synth.sparse_uniform(300, 6, 3)
    elif kind == "geometric":
        rp, cols, costs = synth.sparse_geometric(400, 4)
    else:   # row 0's arcs removed: column coverage fails for a planted graph of degree 0
        rp, cols, costs = synth.sparse_uniform(120, 0, 5)
        keep = np.ones(cols.size, dtype=bool)
        keep[rp[0]:rp[1]] = False
        cols, costs = cols[keep], costs[keep]
        rp = rp - np.minimum(rp, rp[1] - rp[0])
        rp[0] = 0
    n = rp.size - 1
    # scipy treats absent entries as missing arcs: shift costs to >= 1 so no
    # arc is stored as an explicit zero (the optimum shifts by n)
    m = sp.csr_matrix(((costs.astype(np.int64) + 1).astype(np.float64), cols, rp), shape=(n, n))
    if kind == "infeasible":
        with pytest.raises(ValueError):
            csgraph.min_weight_full_bipartite_matching(m)
        with pytest.raises(oracle.Infeasible):
            oracle.sparse_ssp(rp, cols, costs)
        return
    r, c = csgraph.min_weight_full_bipartite_matching(m)
    want = int(round(m[r, c].sum())) - n
    cost, match, u, v = oracle.sparse_ssp(rp, cols, costs)
    assert cost == want
    assert oracle.sparse_check_duals(rp, cols, costs, match, u, v) == 0


def test_sparse_checkers_reject_bad_claims():
    rp, cols, costs = to_csr(3, [(0, 0, 1), (0, 1, 2), (1, 0, 2), (1, 2, 9), (2, 1, 3), (2, 2, 4)])
    cost, match, u, v = oracle.sparse_ssp(rp, cols, costs)
    assert cost == 8
    assert oracle.sparse_check_matching(rp, cols, costs, match, cost) == 0
    assert oracle.sparse_check_matching(rp, cols, costs, match, cost + 1) != 0
    assert oracle.sparse_check_matching(rp, cols, costs, np.array([0, 0, 2]), cost) != 0   # not a permutation
    assert oracle.sparse_check_matching(rp, cols, costs, np.array([2, 0, 1]), 13) != 0     # (0, 2) is no arc
    bad_u = u.copy()
    bad_u[0] += 1
    assert oracle.sparse_check_duals(rp, cols, costs, match, bad_u, v) != 0
    # eps-CS at eps = 1 on costs scaled by n + 1: prices from the duals hold,
    # a matching that is not optimal has no such prices (here: the greedy one)
    p = (len(match) + 1) * v
    assert oracle.sparse_check_eps_cs(rp, cols, costs, match, p, 1) == 0
    assert oracle.sparse_check_eps_cs(rp, cols, costs, np.array([0, 2, 1]), p, 1) != 0


def test_sparse_generators_plant_a_perfect_matching():
    for rp, cols, costs in (synth.sparse_uniform(500, 3, 9), synth.sparse_geometric(700, 9)):
        n = rp.size - 1
        assert rp[0] == 0 and rp[-1] == cols.size == costs.size
        assert np.all(np.diff(rp) >= 1)
        for x in range(n):   # rows are sorted and duplicate free
            seg = cols[rp[x]:rp[x + 1]]
            assert np.all(np.diff(seg) > 0)
        oracle.sparse_ssp(rp, cols, costs)   # feasible
