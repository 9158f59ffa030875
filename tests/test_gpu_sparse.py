"""GPU parity of la_solve_sparse against the CPU oracle (sparse graphs).

Every result is checked element by element against the oracle's successive
shortest paths on the same seeded graph: the exact optimal cost, a matching
made of arcs at that cost, and agreement on infeasibility. At the full
workload size (n = 65536), where the oracle's search is too slow, the
returned prices must certify the returned matching: eps-complementary
slackness at eps = 1 on costs scaled by n + 1 (Sect. 5.1, Lemma 5.6) proves it
optimal at any size.
"""

import glob
import os

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

from test_oracle_sparse import load_sparse_fixture, random_sparse, to_csr

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sparse")


@pytest.fixture(scope="module")
def la():
    import torch
    from paper_1110_6231_gb300 import build
    build.build()
    import paper_1110_6231_gb300 as la
    assert torch.cuda.is_available()
    return la


def gpu_solve(la, rp, cols, costs, **kw):
    import torch
    t = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda() for a in (rp, cols, costs)]
    return la.solve_sparse(*t, check=False, **kw)


def expect_same(la, rp, cols, costs, **kw):
    sol = gpu_solve(la, rp, cols, costs, want_prices=True, **kw)
    try:
        want = oracle.sparse_ssp(rp, cols, costs)[0]
    except oracle.Infeasible:
        assert sol.stats["status"] == la.LA_ERR_INFEASIBLE, sol.stats["status"]
        return None
    assert sol.stats["status"] == la.LA_OK, la.la_status_string(sol.stats["status"])
    assert sol.cost == want
    match = sol.match.cpu().numpy()
    assert oracle.sparse_check_matching(rp, cols, costs, match, want) == 0
    assert oracle.sparse_check_eps_cs(rp, cols, costs, match, sol.prices.cpu().numpy(), 1) == 0
    return sol


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))), ids=os.path.basename)
def test_sparse_fixtures(la, path):
    (rp, cols, costs), cost, match = load_sparse_fixture(path)
    sol = expect_same(la, rp, cols, costs)
    if cost is None:
        assert sol is None
    else:
        assert sol.cost == cost
        if match is not None:
            np.testing.assert_array_equal(sol.match.cpu().numpy(), match)


def test_small_random_graphs_with_ties_duplicates_and_infeasible_ones(la):
    rng = np.random.default_rng(21)
    feasible = infeasible = 0
    for trial in range(160):
        n = int(rng.integers(1, 41))
        lo, hi = [(0, 1), (-50, 50), (0, 10_000), (-(1 << 20), 1 << 20)][trial % 4]
        arcs = random_sparse(rng, n, float(rng.uniform(0.05, 0.6)), lo, hi, dup=trial % 3 == 0)
        rp, cols, costs = to_csr(n, arcs)
        if expect_same(la, rp, cols, costs) is None:
            infeasible += 1
        else:
            feasible += 1
    assert feasible > 30 and infeasible > 30


def test_hall_violation_found_by_the_zero_cost_phase(la):
    """Every row and column has arcs, but 12 rows reach only 11 columns: the
    degree checks pass and only the feasibility phase can tell."""
    rp, cols, costs = synth.sparse_uniform(600, 6, 8)
    n = rp.size - 1
    rows = [list(zip(cols[rp[x]:rp[x + 1]], costs[rp[x]:rp[x + 1]])) for x in range(n)]
    for x in range(12):
        rows[x] = [(int(y), 7 + x) for y in range(11)]
    arcs = [(x, int(y), int(c)) for x in range(n) for y, c in rows[x]]
    rp2, cols2, costs2 = to_csr(n, arcs)
    assert np.unique(cols2).size == n
    with pytest.raises(oracle.Infeasible):
        oracle.sparse_ssp(rp2, cols2, costs2)
    sol = gpu_solve(la, rp2, cols2, costs2)
    assert sol.stats["status"] == la.LA_ERR_INFEASIBLE


@pytest.mark.parametrize("kind,n", [("uniform", 3000), ("geometric", 4000), ("uniform-d1", 2500)])
def test_medium_graphs_match_oracle(la, kind, n):
    if kind == "uniform":
        g = synth.sparse_uniform(n, 8, 31)
    elif kind == "geometric":
        g = synth.sparse_geometric(n, 32)
    else:   # the planted matching plus one random arc per row: many rows of degree 1 or 2
        g = synth.sparse_uniform(n, 1, 33)
    expect_same(la, *g)


@pytest.mark.parametrize("name", sorted(synth.SPARSE_WORKLOADS))
def test_full_size_workloads_certified(la, name):
    rp, cols, costs = synth.sparse_instance(name, 0)
    sol = gpu_solve(la, rp, cols, costs, want_prices=True)
    assert sol.stats["status"] == la.LA_OK
    match = sol.match.cpu().numpy()
    assert oracle.sparse_check_matching(rp, cols, costs, match, sol.cost) == 0
    assert oracle.sparse_check_eps_cs(rp, cols, costs, match, sol.prices.cpu().numpy(), 1) == 0


def test_complete_graph_equals_dense_solver(la):
    import torch
    n = 300
    C = synth.uniform_costs(n, 0, 1000, 2)
    rp = (np.arange(n + 1) * n).astype(np.int32)
    cols = np.tile(np.arange(n, dtype=np.int32), n)
    sol = gpu_solve(la, rp, cols, C.ravel())
    assert sol.cost == la.solve(torch.from_numpy(C).cuda()).cost == oracle.hungarian(C)[0]


def test_malformed_csr_rejected_on_device(la):
    rp, cols, costs = to_csr(3, [(0, 0, 1), (1, 1, 1), (2, 2, 1)])
    for bad_rp, bad_cols in (([1, 1, 2, 3], cols), ([0, 2, 1, 3], cols), ([0, 1, 2, 2], cols),
                             (rp, np.array([0, 3, 2], np.int32)), (rp, np.array([0, -1, 2], np.int32))):
        sol = gpu_solve(la, np.array(bad_rp, np.int32), bad_cols, costs)
        assert sol.stats["status"] == la.LA_ERR_INVALID


def test_empty_and_single(la):
    assert gpu_solve(la, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)).cost == 0
    sol = gpu_solve(la, np.array([0, 2], np.int32), np.array([0, 0], np.int32), np.array([5, -3], np.int32))
    assert sol.cost == -3
    sol = gpu_solve(la, np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert sol.stats["status"] == la.LA_ERR_INFEASIBLE


def test_budget_exhaustion_then_a_clean_solve(la):
    g = synth.sparse_uniform(2000, 8, 40)
    sol = gpu_solve(la, *g, scan_budget=3000)
    assert sol.stats["status"] == la.LA_ERR_ITER_LIMIT
    expect_same(la, *g)
