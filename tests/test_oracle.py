"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself: hand-worked
and closed-form instances under ``tests/golden/``, an independent pure-Python
enumeration, scipy's ``linear_sum_assignment``, the LP duality certificate,
the paper's epsilon-optimality error bound (Sect. 5.1, Lemma 5.6 with the
n + 1 scaling) and its invariants (Lemma 5.2: prices never increase), and a
hand-computed epsilon schedule (Algorithm 5.0's outer loop).
"""

import glob
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_fixture(path):
    lines = [l for l in open(path) if l.strip() and not l.startswith("#")]
    cost = int(lines[0].split()[1])
    m = lines[1].split()[1:]
    match = None if m == ["any"] else np.array([int(t) for t in m], dtype=np.int32)
    assert lines[2].strip() == "matrix"
    C = np.array([[int(t) for t in l.split()] for l in lines[3:]], dtype=np.int32)
    return C, cost, match


FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


def python_enumeration(C):
    n = C.shape[0]
    best = None
    for p in itertools.permutations(range(n)):
        s = sum(int(C[x, p[x]]) for x in range(n))
        if best is None or s < best:
            best = s
    return 0 if best is None else best


@pytest.mark.parametrize("path", FIXTURES, ids=os.path.basename)
def test_fixtures_all_oracles(path):
    C, cost, match = load_fixture(path)
    results = [oracle.hungarian(C)[:2], oracle.cost_scaling(C, check=True)[:2]]
    if C.shape[0] <= 10:
        results.append(oracle.brute_force(C))
    for got_cost, got_match in results:
        assert got_cost == cost
        assert oracle.check_matching(C, got_match, cost) == 0
        if match is not None:
            np.testing.assert_array_equal(got_match, match)


def test_brute_force_matches_python_enumeration():
    rng = np.random.default_rng(11)
    for _ in range(150):
        n = int(rng.integers(1, 7))
        C = rng.integers(-20, 20, size=(n, n)).astype(np.int32)
        assert oracle.brute_force(C)[0] == python_enumeration(C)


def _tiny_instances(rng, count):
    kinds = ["uniform", "ties", "negative", "extreme", "binary"]
    for t in range(count):
        n = int(rng.integers(1, 9))
        kind = kinds[t % len(kinds)]
        if kind == "uniform":
            C = rng.integers(0, 1000, size=(n, n))
        elif kind == "ties":
            C = rng.integers(0, 3, size=(n, n))
        elif kind == "negative":
            C = rng.integers(-10**6, 10, size=(n, n))
        elif kind == "extreme":
            C = rng.choice([-(2**31), 2**31 - 1, 0, -1, 1], size=(n, n))
        else:
            C = rng.integers(0, 2, size=(n, n))
        yield kind, C.astype(np.int32)


def test_hungarian_and_cost_scaling_match_brute_force():
    rng = np.random.default_rng(2024)
    for kind, C in _tiny_instances(rng, 600):
        b, bm = oracle.brute_force(C)
        h, hm, u, v = oracle.hungarian(C)
        g, gm, p, _ = oracle.cost_scaling(C, check=True)
        assert b == h == g, (kind, C)
        assert oracle.check_matching(C, bm, b) == 0
        assert oracle.check_matching(C, hm, h) == 0
        assert oracle.check_matching(C, gm, g) == 0
        assert oracle.check_duals(C, hm, u, v) == 0
        assert oracle.check_eps_cs(C, gm, p, 1) == 0


@pytest.mark.parametrize("n", [2, 3, 17, 64, 129, 300])
def test_hungarian_dual_certificate_and_scipy(n):
    scipy_opt = pytest.importorskip("scipy.optimize")
    for seed in range(3):
        C = synth.uniform_costs(n, -500, 500, seed)
        h, hm, u, v = oracle.hungarian(C)
        assert oracle.check_duals(C, hm, u, v) == 0
        assert int(u.sum() + v.sum()) == h
        r, c = scipy_opt.linear_sum_assignment(C)
        assert int(C[r, c].sum()) == h


@pytest.mark.parametrize("kind,n", [("uniform", 100), ("uniform", 257), ("uniform", 512),
                                    ("geometric", 128), ("geometric", 384)])
def test_cost_scaling_equals_hungarian(kind, n):
    for seed in range(2):
        if kind == "uniform":
            C = synth.uniform_costs(n, 0, (1 << 20) - 1, seed)
        else:
            C = synth.geometric_costs(n, seed)
        h, *_ = oracle.hungarian(C)
        g, gm, p, st = oracle.cost_scaling(C, check=True)
        assert g == h
        assert oracle.check_eps_cs(C, gm, p, 1) == 0
        assert st["scans"] >= n * st["phases"]     # every phase scans every row once


def test_eps_schedule_hand_computed():
    # C~ = 257 * 1000 (n = 256, costs in [0, 1000]); floor-divide by 10 until 1.
    assert oracle.eps_schedule(257_000) == [25_700, 2_570, 257, 25, 2, 1]
    # C~ = 4097 * (2^20 - 1) = 4_296_014_751.
    assert oracle.eps_schedule(4_296_014_751) == [
        429_601_475, 42_960_147, 4_296_014, 429_601, 42_960, 4_296, 429, 42, 4, 1]
    assert oracle.eps_schedule(0) == [1]          # all costs equal
    assert oracle.eps_schedule(9) == [1]
    assert oracle.eps_schedule(100, alpha=4) == [25, 6, 1]


def test_cost_scaling_phase_count_follows_schedule():
    C = synth.uniform_costs(256, 0, 1000, 5)
    Ct = 257 * (int(C.max()) - int(C.min()))
    _, _, _, st = oracle.cost_scaling(C)
    sched = oracle.eps_schedule(Ct)
    assert st["phases"] == len(sched)
    assert st["eps_first"] == sched[0] == Ct // 10


@pytest.mark.parametrize("E", [2, 7, 50, 1000, 25_000])
def test_early_stop_error_bound(E):
    """Stopping after the phase run at eps <= E leaves an eps-optimal
    assignment; summing eps-CS over the n rows on costs scaled by n + 1 gives
    (n + 1)(cost - OPT) <= n * eps_last (Sect. 5.1; Lemma 5.6)."""
    for seed in range(4):
        C = synth.uniform_costs(60, 0, 1000, 100 + seed)
        n = C.shape[0]
        opt, *_ = oracle.hungarian(C)
        Ct = (n + 1) * (int(C.max()) - int(C.min()))
        eps_last = oracle.eps_schedule(Ct, final_eps=E)[-1]
        g, gm, p, st = oracle.cost_scaling(C, final_eps=E, check=True)
        assert oracle.check_eps_cs(C, gm, p, eps_last) == 0
        assert 0 <= (n + 1) * (g - opt) <= n * eps_last


@pytest.mark.parametrize("alpha", [2, 3, 4, 8, 16, 100])
def test_alpha_does_not_change_optimum(alpha):
    C = synth.geometric_costs(200, 3)
    h, *_ = oracle.hungarian(C)
    assert oracle.cost_scaling(C, alpha=alpha, check=True)[0] == h


def test_any_start_prices_reach_the_optimum():
    """Refine's initialisation makes any price vector eps-optimal (Alg. 5.2,
    refine initialisation), so warm starts change speed, never the result."""
    rng = np.random.default_rng(7)
    C = synth.uniform_costs(150, 0, 5000, 9)
    h, *_ = oracle.hungarian(C)
    for eps0 in (0, 1, 10, 151 * 7):
        init = rng.integers(-10**7, 10**7, size=150).astype(np.int64)
        assert oracle.cost_scaling(C, eps0=eps0, init_prices=init, check=True)[0] == h


def test_optimal_duals_as_start_prices_need_few_scans():
    """Prices from optimal duals (p(y) = (n+1) v(y)) are already 0-optimal:
    with eps0 small the single refine at eps = 1 needs about one scan per row."""
    C = synth.uniform_costs(200, 0, 1000, 4)
    h, hm, u, v = oracle.hungarian(C)
    g, gm, p, st = oracle.cost_scaling(C, eps0=1, init_prices=201 * v)
    assert g == h and st["phases"] == 1
    cold = oracle.cost_scaling(C)[3]
    assert st["scans"] < cold["scans"] / 3


def test_degenerate_sizes():
    for f in (oracle.hungarian, oracle.cost_scaling):
        assert f(np.zeros((0, 0), np.int32))[0] == 0
        assert f(np.array([[42]], np.int32))[0] == 42
    assert oracle.brute_force(np.zeros((0, 0), np.int32))[0] == 0


def test_certificates_reject_bad_claims():
    C = synth.uniform_costs(30, 0, 100, 1)
    h, hm, u, v = oracle.hungarian(C)
    assert oracle.check_matching(C, hm, h + 1) == 11
    bad = hm.copy()
    bad[0] = bad[1]
    assert oracle.check_matching(C, bad, h) == 10
    assert oracle.check_duals(C, hm, u + 1, v) == 12
    swapped = hm.copy()
    swapped[[0, 1]] = swapped[[1, 0]]
    res = oracle.check_duals(C, swapped, u, v)
    assert res in (13, 0)
    _, gm, p, _ = oracle.cost_scaling(C)
    worse = gm.copy()
    worse[[0, 1]] = worse[[1, 0]]
    if oracle.check_matching(C, worse, h) != 0:  # a strictly worse matching
        assert oracle.check_eps_cs(C, worse, p, 1) == 15


def test_certificate_without_duals_accepts_exactly_the_optima():
    """or_certify_optimal (negative-cycle criterion): on every permutation of
    small matrices it accepts exactly those of least cost (enumeration); on
    larger instances it accepts the Hungarian optimum with duals that pass
    the LP check, and rejects a matching one swap away from it."""
    rng = np.random.default_rng(17)
    for t in range(60):
        n = int(rng.integers(1, 6))
        C = rng.integers(-9, 9 if t % 3 else 2, size=(n, n)).astype(np.int32)
        best = min(sum(int(C[x, p[x]]) for x in range(n)) for p in itertools.permutations(range(n)))
        for p in itertools.permutations(range(n)):
            m = np.array(p, dtype=np.int32)
            rc, u, v = oracle.certify_optimal(C, m)
            assert (rc == 0) == (int(C[np.arange(n), m].sum()) == best)
            if rc == 0:
                assert oracle.check_duals(C, m, u, v) == 0
    for C in (synth.uniform_costs(300, 0, 10**6, 3), synth.geometric_costs(256, 4)):
        cost, m, _, _ = oracle.hungarian(C)
        rc, u, v = oracle.certify_optimal(C, m)
        assert rc == 0 and oracle.check_duals(C, m, u, v) == 0
        # every strictly worse neighbour (two rows swap columns) is rejected
        for a, b in ((0, 1), (5, 77), (100, 200)):
            w = m.copy()
            w[a], w[b] = m[b], m[a]
            worse = int(C[np.arange(C.shape[0]), w].sum()) > cost
            assert (oracle.certify_optimal(C, w)[0] == 16) == worse
    assert oracle.certify_optimal(np.zeros((0, 0), np.int32), np.zeros(0, np.int32))[0] == 0
    assert oracle.certify_optimal(np.eye(3, dtype=np.int32), np.array([1, 1, 2], np.int32))[0] == 10
