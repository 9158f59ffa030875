"""Seeded generators: reproducible bytes, the shapes and value ranges of the
workloads, and the structure of the geometric instances."""

import hashlib
import json
import os

import numpy as np
import pytest

from paper_1110_6231_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "optimal_costs.json")


def test_digests_match_stored_instances():
    cases = json.load(open(GOLDEN))["cases"]
    seen = set()
    for c in cases:
        key = (c["workload"], c["n"])
        if key in seen and c["n"] > 1024:
            continue
        seen.add(key)
        C = synth.instance(c["workload"], c["seed"], c["n"])
        assert hashlib.sha256(C.tobytes()).hexdigest() == c["sha256"], c


def test_uniform_range_and_determinism():
    a = synth.uniform_costs(300, 0, 1000, 3)
    b = synth.uniform_costs(300, 0, 1000, 3)
    assert a.dtype == np.int32 and a.shape == (300, 300)
    assert np.array_equal(a, b)
    assert a.min() == 0 and a.max() == 1000
    assert not np.array_equal(a, synth.uniform_costs(300, 0, 1000, 4))
    assert abs(a.mean() - 500) < 5


def test_geometric_structure():
    n = 2000
    a, pi, b = synth.geometric_points(n, 1)
    assert np.array_equal(np.sort(pi), np.arange(n))
    jitter = b - a[pi]
    assert abs(jitter.std() - 0.01) < 0.001
    C = synth.geometric_costs(n, 1)
    assert C.min() >= 0 and C.max() <= 25000
    inv = np.empty(n, dtype=np.int64)
    inv[pi] = np.arange(n)
    # the planted matching x -> pi^-1(x) costs about 2 sigma^2 1e4 = 2 per row
    planted = C[np.arange(n), inv].astype(np.int64).sum()
    assert planted < 4 * n


def test_batch_sizes_log_uniform():
    ns = synth.batch_sizes(20000, 0)
    assert ns.min() >= 16 and ns.max() <= 1024
    frac_small = np.mean(ns < 128)          # ln(128/16) / ln(1024/16) = 0.5
    assert abs(frac_small - 0.5) < 0.02


def test_batch_packing():
    flat, off, ns = synth.batch(6, 0, lo=4, hi=12)
    assert len(off) == len(ns) == 6
    for i in range(6):
        n = int(ns[i])
        blk = flat[off[i]:off[i] + n * n].reshape(n, n)
        ref = synth.uniform_costs(n, 0, 10000, i) if i % 2 == 0 else synth.geometric_costs(n, i)
        assert np.array_equal(blk, ref)
    assert off[-1] + int(ns[-1]) ** 2 == flat.size


def test_torch_twin_of_the_uniform_generator_is_bit_identical():
    """uniform_costs_torch (int64 torch arithmetic) draws the same int32
    matrices as the numpy generator, over full int32 ranges too."""
    torch = pytest.importorskip("torch")
    for n, lo, hi, seed in ((0, 0, 5, 1), (1, 0, 5, 1), (7, -50, 1000, 3), (64, 0, (1 << 20) - 1, 0),
                            (129, 0, 10**4, 9), (33, -(1 << 31), (1 << 31) - 1, 5)):
        a = synth.uniform_costs(n, lo, hi, seed)
        b = synth.uniform_costs_torch(n, lo, hi, seed, device="cpu").numpy()
        assert a.dtype == b.dtype and np.array_equal(a, b), (n, lo, hi, seed)


def test_geometric_instances_have_their_planted_structure():
    """The geometric recipe plants a permutation: b_j is a_pi(j) moved by
    N(0, 0.01^2) per coordinate, so the optimum pairs most rows with their
    planted partner while the points are sparse next to the jitter, and
    fewer as they crowd (the mean spacing is about 1/sqrt(n)). A generator
    that lost the pairing would match almost none."""
    import oracle
    rates = []
    for n, seed in ((256, 1), (512, 2)):
        a, pi, b = synth.geometric_points(n, seed)
        C = synth.geometric_costs(n, seed)
        planted = np.empty(n, dtype=np.int64)
        planted[pi] = np.arange(n)
        cost, match, _, _ = oracle.hungarian(C)
        assert cost <= int(C[np.arange(n), planted].sum())
        rates.append(float((match == planted).mean()))
    assert rates[0] > 0.85 and rates[1] > 0.75 and rates[1] < rates[0], rates
