"""Pins for the max-flow oracle (no GPU).

Dinic's algorithm is checked against facts that do not come from itself: the
minimum cut by enumeration (max-flow min-cut theorem), closed forms (series,
parallel, disconnected), hand-worked grid fixtures under
``tests/golden/maxflow/``, scipy's ``maximum_flow``, and the capacity of the
cut it returns.
"""

import glob
import os

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "maxflow")


def load_grid_fixture(path):
    kv = {}
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        parts = line.split()
        kv[parts[0]] = parts[1:]
    H, W = int(kv["H"][0]), int(kv["H"][2])
    cap = np.array([[int(v) for v in kv[k]] for k in ("right", "left", "down", "up")], np.int32).reshape(4, H, W)
    src = np.array([int(v) for v in kv["src"]], np.int32).reshape(H, W)
    snk = np.array([int(v) for v in kv["snk"]], np.int32).reshape(H, W)
    side = np.array([int(v) for v in kv["side"]], np.uint8).reshape(H, W)
    return cap, src, snk, int(kv["flow"][0]), side


def random_graph(rng, nn, density, hi):
    arcs = [(a, b, int(rng.integers(0, hi + 1))) for a in range(nn) for b in range(nn)
            if a != b and rng.random() < density]
    arcs += [(a, b, int(rng.integers(0, hi + 1))) for a, b, _ in arcs[: len(arcs) // 5]]   # parallel arcs
    tail = np.array([a[0] for a in arcs], np.int32)
    head = np.array([a[1] for a in arcs], np.int32)
    cap = np.array([a[2] for a in arcs], np.int64)
    return tail, head, cap


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))), ids=os.path.basename)
def test_grid_fixtures(path):
    cap, src, snk, flow, side = load_grid_fixture(path)
    g = oracle.grid_arcs(cap, src, snk)
    v, s = oracle.maxflow_dinic(*g)
    assert v == flow
    assert oracle.min_cut_brute(*g)[0] == flow
    assert oracle.cut_capacity(*g, side=np.concatenate([side.ravel(), [1, 0]])) == flow
    assert oracle.cut_capacity(*g, side=s) == flow


def test_dinic_equals_enumerated_min_cut():
    rng = np.random.default_rng(41)
    for trial in range(300):
        nn = int(rng.integers(2, 11))
        tail, head, cap = random_graph(rng, nn, float(rng.uniform(0.1, 0.7)), [1, 5, 100][trial % 3])
        s, t = 0, nn - 1
        want, _ = oracle.min_cut_brute(nn, tail, head, cap, s, t)
        v, side = oracle.maxflow_dinic(nn, tail, head, cap, s, t)
        assert v == want
        assert side[s] == 1 and side[t] == 0
        assert oracle.cut_capacity(nn, tail, head, cap, s, t, side) == v


def test_closed_forms():
    # series: s - a - b - t, the bottleneck
    assert oracle.maxflow_dinic(4, [0, 1, 2], [1, 2, 3], [7, 3, 9], 0, 3)[0] == 3
    # k disjoint parallel paths: the sum of their bottlenecks
    k = 20
    tail = [0] * k + list(range(2, k + 2))
    head = list(range(2, k + 2)) + [1] * k
    cap = list(range(1, k + 1)) + [k + 1 - i for i in range(1, k + 1)]
    assert oracle.maxflow_dinic(k + 2, tail, head, cap, 0, 1)[0] == sum(min(i, k + 1 - i) for i in range(1, k + 1))
    # disconnected: 0; only arcs into s: 0
    assert oracle.maxflow_dinic(4, [0, 2], [1, 3], [5, 5], 0, 3)[0] == 0
    assert oracle.maxflow_dinic(3, [1, 2], [0, 0], [5, 5], 0, 2)[0] == 0
    # unit bipartite matching r1-c1, r1-c2, r2-c1 with r1 -> c1 tried first:
    # the second unit of flow needs the backward arc c1 -> r1 (a reroute)
    assert oracle.maxflow_dinic(6, [0, 0, 1, 1, 2, 3, 4], [1, 2, 3, 4, 3, 5, 5], [1] * 7, 0, 5)[0] == 2
    # a grid with no source arcs carries nothing
    cap, src, snk = synth.grid_cut(9, 7, 1)
    assert oracle.maxflow_dinic(*oracle.grid_arcs(cap, 0 * src, snk))[0] == 0


@pytest.mark.parametrize("case", ["grid-32x24", "grid-64x64", "random-200"])
def test_dinic_matches_scipy(case):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    if case.startswith("grid"):
        H, W = (32, 24) if case == "grid-32x24" else (64, 64)
        nn, tail, head, cap, s, t = oracle.grid_arcs(*synth.grid_cut(H, W, 3))
    else:
        rng = np.random.default_rng(5)
        nn = 200
        tail, head, cap = random_graph(rng, nn, 0.05, 50)
        s, t = 0, nn - 1
    keep = (cap > 0) & (tail != head)
    m = sp.csr_matrix((cap[keep].astype(np.int32), (tail[keep], head[keep])), shape=(nn, nn))
    want = csgraph.maximum_flow(m, s, t).flow_value
    v, side = oracle.maxflow_dinic(nn, tail, head, cap, s, t)
    assert v == want
    assert oracle.cut_capacity(nn, tail, head, cap, s, t, side) == v


def test_cut_capacity_rejects_bad_sides():
    nn, tail, head, cap, s, t = oracle.grid_arcs(*synth.grid_cut(6, 5, 2))
    side = np.zeros(nn, np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.cut_capacity(nn, tail, head, cap, s, t, side)      # s not on the source side
    v, good = oracle.maxflow_dinic(nn, tail, head, cap, s, t)
    worse = good.copy()
    inner = np.nonzero(good[: nn - 2] == 0)[0]
    if inner.size:
        worse[inner[0]] = 1
        assert oracle.cut_capacity(nn, tail, head, cap, s, t, worse) >= v


def test_grid_generator_is_symmetric_and_bounded():
    cap, src, snk = synth.grid_cut(40, 30, 7)
    assert cap.shape == (4, 40, 30) and src.shape == snk.shape == (40, 30)
    assert (cap >= 0).all() and (src >= 0).all() and (snk >= 0).all()
    np.testing.assert_array_equal(cap[0, :, :-1], cap[1, :, 1:])
    np.testing.assert_array_equal(cap[2, :-1, :], cap[3, 1:, :])
    assert (cap[0, :, -1] == 0).all() and (cap[1, :, 0] == 0).all()
    assert (cap[2, -1, :] == 0).all() and (cap[3, 0, :] == 0).all()
