"""GPU parity of la_maxflow_grid against the CPU oracle (maximum flow).

The flow value is compared with Dinic's algorithm on the same seeded grid,
exactly (integer capacities); the returned cut is checked as a certificate:
its source side holds no t, and the capacity of the arcs leaving it equals
the flow value (max-flow min-cut theorem), which proves both optimal.
"""

import glob
import os

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

from test_oracle_maxflow import load_grid_fixture

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "maxflow")


@pytest.fixture(scope="module")
def la():
    import torch
    from paper_1110_6231_gb300 import build
    build.build()
    import paper_1110_6231_gb300 as la
    assert torch.cuda.is_available()
    return la


def gpu_flow(la, cap, src, snk, **kw):
    import torch
    t = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda() for a in (cap, src, snk)]
    return la.maxflow_grid(*t, check=False, **kw)


def expect_same(la, cap, src, snk, **kw):
    res = gpu_flow(la, cap, src, snk, **kw)
    assert res.stats["status"] == la.LA_OK, la.la_status_string(res.stats["status"])
    g = oracle.grid_arcs(cap, src, snk)
    want, _ = oracle.maxflow_dinic(*g)
    assert res.flow == want
    side = np.concatenate([res.cut.cpu().numpy().ravel(), [1, 0]]).astype(np.uint8)
    assert oracle.cut_capacity(*g, side=side) == want
    return res


def random_grid(rng, H, W, hi, one_way=False):
    cap = rng.integers(0, hi + 1, size=(4, H, W)).astype(np.int32)
    cap[0, :, -1] = 0
    cap[1, :, 0] = 0
    cap[2, -1, :] = 0
    cap[3, 0, :] = 0
    if one_way:
        cap[1] = 0
        cap[3] = 0
    src = (rng.integers(0, hi + 1, size=(H, W)) * (rng.random((H, W)) < 0.4)).astype(np.int32)
    snk = (rng.integers(0, hi + 1, size=(H, W)) * (rng.random((H, W)) < 0.4)).astype(np.int32)
    return cap, src, snk


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))), ids=os.path.basename)
def test_fixtures(la, path):
    cap, src, snk, flow, side = load_grid_fixture(path)
    res = expect_same(la, cap, src, snk)
    assert res.flow == flow


def test_small_random_grids(la):
    rng = np.random.default_rng(51)
    for trial in range(60):
        H, W = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        expect_same(la, *random_grid(rng, H, W, [1, 9, 1000][trial % 3], one_way=trial % 4 == 0))


@pytest.mark.parametrize("H,W,cycle", [(64, 64, 0), (97, 131, 7), (256, 256, 0), (256, 256, 500)])
def test_graph_cut_instances(la, H, W, cycle):
    expect_same(la, *synth.grid_cut(H, W, H + W), cycle=cycle)


def test_full_size_workload(la):
    res = expect_same(la, *synth.grid_instance("gridcut-1024x1024", 0))
    assert res.stats["rounds"] >= 1 and res.stats["global_relabels"] == res.stats["rounds"] + 1


@pytest.mark.parametrize("H,W", [(128, 128), (256, 256), (70, 300)])
def test_crossing_grids(la, H, W):
    """Every unit of flow crosses the grid from the left to the right column."""
    expect_same(la, *synth.grid_crossing(H, W, H + 7 * W))


def test_crossing_workload_certified(la):
    """512 x 512 crossing grid (Dinic needs about a minute here): the cut the
    GPU returns has exactly the capacity of its flow, which proves both
    optimal (weak duality), and it separates the left column from the right."""
    cap, src, snk = synth.grid_instance("gridcross-512x512", 0)
    res = gpu_flow(la, cap, src, snk)
    assert res.stats["status"] == la.LA_OK
    side = res.cut.cpu().numpy()
    g = oracle.grid_arcs(cap, src, snk)
    assert oracle.cut_capacity(*g, side=np.concatenate([side.ravel(), [1, 0]]).astype(np.uint8)) == res.flow
    assert res.flow == res.stats["flow"] > 0


def test_degenerate_grids(la):
    one = [np.zeros((4, 1, 1), np.int32), np.array([[5]], np.int32), np.array([[3]], np.int32)]
    assert expect_same(la, *one).flow == 3
    cap, src, snk = synth.grid_cut(33, 17, 2)
    assert expect_same(la, cap, 0 * src, snk).flow == 0            # no source arcs
    assert expect_same(la, cap, src, 0 * snk).flow == 0            # no sink arcs
    assert expect_same(la, 0 * cap, src, snk).flow == int(np.minimum(src, snk).sum())   # no grid arcs


def test_invalid_capacities_rejected_on_device(la):
    cap, src, snk = synth.grid_cut(8, 9, 3)
    bad = cap.copy()
    bad[0, 2, -1] = 1                                               # an arc leaving the grid
    assert gpu_flow(la, bad, src, snk).stats["status"] == la.LA_ERR_INVALID
    neg = src.copy()
    neg[1, 1] = -1
    assert gpu_flow(la, cap, neg, snk).stats["status"] == la.LA_ERR_INVALID
    expect_same(la, cap, src, snk)                                  # the workspace is still good


def test_round_limit_then_a_clean_solve(la):
    g = synth.grid_cut(128, 128, 9)
    res = gpu_flow(la, *g, cycle=1, max_rounds=1)
    assert res.stats["status"] == la.LA_ERR_ITER_LIMIT
    expect_same(la, *g)
