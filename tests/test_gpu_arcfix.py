"""GPU parity of arc fixing (Sect. 5.2) against the oracle.

After every phase but the last the refine drops each arc whose reduced
cost exceeds 2 n eps; a row whose remaining arcs fit in its candidate list
keeps only those. The optimal cost must stay the oracle's bit for bit, and
the returned matching must pass the oracle's certificates: a permutation of
the claimed cost, and optimal by the negative-cycle criterion, which needs
no prices (the final prices certify only the arcs kept, so arc fixing is
off whenever prices are requested).
"""

import json
import os

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def la():
    import torch
    from paper_1110_6231_gb300 import build
    build.build()
    import paper_1110_6231_gb300 as la
    assert torch.cuda.is_available()
    return la


def solve(la, C, **kw):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(C, dtype=np.int32)).cuda()
    # arc fixing belongs to the general path (small instances are otherwise
    # solved whole in one CTA's shared memory)
    kw["flags"] = kw.get("flags", 0) | la.LA_FLAG_NO_SMALL_KERNEL
    sol = la.solve(t, **kw)
    return sol.cost, sol.match.cpu().numpy(), sol.stats


CASES = {
    "uniform-n257-c1000": lambda: synth.uniform_costs(257, 0, 1000, 1),
    "uniform-n1000-c1000": lambda: synth.uniform_costs(1000, 0, 1000, 2),
    "uniform-n1024-c2^20": lambda: synth.uniform_costs(1024, 0, (1 << 20) - 1, 3),
    "geometric-n1023": lambda: synth.geometric_costs(1023, 4),
    "geometric-n2048": lambda: synth.geometric_costs(2048, 5),
    "ties-n515": lambda: np.random.default_rng(6).integers(0, 4, size=(515, 515)).astype(np.int32),
}


@pytest.mark.parametrize("alpha", [10, 64])
@pytest.mark.parametrize("name", sorted(CASES))
def test_arc_fixing_keeps_the_optimum(la, name, alpha):
    C = CASES[name]()
    ref = oracle.hungarian(C)[0]
    cost, match, st = solve(la, C, alpha=alpha)
    assert cost == ref
    assert oracle.check_matching(C, match, cost) == 0
    assert oracle.certify_optimal(C, match)[0] == 0
    # the oracle with the same rule reaches the same optimum
    assert oracle.cost_scaling_arcfix(C, alpha=alpha)[0] == ref
    if name.startswith("uniform") and alpha == 10:
        # late phases run on rows cut down to a few arcs
        assert st["fixed_rows"] > C.shape[0] // 2
        assert 0 < st["fixed_arcs"] <= 128 * st["fixed_rows"]
    off = solve(la, C, alpha=alpha, flags=la.LA_FLAG_NO_ARC_FIXING)
    assert off[0] == ref and off[2]["fixed_rows"] == 0


def test_no_arc_fixing_when_prices_are_requested(la):
    import torch
    C = synth.uniform_costs(600, 0, 1000, 7)
    sol = la.solve(torch.from_numpy(C).cuda(), want_prices=True, flags=la.LA_FLAG_NO_SMALL_KERNEL)
    assert sol.stats["fixed_rows"] == 0
    assert oracle.check_eps_cs(C, sol.match.cpu().numpy(), sol.prices.cpu().numpy(), 1) == 0


@pytest.mark.parametrize("name", ["uniform-n1000-c1000", "geometric-n2048", "ties-n515"])
def test_phase_invariants_with_arc_fixing(la, name):
    """LA_FLAG_CHECK_PHASES with fixing on: every phase ends with a perfect
    assignment, eps-optimal over each row's remaining arcs, and no price rose."""
    C = CASES[name]()
    cost, match, st = solve(la, C, alpha=10, flags=la.LA_FLAG_CHECK_PHASES)
    assert st["check_violations"] == 0 and st["checked_phases"] == st["phases"]
    assert cost == oracle.hungarian(C)[0]


def test_full_size_geometric_n8192_stored_optima(la):
    """The n = 8192 geometric workload of the throughput line, arc fixing on,
    against the optima stored by the oracle's Hungarian method."""
    cases = [c for c in json.load(open(os.path.join(GOLDEN, "optimal_costs.json")))["cases"]
             if c["workload"] == "geometric-n8192" and c["n"] == 8192]
    assert len(cases) >= 4
    for c in cases[:2]:
        C = synth.instance(c["workload"], c["seed"])
        cost, match, st = solve(la, C, alpha=10)
        assert cost == c["cost"], c
        assert oracle.check_matching(C, match, cost) == 0
        assert st["fixed_rows"] > 0
