"""GPU parity of the one-CTA solver for small instances against the oracle.

For n <= 300 with a cost range that fits 16 bits (n <= 224 otherwise) the
whole solve runs on one CTA with the matrix and the column keys in shared
memory. Every case compares the exact optimal cost with the oracle's and
checks the matching and, with the returned prices, the 1-optimality of
every row on costs scaled by n + 1 (which proves optimality), on both sides
of the size and range limits; the same instances through the general path
(LA_FLAG_NO_SMALL_KERNEL) must give the same optimum.
"""

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def la():
    import torch
    from paper_1110_6231_gb300 import build
    build.build()
    import paper_1110_6231_gb300 as la
    assert torch.cuda.is_available()
    return la


def run(la, C, **kw):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(C, dtype=np.int32)).cuda()
    sol = la.solve(t, want_prices=True, **kw)
    return sol.cost, sol.match.cpu().numpy(), sol.prices.cpu().numpy(), sol.stats


CASES = [
    ("uniform", 2, 1000), ("uniform", 3, 5), ("uniform", 31, 1000), ("uniform", 128, 1000),
    ("uniform", 256, 1000), ("uniform", 299, 65535), ("uniform", 300, 1000), ("uniform", 301, 1000),
    ("uniform", 200, 1 << 20), ("uniform", 224, 1 << 20), ("uniform", 225, 1 << 20),
    ("geometric", 100, None), ("geometric", 300, None), ("ties", 257, 2), ("negative", 150, None),
]


def make(kind, n, hi, seed):
    if kind == "uniform":
        return synth.uniform_costs(n, 0, hi, seed)
    if kind == "geometric":
        return synth.geometric_costs(n, seed)
    rng = np.random.default_rng(seed)
    if kind == "ties":
        return rng.integers(0, hi, size=(n, n)).astype(np.int32)
    return rng.integers(-(2**31), 2**31 - 1, size=(n, n), dtype=np.int64).astype(np.int32)


@pytest.mark.parametrize("kind,n,hi", CASES, ids=[f"{k}-{n}-{h}" for k, n, h in CASES])
def test_small_kernel_is_exact(la, kind, n, hi):
    for seed in range(3):
        C = make(kind, n, hi, seed)
        ref = oracle.hungarian(C)[0]
        cost, match, prices, st = run(la, C)
        assert cost == ref
        assert oracle.check_matching(C, match, cost) == 0
        assert oracle.check_eps_cs(C, match, prices, 1) == 0
        rng = int(C.max()) - int(C.min())
        expect_small = (rng <= 65535 and n <= 300) or n <= 224
        assert st["small_kernel"] == int(expect_small), (n, rng)
        if expect_small:
            assert st["scans"] >= n * st["phases"] and st["full_scans"] == st["scans"]
        gen = run(la, C, flags=la.LA_FLAG_NO_SMALL_KERNEL)
        assert gen[0] == ref and gen[3]["small_kernel"] == 0


def test_small_kernel_options(la):
    """Alpha, eps0, warm start prices and the scan budget on the small path."""
    import torch
    C = synth.uniform_costs(256, 0, 1000, 9)
    h, hm, u, v = oracle.hungarian(C)
    for alpha in (2, 4, 64):
        assert run(la, C, alpha=alpha)[0] == h
    assert run(la, C, eps0=1)[0] == h
    duals = torch.from_numpy(257 * v).cuda()
    cost, match, prices, st = run(la, C, init_prices=duals, eps0=1)
    assert cost == h and st["small_kernel"] == 1 and st["scans"] <= 2 * 256
    t = torch.from_numpy(C).cuda()
    stopped = la.solve(t, scan_budget=100, check=False)
    assert stopped.stats["status"] == la.LA_ERR_ITER_LIMIT
    assert la.solve(t).cost == h
