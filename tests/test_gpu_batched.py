"""GPU parity of la_solve_batched against the CPU oracle, instance by
instance: exact optimal cost and a valid matching of that cost."""

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


def pack(instances):
    ns = np.array([c.shape[0] for c in instances], dtype=np.int32)
    offsets = np.zeros(len(instances), dtype=np.int64)
    sizes = ns.astype(np.int64) ** 2
    if len(instances) > 1:
        offsets[1:] = np.cumsum(sizes)[:-1]
    flat = np.concatenate([c.ravel() for c in instances]) if instances else np.zeros(0, np.int32)
    return flat.astype(np.int32), offsets, ns


def run(la, flat, offsets, ns, **kw):
    import torch
    sol = la.solve_batched(torch.from_numpy(flat).cuda(), torch.from_numpy(offsets).cuda(),
                           torch.from_numpy(ns).cuda(), options=la.batch_options(**kw) if kw else None,
                           check=False)
    return sol


def verify(flat, offsets, ns, sol, expected=None):
    costs = sol.costs.cpu().numpy()
    match = sol.match.cpu().numpy()
    status = sol.status.cpu().numpy()
    mo = 0
    for i in range(len(ns)):
        n = int(ns[i])
        C = flat[offsets[i]:offsets[i] + n * n].reshape(n, n)
        ref = expected[i] if expected is not None else oracle.hungarian(C)[0]
        assert status[i] == 0, (i, n, status[i])
        assert costs[i] == ref, (i, n)
        if n:
            assert oracle.check_matching(C, match[mo:mo + n], ref) == 0, (i, n)
        mo += n


@pytest.mark.parametrize("lists", [-1, 1])
def test_mixed_small_batch(la, lists):
    rng = np.random.default_rng(3)
    inst = []
    for i, n in enumerate([0, 1, 2, 3, 5, 17, 31, 32, 33, 64, 100, 129, 255, 256, 300, 513]):
        if i % 3 == 0:
            inst.append(synth.uniform_costs(n, -50, 1000, i))
        elif i % 3 == 1:
            inst.append(synth.geometric_costs(n, i))
        else:
            inst.append(rng.integers(0, 3, size=(n, n)).astype(np.int32))   # heavy ties
    flat, off, ns = pack(inst)
    sol = run(la, flat, off, ns, lists=lists)
    assert sol.stats["rc"] == 0 and sol.stats["lists"] == (lists > 0)
    if lists > 0:
        assert 0 < sol.stats["full_scans"] < sol.stats["scans"]
    else:
        assert sol.stats["full_scans"] == sol.stats["scans"]
    verify(flat, off, ns, sol)


@pytest.mark.parametrize("block,slots", [(64, 1), (128, 2), (256, 4), (512, 8), (1024, 3), (512, 0)])
def test_cta_shapes_and_no_graph(la, block, slots):
    """Every CTA shape (threads x resident instances, more slots than warps
    included) gives the oracle's costs, launched directly or from a graph."""
    flat, off, ns = synth.batch(40, 7, lo=16, hi=400)
    expected = [oracle.cost_scaling(flat[off[i]:off[i] + int(ns[i]) ** 2].reshape(int(ns[i]), int(ns[i])))[0]
                for i in range(len(ns))]
    for no_graph in (False, True):
        sol = run(la, flat, off, ns, block_threads=block, slots=slots, no_graph=no_graph, max_n=512)
        assert sol.stats["rc"] == 0
        assert sol.stats["graph"] == (0 if no_graph else 1)
        assert sol.stats["slots"] == (slots or 4)
        verify(flat, off, ns, sol, expected)


def test_slots_bounded_by_shared_memory(la):
    """Eight slots of max_n = 8192 keys would need 512 KB: the launch keeps
    as many as fit in 192 KB (three) and still solves a large instance."""
    inst = [synth.uniform_costs(n, 0, 1000, n) for n in (2000, 700, 5)]
    flat, off, ns = pack(inst)
    sol = run(la, flat, off, ns, slots=8, max_n=8192)
    assert sol.stats["rc"] == 0 and sol.stats["slots"] == 3
    verify(flat, off, ns, sol)


def test_shared_memory_at_exactly_48KB(la):
    """Six slots of max_n = 1024 keys are exactly 48 KB of dynamic shared
    memory; with the kernel's slot records the CTA needs more than 48 KB,
    so the launch must opt in to the larger size."""
    flat, off, ns = synth.batch(30, 9, lo=16, hi=300)
    sol = run(la, flat, off, ns, slots=6, max_n=1024)
    assert sol.stats["rc"] == 0 and sol.stats["slots"] == 6
    verify(flat, off, ns, sol)


def test_batch_workload_sample_and_graph_replay(la):
    """A sample of the 10,000-instance workload (n log-uniform in [16, 1024],
    half uniform [0, 10^4], half geometric), solved twice from the cached
    graph, with the data changed in place between the two launches."""
    import torch
    flat, off, ns = synth.batch(120, 0)
    expected = [oracle.cost_scaling(flat[off[i]:off[i] + int(ns[i]) ** 2].reshape(int(ns[i]), int(ns[i])))[0]
                for i in range(len(ns))]
    dc, do, dn = (torch.from_numpy(a).cuda() for a in (flat, off, ns))
    opt = la.batch_options(max_n=1024, alpha=[0] * 4 + [4] * 12)
    s1 = la.solve_batched(dc, do, dn, options=opt)
    verify(flat, off, ns, s1, expected)
    flat2, off2, ns2 = synth.batch(120, 0, cost_hi=5000)           # same sizes, new costs
    assert np.array_equal(ns2, ns)
    dc.copy_(torch.from_numpy(flat2))
    s2 = la.solve_batched(dc, do, dn, options=opt)
    assert s2.stats["graph"] == 1
    verify(flat2, off2, ns2, s2)


def test_full_batch_workload_as_timed_is_certified_optimal(la):
    """The whole 10,000-instance workload, tuned and launched the way the
    throughput measurement launches it (autotuned CTA shape, slots and
    alpha per size bucket; graph capture, then a timed-style replay). For
    every instance: status 0, a permutation of the claimed cost, and the
    oracle's negative-cycle certificate proves it optimal at any n. Every
    250th instance is also solved by the oracle's Hungarian method."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    import torch
    from paper_1110_6231_gb300 import tune
    flat, off, ns = synth.batch(10_000, 0)
    dc, do, dn = (torch.from_numpy(a).cuda() for a in (flat, off, ns))
    table = tune.autotune_batched(dc, do, dn, reps=1)
    opt = tune.options_from_table(table, profile=True)
    la.solve_batched(dc, do, dn, options=opt)
    sol = la.solve_batched(dc, do, dn, options=opt)
    assert sol.stats["rc"] == 0 and sol.stats["graph"] == 1 and sol.stats["failed"] == 0
    costs = sol.costs.cpu().numpy()
    match = sol.match.cpu().numpy()
    status = sol.status.cpu().numpy()
    mo = np.zeros(len(ns) + 1, dtype=np.int64)
    mo[1:] = np.cumsum(ns.astype(np.int64))

    def one(i):   # the oracle's C calls release the GIL
        n = int(ns[i])
        C = flat[off[i]:off[i] + n * n].reshape(n, n)
        m = match[mo[i]:mo[i + 1]]
        res = (int(status[i]), oracle.check_matching(C, m, int(costs[i])), oracle.certify_optimal(C, m)[0])
        if i % 250 == 0:
            res += (int(oracle.hungarian(C)[0] != costs[i]),)
        return i, res

    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        bad = [(i, r) for i, r in ex.map(one, range(len(ns))) if any(r)]
    assert not bad, bad[:5]


def test_concurrent_n4096_instances_one_per_cta(la):
    """The ten stored n = 4096 optima (costs in [0, 2^20), 64-bit reduced
    costs) solved concurrently, one instance per CTA, from matrices drawn on
    the GPU by the torch twin of the generator (checked against the stored
    digests first); then in the throughput line's shape at every alpha its
    tuner may pick."""
    import hashlib
    import json
    import os

    import torch
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "optimal_costs.json")
    cases = [c for c in json.load(open(path))["cases"] if c["workload"] == "uniform-n4096-c2^20"]
    n = 4096
    dc = torch.empty(len(cases) * n * n, dtype=torch.int32, device="cuda")
    for i, c in enumerate(cases):
        m = synth.uniform_costs_torch(n, 0, (1 << 20) - 1, c["seed"], device="cuda")
        assert hashlib.sha256(m.cpu().numpy().tobytes()).hexdigest() == c["sha256"]
        dc[i * n * n:(i + 1) * n * n] = m.view(-1)
    off = torch.arange(len(cases), dtype=torch.int64, device="cuda") * (n * n)
    ns = torch.full((len(cases),), n, dtype=torch.int32, device="cuda")
    for lists in (0, -1):   # 0: the library's choice for n = 4096 is lists on
        sol = la.solve_batched(dc, off, ns, options=la.batch_options(block_threads=256, slots=1, max_n=n,
                                                                      alpha=[48] * 16, lists=lists))
        assert sol.stats["rc"] == 0 and sol.stats["lists"] == (lists == 0)
        assert sol.costs.cpu().tolist() == [c["cost"] for c in cases]
        match = sol.match.cpu().numpy()
        C0 = synth.instance("uniform-n4096-c2^20", cases[0]["seed"])
        assert oracle.check_matching(C0, match[:n], cases[0]["cost"]) == 0
    # the shape and every alpha the throughput line may be tuned to
    from paper_1110_6231_gb300 import tune
    shape = dict(block_threads=256, slots=2, max_n=n, lists=1)
    tuned = tune.autotune_batch_alpha(dc, off, ns, **shape)
    assert tuned["alpha"] in tune.DEFAULT_BATCH_ALPHAS
    assert sorted(tuned["device_ms"]) == sorted(tune.DEFAULT_BATCH_ALPHAS)
    for a in tune.DEFAULT_BATCH_ALPHAS:
        sol = la.solve_batched(dc, off, ns, options=la.batch_options(alpha=[a] * 16, **shape))
        assert sol.costs.cpu().tolist() == [c["cost"] for c in cases], a


def test_invalid_sizes_flagged_per_instance(la):
    inst = [synth.uniform_costs(20, 0, 9, 1), synth.uniform_costs(40, 0, 9, 2)]
    flat, off, ns = pack(inst)
    sol = run(la, flat, off, ns, max_n=32)
    status = sol.status.cpu().numpy()
    assert status[0] == 0 and status[1] == la.LA_ERR_INVALID
    assert sol.stats["rc"] == la.LA_ERR_INVALID and sol.stats["failed"] == 1
    assert int(sol.costs[0].item()) == oracle.hungarian(inst[0])[0]


def test_empty_batch(la):
    import torch
    z = torch.zeros(0, dtype=torch.int32, device="cuda")
    sol = la.solve_batched(z, torch.zeros(0, dtype=torch.int64, device="cuda"), z)
    assert sol.costs.numel() == 0


def test_instances_that_run_out_of_budget_fail_alone(la):
    """With one row scan per row and phase (plus a slack of 4096), the large
    instances run out of budget inside their chains: their rows are given up
    one by one, each such instance ends with LA_ERR_ITER_LIMIT and frees its
    slot, while the small instances of the same CTAs are still solved
    exactly. The same batch then solves cleanly with the default budget."""
    small = [synth.uniform_costs(n, 0, 50, 100 + n) for n in (3, 8, 16, 24)]
    large = [synth.uniform_costs(n, 0, (1 << 20) - 1, 200 + n) for n in (400, 512, 640, 700)]
    inst = [c for pair in zip(small, large) for c in pair]
    flat, off, ns = pack(inst)
    sol = run(la, flat, off, ns, budget_factor=1, slots=4, block_threads=128)
    status = sol.status.cpu().numpy()
    costs = sol.costs.cpu().numpy()
    assert sol.stats["rc"] == la.LA_ERR_ITER_LIMIT
    for i, C in enumerate(inst):
        if C.shape[0] <= 24:
            assert status[i] == 0 and costs[i] == oracle.hungarian(C)[0]
        else:
            assert status[i] == la.LA_ERR_ITER_LIMIT
    assert sol.stats["failed"] == len(large)
    verify(flat, off, ns, run(la, flat, off, ns, slots=4, block_threads=128))
