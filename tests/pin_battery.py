"""A compact battery of the oracle's pins, runnable against any build of
``oracle.c``. ``tests/test_oracle_mutations.py`` runs it on the real oracle
(it must pass) and on copies with planted mistakes (each must fail).

Usage: ``python pin_battery.py [path/to/oracle.c]`` exits 0 when every pin
holds and 1 at the first failure.
"""

import glob
import itertools
import os
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _fixture(path):
    lines = [l for l in open(path) if l.strip() and not l.startswith("#")]
    cost = int(lines[0].split()[1])
    m = lines[1].split()[1:]
    match = None if m == ["any"] else [int(t) for t in m]
    C = np.array([[int(t) for t in l.split()] for l in lines[3:]], dtype=np.int32)
    return C, cost, match


def _enumerate(C):
    n = C.shape[0]
    return min(sum(int(C[x, p[x]]) for x in range(n))
               for p in itertools.permutations(range(n)))


def run_all_pins(orc):
    from paper_1110_6231_gb300 import synth
    for path in sorted(glob.glob(os.path.join(HERE, "golden", "*.txt"))):
        C, cost, match = _fixture(path)
        outs = [orc.hungarian(C)[:2], orc.cost_scaling(C)[:2]]
        if C.shape[0] <= 10:
            outs.append(orc.brute_force(C))
        for c, m in outs:
            assert c == cost, path
            assert sum(int(C[x, m[x]]) for x in range(len(m))) == cost, path
            if match is not None:
                assert list(m) == match, path
    rng = np.random.default_rng(5)
    for t in range(200):
        n = int(rng.integers(1, 7))
        C = rng.integers(-30, 30, size=(n, n)).astype(np.int32)
        ref = _enumerate(C)
        assert orc.brute_force(C)[0] == ref
        assert orc.hungarian(C)[0] == ref
        g, gm, p, _ = orc.cost_scaling(C)
        assert g == ref
    from scipy.optimize import linear_sum_assignment
    for seed in range(3):
        for C in (synth.uniform_costs(97, 0, 10**5, seed), synth.geometric_costs(96, seed)):
            r, c = linear_sum_assignment(C)
            ref = int(C[r, c].sum())
            h, hm, u, v = orc.hungarian(C)
            assert h == ref and orc.check_duals(C, hm, u, v) == 0
            g, gm, p, st = orc.cost_scaling(C)
            assert g == ref and orc.check_eps_cs(C, gm, p, 1) == 0
            Ct = 97 * (int(C.max()) - int(C.min()))
            assert st["phases"] == len(orc.eps_schedule(Ct))


def run_arcfix_pins(orc):
    """Arc fixing (Sect. 5.2): the optimum with fixing equals enumeration,
    and no optimal permutation uses a deleted arc."""
    from paper_1110_6231_gb300 import synth
    rng = np.random.default_rng(41)
    for t in range(160):
        n = int(rng.integers(2, 8))
        lo, hi = [(0, 4), (0, 30), (-50, 50), (0, 1000)][t % 4]
        C = rng.integers(lo, hi, size=(n, n)).astype(np.int32)
        best, opt = None, []
        for p in itertools.permutations(range(n)):
            s = sum(int(C[x, p[x]]) for x in range(n))
            if best is None or s < best:
                best, opt = s, [p]
            elif s == best:
                opt.append(p)
        c, m, _, fixed, _ = orc.cost_scaling_arcfix(C, alpha=[2, 3, 4, 10][(t // 4) % 4])
        assert c == best
        for p in opt:
            assert not fixed[np.arange(n), np.array(p)].any()
    for seed in range(2):
        for C in (synth.uniform_costs(120, 0, 1000, seed), synth.geometric_costs(120, seed)):
            assert orc.cost_scaling_arcfix(C)[0] == orc.hungarian(C)[0]


def run_certify_pins(orc):
    """The negative-cycle certificate against enumeration: over every
    permutation of small matrices (heavy ties included) it accepts exactly
    the optimal ones, and the duals it returns pass the LP check."""
    rng = np.random.default_rng(11)
    for t in range(40):
        n = int(rng.integers(1, 6))
        C = rng.integers(-6, 6 if t % 2 else 2, size=(n, n)).astype(np.int32)
        best = _enumerate(C)
        for p in itertools.permutations(range(n)):
            m = np.array(p, dtype=np.int32)
            rc, u, v = orc.certify_optimal(C, m)
            assert (rc == 0) == (int(C[np.arange(n), m].sum()) == best)
            if rc == 0:
                assert orc.check_duals(C, m, u, v) == 0
    assert orc.certify_optimal(np.zeros((3, 3), np.int32), np.array([0, 0, 1], np.int32))[0] == 10


def _sparse_fixture(path):
    lines = [l for l in open(path) if l.strip() and not l.startswith("#")]
    c = lines[0].split()[1]
    cost = None if c == "infeasible" else int(c)
    n = int(lines[2].split()[1])
    arcs = sorted((tuple(int(t) for t in l.split()) for l in lines[4:]), key=lambda a: a[0])
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for r, _, _ in arcs:
        row_ptr[r + 1] += 1
    return (np.cumsum(row_ptr).astype(np.int32), np.array([a[1] for a in arcs], dtype=np.int32),
            np.array([a[2] for a in arcs], dtype=np.int32)), cost


def run_sparse_pins(orc):
    from paper_1110_6231_gb300 import synth
    for path in sorted(glob.glob(os.path.join(HERE, "golden", "sparse", "*.txt"))):
        (rp, cols, costs), cost = _sparse_fixture(path)
        for solve in (orc.sparse_brute_force, orc.sparse_ssp):
            try:
                got = solve(rp, cols, costs)[0]
            except orc.Infeasible:
                got = None
            assert got == cost, path
    rng = np.random.default_rng(6)
    for t in range(150):
        n = int(rng.integers(1, 7))
        arcs = [(x, y, int(rng.integers(-20, 20))) for x in range(n) for y in range(n) if rng.random() < 0.6]
        if t % 2 and arcs:   # parallel arcs: a matching uses the cheaper one
            arcs += [(a[0], a[1], int(rng.integers(-20, 20))) for a in arcs[: max(1, len(arcs) // 3)]]
        arcs.sort(key=lambda a: a[0])
        w = {}
        for r, c, x in arcs:
            w[(r, c)] = min(x, w.get((r, c), x))
        feas = [sum(w[(x, p[x])] for x in range(n)) for p in itertools.permutations(range(n))
                if all((x, p[x]) in w for x in range(n))]
        ref = min(feas) if feas else None
        row_ptr = np.zeros(n + 1, dtype=np.int32)
        for r, _, _ in arcs:
            row_ptr[r + 1] += 1
        rp = np.cumsum(row_ptr).astype(np.int32)
        cols = np.array([a[1] for a in arcs], dtype=np.int32)
        costs = np.array([a[2] for a in arcs], dtype=np.int32)
        for solve in (orc.sparse_brute_force, orc.sparse_ssp):
            try:
                got = solve(rp, cols, costs)
            except orc.Infeasible:
                got = None
            assert (got and got[0]) == ref if ref is not None else got is None
            if got is not None and solve is orc.sparse_ssp:
                assert orc.sparse_check_duals(rp, cols, costs, got[1], got[2], got[3]) == 0
    rp, cols, costs = synth.sparse_uniform(150, 5, 2)
    c, m, u, v = orc.sparse_ssp(rp, cols, costs)
    assert orc.sparse_check_duals(rp, cols, costs, m, u, v) == 0
    assert int(u.sum() + v.sum()) == c


def run_maxflow_pins(orc):
    from paper_1110_6231_gb300 import synth
    for path in sorted(glob.glob(os.path.join(HERE, "golden", "maxflow", "*.txt"))):
        kv = {}
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                kv[parts[0]] = parts[1:]
        H, W = int(kv["H"][0]), int(kv["H"][2])
        cap = np.array([[int(v) for v in kv[k]] for k in ("right", "left", "down", "up")]).reshape(4, H, W)
        g = orc.grid_arcs(cap, np.array([int(v) for v in kv["src"]]).reshape(H, W),
                          np.array([int(v) for v in kv["snk"]]).reshape(H, W))
        assert orc.maxflow_dinic(*g)[0] == int(kv["flow"][0]), path
        assert orc.min_cut_brute(*g)[0] == int(kv["flow"][0]), path
    # unit matching r1-c1, r1-c2, r2-c1 with r1 -> c1 tried first: the second
    # unit needs the first path rerouted through the backward arc c1 -> r1
    assert orc.maxflow_dinic(6, [0, 0, 1, 1, 2, 3, 4], [1, 2, 3, 4, 3, 5, 5], [1] * 7, 0, 5)[0] == 2
    rng = np.random.default_rng(8)
    for t in range(120):
        nn = int(rng.integers(2, 9))
        arcs = [(a, b, int(rng.integers(0, 20))) for a in range(nn) for b in range(nn)
                if a != b and rng.random() < 0.45]
        tail = np.array([a[0] for a in arcs], np.int32)
        head = np.array([a[1] for a in arcs], np.int32)
        cap = np.array([a[2] for a in arcs], np.int64)
        ref = orc.min_cut_brute(nn, tail, head, cap, 0, nn - 1)[0]
        v, side = orc.maxflow_dinic(nn, tail, head, cap, 0, nn - 1)
        assert v == ref
        assert orc.cut_capacity(nn, tail, head, cap, 0, nn - 1, side) == v
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_flow
    nn, tail, head, cap, s, t = orc.grid_arcs(*synth.grid_cut(20, 17, 4))
    keep = cap > 0
    m = csr_matrix((cap[keep].astype(np.int32), (tail[keep], head[keep])), shape=(nn, nn))
    assert orc.maxflow_dinic(nn, tail, head, cap, s, t)[0] == maximum_flow(m, s, t).flow_value


def main(argv):
    import oracle as orc
    if len(argv) > 1:
        src = os.path.abspath(argv[1])
        tmp = tempfile.mkdtemp(prefix="oracle_mut_")
        orc._SRC = src
        orc._LIB = os.path.join(tmp, "liboracle.so")
    try:
        run_all_pins(orc)
        run_arcfix_pins(orc)
        run_certify_pins(orc)
        run_sparse_pins(orc)
        run_maxflow_pins(orc)
    except AssertionError:
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
