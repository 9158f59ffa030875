"""The lock-free bidding protocol of the parallel refine, emulated by host
threads with C11 atomics (tests/lockfree_emulation.c) and run under
ThreadSanitizer: no data race may be reported, every run must end, and the
result must be the exact optimum (the oracle's Hungarian cost, a permutation
of that cost, and eps-CS at eps = 1 with the final prices). The same holds
with candidate lists, whose bound must stay sound across the price shifts
between phases (two planted mistakes in the list rule must be seen), and
when scans read prices from a mirror that lags the keys, as the
single-solve refine does. Every
run also checks the price bounds that decide when the GPU may use 32-bit
values (the emulation exits with status 3 if one breaks), and a sequential
restatement shows that those bounds are reached. Nothing here touches a
GPU."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lockfree_emulation.c")


def _build(tmp_path, tsan, mutant=0):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    plain = str(tmp_path / f"emu{mutant}")
    r = subprocess.run([cc, "-O2", "-std=c11", "-pthread", f"-DLIST_MUTANT={mutant}", SRC, "-o", plain],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    if not tsan:
        return plain
    exe = str(tmp_path / "emu_tsan")
    r = subprocess.run([cc, "-O1", "-g", "-fsanitize=thread", "-std=c11", "-pthread", SRC, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:   # the source compiles: only the sanitizer is missing
        pytest.skip("ThreadSanitizer unavailable: " + r.stderr[-200:])
    return exe


def _run(exe, C, alpha, threads, tmp_path, lanes=0, per_lane=0, mirror=0, timeout=120):
    """Returns cost, phases, bids, match, prices, list scans, full scans."""
    n = C.shape[0]
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        np.array([n, alpha, threads, lanes, per_lane, mirror], dtype=np.int32).tofile(f)
        np.ascontiguousarray(C, dtype=np.int32).tofile(f)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    r = subprocess.run([exe, str(inp), str(out)], capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    raw = open(out, "rb").read()
    head = np.frombuffer(raw[:24], dtype=np.int64)
    match = np.frombuffer(raw[24:24 + 4 * n], dtype=np.int32)
    prices = np.frombuffer(raw[24 + 4 * n:24 + 12 * n], dtype=np.int64)
    scans = np.frombuffer(raw[24 + 12 * n:24 + 12 * n + 16], dtype=np.int64)
    return int(head[0]), int(head[1]), int(head[2]), match, prices, int(scans[0]), int(scans[1])


def _exact(C, cost, match, prices):
    return (cost == oracle.hungarian(C)[0] and oracle.check_matching(C, match, cost) == 0
            and oracle.check_eps_cs(C, match, prices, 1) == 0)


def _check(C, cost, match, prices):
    assert cost == oracle.hungarian(C)[0]
    assert oracle.check_matching(C, match, cost) == 0
    assert oracle.check_eps_cs(C, match, prices, 1) == 0


def test_protocol_is_race_free_under_threadsanitizer(tmp_path):
    exe = _build(tmp_path, tsan=True)
    cases = [synth.uniform_costs(40, 0, 1000, 1), synth.geometric_costs(48, 2),
             np.random.default_rng(3).integers(0, 3, size=(33, 33)).astype(np.int32),   # heavy ties
             synth.uniform_costs(1, -5, 5, 4), synth.uniform_costs(2, 0, 9, 5)]
    for C in cases:
        cost, phases, bids, match, prices, lists, full = _run(exe, C, 10, 8, tmp_path)
        _check(C, cost, match, prices)
        assert bids >= C.shape[0] and lists == 0 and full == bids


@pytest.mark.parametrize("threads,alpha", [(1, 10), (4, 4), (16, 10), (32, 64)])
def test_protocol_is_exact_with_many_bidders(tmp_path, threads, alpha):
    exe = _build(tmp_path, tsan=False)
    for seed, C in enumerate((synth.uniform_costs(200, 0, 10**5, 6), synth.geometric_costs(256, 7))):
        cost, phases, bids, match, prices, _, _ = _run(exe, C, alpha, threads, tmp_path)
        _check(C, cost, match, prices)
        Ct = (C.shape[0] + 1) * (int(C.max()) - int(C.min()))
        assert phases == len(oracle.eps_schedule(Ct, alpha))


# (lanes, entries per lane): the GPU's 32 x 4, and narrower lists whose bound
# theta is tighter, so that they fall back to full scans more often
LIST_SHAPES = [(32, 4), (4, 2), (8, 1)]


@pytest.mark.parametrize("lanes,per_lane", LIST_SHAPES)
def test_lists_are_race_free_under_threadsanitizer(tmp_path, lanes, per_lane):
    """The list of a row is written by the thread that holds the row and read
    by the next holder, which took the row over by a compare-and-swap or at
    the phase barrier: ThreadSanitizer must see that order."""
    exe = _build(tmp_path, tsan=True)
    cases = [synth.uniform_costs(200, 0, 10**5, 6), synth.geometric_costs(96, 2),
             np.random.default_rng(3).integers(0, 3, size=(65, 65)).astype(np.int32),
             synth.uniform_costs(1, -5, 5, 4), synth.uniform_costs(2, 0, 9, 5)]
    for C in cases:
        cost, phases, bids, match, prices, lists, full = _run(exe, C, 10, 8, tmp_path, lanes, per_lane)
        _check(C, cost, match, prices)
        assert lists + full == bids


@pytest.mark.parametrize("lanes,per_lane", LIST_SHAPES)
@pytest.mark.parametrize("threads,alpha", [(1, 10), (8, 4), (16, 64)])
def test_lists_keep_every_bid_exact(tmp_path, lanes, per_lane, threads, alpha):
    exe = _build(tmp_path, tsan=False)
    for C in (synth.uniform_costs(200, 0, 10**5, 6), synth.geometric_costs(256, 7),
              synth.uniform_costs(64, 0, 1000, 8)):
        cost, phases, bids, match, prices, lists, full = _run(exe, C, alpha, threads, tmp_path, lanes, per_lane)
        _check(C, cost, match, prices)
        assert lists + full == bids


def test_lists_answer_most_bids(tmp_path):
    """With the GPU's 32 x 4 lists on rows wider than 128 columns, most bids
    are decided by the list alone (the test is not vacuous)."""
    exe = _build(tmp_path, tsan=False)
    for C in (synth.uniform_costs(200, 0, 10**5, 6), synth.geometric_costs(256, 7)):
        cost, phases, bids, match, prices, lists, full = _run(exe, C, 10, 1, tmp_path, 32, 4)
        _check(C, cost, match, prices)
        assert lists > 3 * full


@pytest.mark.parametrize("mutant", [1, 2])
def test_a_broken_list_rule_is_seen(tmp_path, mutant):
    """Mistakes planted in the list rule: 1 ignores the price shift between
    phases, 2 takes the largest per-class bound instead of the least. One
    thread makes the runs deterministic; each mutant must give a result that
    is not the exact optimum on at least one of these, while the correct
    rule is exact on all of them."""
    good = _build(tmp_path, tsan=False)
    bad = _build(tmp_path, tsan=False, mutant=mutant)
    seen = 0
    for C in (synth.uniform_costs(200, 0, 10**5, 6), synth.geometric_costs(256, 7),
              synth.uniform_costs(64, 0, 1000, 8)):
        for lanes, per_lane in ((4, 2), (8, 1)):
            r = _run(good, C, 10, 1, tmp_path, lanes, per_lane)
            assert _exact(C, r[0], r[3], r[4])
            r = _run(bad, C, 10, 1, tmp_path, lanes, per_lane)
            seen += not _exact(C, r[0], r[3], r[4])
    assert seen > 0


def test_price_bounds_hold_under_concurrency(tmp_path):
    """The emulation stops with status 3 if a committed price passes
    S + 2 C~ + 2 eps within a phase or the spread passes C~ + eps after it;
    many small instances, thread counts and alphas must all finish cleanly."""
    exe = _build(tmp_path, tsan=False)
    rng = np.random.default_rng(9)
    for t in range(40):
        n = int(rng.integers(1, 41))
        kind = t % 3
        if kind == 0:
            C = synth.uniform_costs(n, 0, int(rng.choice([1, 3, 100, 10**4])), t)
        elif kind == 1:
            C = synth.geometric_costs(max(n, 2), t)
        else:
            C = rng.integers(-5, 5, size=(n, n)).astype(np.int32)
        for threads, alpha, lanes, per_lane in ((4, 2, 0, 0), (32, 10, 0, 0), (16, 64, 4, 1)):
            cost, *_ = _run(exe, C, alpha, threads, tmp_path, lanes, per_lane)
            assert cost == oracle.hungarian(C)[0]


def _sequential_peaks(C, alpha, rng):
    """Plain sequential double pushes with the free row drawn at random.
    Returns, over the phases, the largest q / (S + 2 C~ + 2 eps) and the
    largest spread / (C~ + eps)."""
    n = C.shape[0]
    cmin = int(C.min())
    Ct = (n + 1) * (int(C.max()) - cmin)
    cs = (C.astype(np.int64) - cmin) * (n + 1)
    q = [0] * n
    e = Ct
    in_phase = after = 0.0
    while True:
        e = max(1, e // alpha)
        m = min(q)
        q = [v - m for v in q]
        S = max(q)
        holder = [-1] * n
        free = list(range(n))
        peak = S
        while free:
            x = free.pop(rng.randrange(len(free)))
            b1 = b2 = w = None
            for y in range(n):
                v = int(cs[x, y]) + q[y]
                if b1 is None or v < b1:
                    b2, b1, w = b1, v, y
                elif b2 is None or v < b2:
                    b2 = v
            if b2 is None:
                b2 = b1
            q[w] += (b2 - b1) + e
            peak = max(peak, q[w])
            if holder[w] >= 0:
                free.append(holder[w])
            holder[w] = x
        in_phase = max(in_phase, peak / (S + 2 * Ct + 2 * e))
        after = max(after, (max(q) - min(q)) / (Ct + e))
        if e == 1:
            return in_phase, after


def test_price_bounds_are_reached():
    """The two bounds hold on sequential schedules too, and are nearly or
    exactly attained: the 32-bit test has no slack to spare."""
    import random
    rng = random.Random(5)
    worst_in = worst_after = 0.0
    for t in range(60):
        n = rng.randint(1, 16)
        if t % 3 == 0:
            C = synth.uniform_costs(n, 0, rng.choice([1, 3, 100]), t)
        elif t % 3 == 1:
            C = synth.geometric_costs(max(n, 2), t)
        else:
            C = np.random.default_rng(t).integers(-5, 5, size=(n, n)).astype(np.int32)
        for alpha in (2, 4, 10):
            a, b = _sequential_peaks(C, alpha, random.Random(31 * t + alpha))
            assert a <= 1.0 and b <= 1.0, (t, alpha, a, b)
            worst_in, worst_after = max(worst_in, a), max(worst_after, b)
    assert worst_in > 0.9 and worst_after == 1.0, (worst_in, worst_after)


@pytest.mark.parametrize("lanes,per_lane", [(0, 0), (32, 4), (4, 2)])
def test_price_mirror_is_race_free_and_exact(tmp_path, lanes, per_lane):
    """Scans read prices from a mirror raised by an atomic maximum after each
    commit attempt, so it can lag the key: stale prices are lower, and a bid
    made from them still keeps its row eps-optimal."""
    tsan = _build(tmp_path, tsan=True)
    for C in (synth.uniform_costs(120, 0, 10**5, 6), synth.geometric_costs(96, 2),
              np.random.default_rng(3).integers(0, 3, size=(65, 65)).astype(np.int32),
              synth.uniform_costs(1, -5, 5, 4), synth.uniform_costs(2, 0, 9, 5)):
        cost, phases, bids, match, prices, lists, full = _run(tsan, C, 10, 8, tmp_path, lanes, per_lane, 1)
        _check(C, cost, match, prices)
    plain = _build(tmp_path, tsan=False)
    for threads, alpha in ((1, 10), (16, 4), (32, 64)):
        for C in (synth.uniform_costs(200, 0, 10**5, 6), synth.geometric_costs(256, 7)):
            cost, phases, bids, match, prices, lists, full = _run(plain, C, alpha, threads, tmp_path,
                                                                  lanes, per_lane, 1)
            _check(C, cost, match, prices)


def test_deeper_lists_halve_the_full_scans(tmp_path):
    """Why 4 entries per lane: each doubling of the entries a lane keeps
    about halves the share of bids that must scan the full row (the bound
    theta rises to a higher order statistic of the lane's values). One
    thread makes the counts deterministic."""
    exe = _build(tmp_path, tsan=False)
    C = synth.uniform_costs(1024, 0, (1 << 20) - 1, 1)
    share = []
    for per_lane in (2, 4, 8):
        cost, phases, bids, match, prices, lists, full = _run(exe, C, 10, 1, tmp_path, 32, per_lane)
        _check(C, cost, match, prices)
        share.append(full / (lists + full))
    assert share[0] > 0.3
    assert share[1] < 0.6 * share[0] and share[2] < 0.6 * share[1], share
