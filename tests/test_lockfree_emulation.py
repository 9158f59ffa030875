"""The lock-free bidding protocol of the parallel refine, emulated by host
threads with C11 atomics (tests/lockfree_emulation.c) and run under
ThreadSanitizer: no data race may be reported, every run must end, and the
result must be the exact optimum (the oracle's Hungarian cost, a permutation
of that cost, and eps-CS at eps = 1 with the final prices). The same holds
with candidate lists, whose bound must stay sound across the price shifts
between phases; two planted mistakes in the list rule must be seen. Nothing
here touches a GPU."""

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


def _run(exe, C, alpha, threads, tmp_path, lanes=0, per_lane=0, timeout=120):
    """Returns cost, phases, bids, match, prices, list scans, full scans."""
    n = C.shape[0]
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        np.array([n, alpha, threads, lanes, per_lane], dtype=np.int32).tofile(f)
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
