"""The hand-off protocol at the end of a refine phase (grid refine -> team
refine -> tail kernel: the hand-off word, the parked rows, the item claims,
the queue set up by the team refine's last thread), emulated by host threads
with C11 atomics (tests/team_emulation.c) and run under ThreadSanitizer: no
data race may be reported, every run must end, every phase must end with a
complete eps-optimal assignment (the emulation exits with status 3
otherwise), and the final cost must be the oracle's optimum with a matching
of that cost. Nothing here touches a GPU."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "team_emulation.c")


def _build(tmp_path, tsan):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    plain = str(tmp_path / "temu")
    r = subprocess.run([cc, "-O2", "-std=c11", "-pthread", SRC, "-o", plain], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    if not tsan:
        return plain
    exe = str(tmp_path / "temu_tsan")
    r = subprocess.run([cc, "-O1", "-g", "-fsanitize=thread", "-std=c11", "-pthread", SRC, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:   # the source compiles: only the sanitizer is missing
        pytest.skip("ThreadSanitizer unavailable: " + r.stderr[-200:])
    return exe


def _run(exe, C, alpha, refine, team, tail, team_T, tail_T, tmp_path, timeout=300):
    inp, out = tmp_path / "tin.bin", tmp_path / "tout.bin"
    n = C.shape[0]
    with open(inp, "wb") as f:
        np.array([n, alpha, refine, team, tail, team_T, tail_T], dtype=np.int32).tofile(f)
        np.ascontiguousarray(C, dtype=np.int32).tofile(f)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    r = subprocess.run([exe, str(inp), str(out)], capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    raw = open(out, "rb").read()
    cost = int(np.frombuffer(raw[:8], dtype=np.int64)[0])
    team_phases, tail_phases = (int(v) for v in np.frombuffer(raw[8:16], dtype=np.int32))
    match = np.frombuffer(raw[16:16 + 4 * n], dtype=np.int32)
    return cost, match, team_phases, tail_phases


def _instances(n, seed):
    return (synth.uniform_costs(n, -50, 1000, seed), synth.geometric_costs(n, seed + 1),
            np.random.default_rng(seed + 2).integers(0, 3, size=(n, n)).astype(np.int32))


def test_hand_off_protocol_is_race_free_under_threadsanitizer(tmp_path):
    exe = _build(tmp_path, tsan=True)
    team = tail = 0
    for C in _instances(40, 1):
        n = C.shape[0]
        cost, match, tp, lp = _run(exe, C, 4, 4, 3, 2, n // 2, n // 8, tmp_path)
        ref = oracle.hungarian(C)[0]
        assert cost == ref and oracle.check_matching(C, match, ref) == 0
        team += tp
        tail += lp
    assert team > 0 and tail > 0


@pytest.mark.parametrize("refine,team,tail,team_T,tail_T", [
    (8, 4, 2, 60, 8),     # every stage
    (1, 1, 1, 60, 8),     # one thread each
    (16, 8, 4, 10**6, 30),  # the team refine from the first match
    (8, 8, 1, 60, 0),     # no tail: the team refine ends every phase
    (8, 1, 1, 0, 0),      # no team refine: the grid refine ends every phase
])
def test_hand_off_protocol_is_exact(tmp_path, refine, team, tail, team_T, tail_T):
    exe = _build(tmp_path, tsan=False)
    for C in _instances(150, 7) + (synth.uniform_costs(97, 0, 10**5, 9),):
        for alpha in (4, 10):
            cost, match, tp, lp = _run(exe, C, alpha, refine, team, tail, team_T, tail_T, tmp_path)
            ref = oracle.hungarian(C)[0]
            assert cost == ref and oracle.check_matching(C, match, ref) == 0
            if team_T == 0:
                assert tp == 0 and lp == 0
            if tail_T == 0:
                assert lp == 0
