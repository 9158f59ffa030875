"""The batched solver's slot protocol (resident instances, claim words,
phase transitions, the shared instance queue), emulated by host threads with
C11 atomics (tests/batched_emulation.c) and run under ThreadSanitizer: no data
race may be reported, every run must end, and every instance's cost must be
the oracle's optimum with a matching of that cost. Every phase of every slot
also checks the price bounds behind the GPU's 32-bit keys (the emulation
exits with status 3 if one breaks). Nothing here touches a GPU."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "batched_emulation.c")


def _build(tmp_path, tsan):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    plain = str(tmp_path / "bemu")
    r = subprocess.run([cc, "-O2", "-std=c11", "-pthread", SRC, "-o", plain], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    if not tsan:
        return plain
    exe = str(tmp_path / "bemu_tsan")
    r = subprocess.run([cc, "-O1", "-g", "-fsanitize=thread", "-std=c11", "-pthread", SRC, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:   # the source compiles: only the sanitizer is missing
        pytest.skip("ThreadSanitizer unavailable: " + r.stderr[-200:])
    return exe


def _batch(sizes, seed):
    rng = np.random.default_rng(seed)
    inst = []
    for i, n in enumerate(sizes):
        if i % 3 == 0:
            inst.append(synth.uniform_costs(n, -50, 1000, seed * 100 + i))
        elif i % 3 == 1:
            inst.append(synth.geometric_costs(n, seed * 100 + i))
        else:
            inst.append(rng.integers(0, 3, size=(n, n)).astype(np.int32))   # heavy ties
    return inst


def _run(exe, inst, slots, threads, alpha, tmp_path, timeout=300):
    inp, out = tmp_path / "bin.bin", tmp_path / "bout.bin"
    with open(inp, "wb") as f:
        np.array([len(inst), slots, threads, alpha], dtype=np.int32).tofile(f)
        np.array([c.shape[0] for c in inst], dtype=np.int32).tofile(f)
        for c in inst:
            np.ascontiguousarray(c, dtype=np.int32).tofile(f)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    r = subprocess.run([exe, str(inp), str(out)], capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    raw = open(out, "rb").read()
    B = len(inst)
    costs = np.frombuffer(raw[:8 * B], dtype=np.int64)
    matches, pos = [], 8 * B
    for c in inst:
        n = c.shape[0]
        matches.append(np.frombuffer(raw[pos:pos + 4 * n], dtype=np.int32))
        pos += 4 * n
    return costs, matches


def _check(inst, costs, matches):
    for c, cost, m in zip(inst, costs, matches):
        ref = oracle.hungarian(c)[0]
        assert int(cost) == ref
        assert oracle.check_matching(c, m, ref) == 0


def test_slot_protocol_is_race_free_under_threadsanitizer(tmp_path):
    exe = _build(tmp_path, tsan=True)
    inst = _batch([1, 2, 3, 5, 8, 17, 20, 33, 40, 24, 13, 1], 1)
    for slots, threads in ((1, 4), (3, 8)):
        costs, matches = _run(exe, inst, slots, threads, 10, tmp_path)
        _check(inst, costs, matches)


@pytest.mark.parametrize("slots,threads,alpha", [(1, 1, 10), (2, 4, 4), (4, 16, 10), (8, 32, 16)])
def test_slot_protocol_is_exact_with_many_warps(tmp_path, slots, threads, alpha):
    exe = _build(tmp_path, tsan=False)
    inst = _batch([200, 129, 100, 64, 50, 33, 32, 17, 8, 5, 3, 2, 1, 150, 90, 40], 2)
    costs, matches = _run(exe, inst, slots, threads, alpha, tmp_path)
    _check(inst, costs, matches)
