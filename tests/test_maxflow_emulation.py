"""The grid max-flow's lock-free push-relabel (Hong's Algorithm 4.5 in cycles
with a global relabel between them, Algorithm 4.8), emulated by host threads
with C11 atomics (tests/maxflow_emulation.c) and run under ThreadSanitizer: no
data race may be reported, every run must end, and the flow must equal the
oracle's (Dinic). Every run also checks the stopping rule's reading: the
flow plus the excess stranded at pixels that cannot reach t is the total
excess, and those pixels (with s) are the source side of a cut whose
capacity is the flow. Nothing here touches a GPU."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1110_6231_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "maxflow_emulation.c")


def _build(tmp_path, tsan):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    plain = str(tmp_path / "memu")
    r = subprocess.run([cc, "-O2", "-std=c11", "-pthread", SRC, "-o", plain], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    if not tsan:
        return plain
    exe = str(tmp_path / "memu_tsan")
    r = subprocess.run([cc, "-O1", "-g", "-fsanitize=thread", "-std=c11", "-pthread", SRC, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:   # the source compiles: only the sanitizer is missing
        pytest.skip("ThreadSanitizer unavailable: " + r.stderr[-200:])
    return exe


def _random_grid(H, W, seed, hi=9):
    rng = np.random.default_rng(seed)
    cap = rng.integers(0, hi + 1, size=(4, H, W)).astype(np.int32)
    cap[0, :, W - 1] = 0
    cap[1, :, 0] = 0
    cap[2, H - 1, :] = 0
    cap[3, 0, :] = 0
    src = (rng.integers(0, 3 * hi, size=(H, W)) * (rng.random((H, W)) < 0.3)).astype(np.int32)
    snk = (rng.integers(0, 3 * hi, size=(H, W)) * (rng.random((H, W)) < 0.3)).astype(np.int32)
    return cap, src, snk


def _run(exe, cap, src, snk, threads, cycle, tmp_path, timeout=300):
    _, H, W = cap.shape
    inp, out = tmp_path / "min.bin", tmp_path / "mout.bin"
    with open(inp, "wb") as f:
        np.array([H, W, threads, cycle], dtype=np.int32).tofile(f)
        np.ascontiguousarray(cap, dtype=np.int32).tofile(f)
        np.ascontiguousarray(src, dtype=np.int32).tofile(f)
        np.ascontiguousarray(snk, dtype=np.int32).tofile(f)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    r = subprocess.run([exe, str(inp), str(out)], capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    raw = open(out, "rb").read()
    flow, rounds, total, stranded = (int(v) for v in np.frombuffer(raw[:32], dtype=np.int64))
    side = np.frombuffer(raw[32:32 + H * W], dtype=np.uint8)
    # the stopping rule's bookkeeping: every unit of excess reached t or is
    # held by a pixel that cannot reach t (a maximum preflow)
    assert flow + stranded == total, (flow, stranded, total)
    # the pixels that cannot reach t, with s, form the source side of a cut
    # whose capacity is the flow: a minimum cut
    nn, tail, head, acap, s, t = oracle.grid_arcs(cap, src, snk)
    full = np.zeros(nn, dtype=np.uint8)
    full[:H * W] = side
    full[s] = 1
    assert oracle.cut_capacity(nn, tail, head, acap, s, t, full) == flow
    return flow, rounds


def _dinic(cap, src, snk):
    return oracle.maxflow_dinic(*oracle.grid_arcs(cap, src, snk))[0]


def test_push_relabel_is_race_free_under_threadsanitizer(tmp_path):
    exe = _build(tmp_path, tsan=True)
    for seed, (H, W) in enumerate(((1, 1), (1, 7), (5, 6), (12, 9))):
        cap, src, snk = _random_grid(H, W, seed)
        for threads, cycle in ((4, 8), (8, 32)):
            flow, _ = _run(exe, cap, src, snk, threads, cycle, tmp_path)
            assert flow == _dinic(cap, src, snk)
    cap, src, snk = synth.grid_crossing(8, 12, 3)
    assert _run(exe, cap, src, snk, 8, 16, tmp_path)[0] == _dinic(cap, src, snk)


@pytest.mark.parametrize("threads,cycle", [(1, 1), (4, 16), (16, 64), (32, 512)])
def test_push_relabel_is_exact_with_many_threads(tmp_path, threads, cycle):
    exe = _build(tmp_path, tsan=False)
    cases = [synth.grid_cut(48, 40, 5), synth.grid_crossing(24, 32, 6), _random_grid(30, 30, 7, hi=50)]
    for cap, src, snk in cases:
        flow, rounds = _run(exe, cap, src, snk, threads, cycle, tmp_path)
        assert flow == _dinic(cap, src, snk)
        assert rounds >= 0
