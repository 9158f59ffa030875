"""The GPU's global price update (Sect. 5.2, Algorithm 5.3) against the
oracle's Dial-bucket restatement, label by label, on frozen mid-phase
states.

The states come from the oracle's sequential cost scaling stopped after a
random number of bids inside a random phase (``oracle.price_update``): every
matched row is eps-optimal and some rows are free. ``la_debug_price_update``
runs one update on such a state, with either kernel the refine can use:
the grid update (``k_pu``) or the one-CTA update the tail kernel runs with
``LA_FLAG_TAIL_PRICE_UPDATE`` (labels in shared memory). For
n <= 128 a row's candidate list holds every column, so the GPU's labels
must equal the oracle's exactly and its new prices must be the given ones
less eps times the labels. For larger n the lists hold part of each row and
a matched row's label is capped by the bound on its unlisted columns: the
labels may then only be lower than the exact ones, and the new prices must
still keep every matched row eps-optimal over every arc.
"""

import random

import numpy as np
import pytest

from oracle import price_update as pu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def la():
    import torch
    from paper_1110_6231_gb300 import build
    build.build()
    import paper_1110_6231_gb300 as la
    assert torch.cuda.is_available()
    return la


def _gpu_update(la, C, state, kernel):
    import torch
    cs, q, holder, free, e = state
    n = C.shape[0]
    row_match = np.full(n, -1, np.int32)
    for y, x in enumerate(holder):
        if x >= 0:
            row_match[x] = y
    prices = -np.array(q, dtype=np.int64)          # the paper's sign: p = -q
    dev = "cuda"
    tC = torch.from_numpy(np.ascontiguousarray(C, dtype=np.int32)).to(dev)
    tp = torch.from_numpy(prices).to(dev)
    tm = torch.from_numpy(row_match).to(dev)
    lab = torch.full((n,), -1, dtype=torch.int32, device=dev)
    pout = torch.zeros(n, dtype=torch.int64, device=dev)
    rc = la.la_debug_price_update(tC, n, tp, tm, e, None, lab, pout, kernel)
    torch.cuda.synchronize()
    assert rc == la.LA_OK, la.la_status_string(rc)
    return lab.cpu().numpy().astype(np.int64), pout.cpu().numpy(), prices


def _states(count, seed, nmin, nmax):
    rng = random.Random(seed)
    out = []
    t = 0
    while len(out) < count:
        n = rng.randint(nmin, nmax)
        hi = (20, 3, 1000, 10**5)[t % 4]
        C = np.random.default_rng(seed * 7919 + t).integers(0, hi, size=(n, n)).astype(np.int32)
        t += 1
        st = pu.mid_phase_state(C.tolist(), rng.choice([2, 4, 10]), rng)
        # the kernel caps the truncation level at 2048 (it keeps the price
        # spread near its usual bound); states whose labels go beyond are
        # not comparable label by label
        if st is not None and st[3] and max(pu.dial_labels(*st)) <= 2048:
            out.append((C, st))
    return out


KERNELS = pytest.mark.parametrize("kernel", [0, 1], ids=["grid", "one_cta"])


@KERNELS
def test_labels_equal_the_dial_buckets_when_every_column_is_listed(la, kernel):
    moved = 0
    for C, st in _states(40, 1, 5, 128):
        cs, q, holder, free, e = st
        want = pu.dial_labels(cs, q, holder, free, e)
        lab, pout, p = _gpu_update(la, C, st, kernel)
        assert list(lab) == want
        assert np.array_equal(pout, p - e * lab)
        assert pu.eps_optimal(cs, pu.apply(q, want, e), holder, e)
        moved += int(lab.any())
    assert moved >= 10        # the update moves prices in many of these states


@KERNELS
def test_capped_labels_on_partial_lists_keep_eps_optimality(la, kernel):
    for C, st in _states(3, 2, 150, 200):
        cs, q, holder, free, e = st
        want = pu.dial_labels(cs, q, holder, free, e)
        lab, pout, p = _gpu_update(la, C, st, kernel)
        assert (lab >= 0).all() and (lab <= np.array(want)).all()
        q2 = list(-pout + int(pout.max()))
        assert pu.eps_optimal(cs, q2, holder, e)


def test_invalid_state_is_rejected(la):
    import torch
    n = 6
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    p = torch.zeros(n, dtype=torch.int64, device="cuda")
    m = torch.tensor([0, 0, -1, -1, -1, -1], dtype=torch.int32, device="cuda")   # column 0 twice
    lab = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    for kernel in (0, 1):
        assert la.la_debug_price_update(C, n, p, m, 1, None, lab, out, kernel) == la.LA_ERR_INVALID
    m = torch.tensor([0, 1, -1, -1, -1, -1], dtype=torch.int32, device="cuda")
    assert la.la_debug_price_update(C, n, p, m, 1, None, lab, out, 2) == la.LA_ERR_INVALID   # no such kernel


def test_both_kernels_give_the_same_labels_on_partial_lists(la):
    for C, st in _states(3, 3, 300, 400):
        lab0, pout0, _ = _gpu_update(la, C, st, 0)
        lab1, pout1, _ = _gpu_update(la, C, st, 1)
        assert np.array_equal(lab0, lab1) and np.array_equal(pout0, pout1)
