"""Autotuners: alpha for single solves, and the shape of batched solves.

``autotune_alpha`` times single solves of sample matrices for a few alphas
(the divisor of eps between refine phases, Algorithm 5.0; the paper uses
10) and keeps the fastest. Any alpha gives the same exact optimum; a larger
one runs fewer phases, and on large instances each phase's end (its last
displacement chains) costs more than the extra bidding inside a phase.

``autotune_batched`` picks, by measurement on the caller's own batch (or a
sample of it):

* alpha per size bucket (bucket k holds 2^k <= n < 2^(k+1)). alpha is the
  divisor of eps between refine phases (Algorithm 5.0; the paper uses 10):
  a larger alpha means fewer phases with more bidding each.
* the CTA shape: its size (warps that bid concurrently) and how many
  instances it keeps resident (slots); its warps take free rows from any
  resident instance.
* the shared-memory key capacity ``max_n`` (the largest n in the batch), which
  sets how many CTAs fit on an SM.

Every candidate is timed with CUDA events through ``la_solve_batched_ex``
(the same kernel the tuned call runs). The result is a small JSON table that
``options_from_table`` turns back into ``la_batch_options``.
"""

from __future__ import annotations

import json

import paper_1110_6231_gb300 as la

DEFAULT_ALPHAS = (4, 6, 8, 10, 16)
DEFAULT_SHAPES = ((256, 2), (512, 2), (512, 4), (1024, 8))   # (threads per CTA, resident instances)


DEFAULT_SINGLE_ALPHAS = (8, 10, 16, 24, 32, 48, 64)

# One alpha for a batch of same-size instances that fills the GPU: its time
# follows the total bidding more than the end of each phase, so larger
# alphas than a single solve's stay in the running.
DEFAULT_BATCH_ALPHAS = (32, 64, 128, 256, 1024)


def autotune_alpha(samples, *, alphas=DEFAULT_SINGLE_ALPHAS, reps: int = 3) -> dict:
    """Fastest alpha for ``la.solve`` on the square int32 CUDA matrices in
    ``samples`` (mean wall time over ``reps`` solves of each, after one
    untimed solve). Returns ``{"alpha": best, "mean_ms": {alpha: ms}}``."""
    import time

    import torch
    mean = {}
    for a in alphas:
        for C in samples:
            la.solve(C, alpha=int(a))
        total = 0.0
        for C in samples:
            for _ in range(reps):
                torch.cuda.synchronize(C.device)
                t0 = time.perf_counter()
                la.solve(C, alpha=int(a))
                torch.cuda.synchronize(C.device)
                total += time.perf_counter() - t0
        mean[int(a)] = 1e3 * total / (reps * len(samples))
    return {"alpha": min(mean, key=mean.get), "mean_ms": mean}


def autotune_batch_alpha(costs, offsets, ns, *, alphas=DEFAULT_BATCH_ALPHAS, reps: int = 1,
                         **options) -> dict:
    """Fastest single alpha for one batch (CUDA tensors: int32 costs, int64
    offsets, int32 ns), every other option fixed by ``options`` (keywords of
    ``la.batch_options``). A candidate under which any instance reports a
    nonzero status is not eligible. Returns ``{"alpha": best, "device_ms":
    {alpha: ms}}``."""
    import torch
    B = int(ns.numel())
    total = int(ns.sum().item())
    match = torch.empty(max(1, total), dtype=torch.int32, device=costs.device)
    out = torch.empty(max(1, B), dtype=torch.int64, device=costs.device)
    status = torch.empty(max(1, B), dtype=torch.int32, device=costs.device)
    ms = {}
    for a in alphas:
        opt = la.batch_options(alpha=int(a), no_graph=True, profile=True, **options)
        best = None
        for _ in range(reps):
            st = la.la_batch_stats()
            rc = la.la_solve_batched_ex(costs, offsets, ns, B, opt, None, match, out, status, st)
            if rc != la.LA_OK:
                raise la.LaError(rc, "autotune_batch_alpha")
            if int((status[:B] != 0).sum().item()):
                best = None
                break
            best = st.device_ms if best is None else min(best, st.device_ms)
        if best is not None:
            ms[int(a)] = best
    if not ms:
        raise la.LaError(la.LA_ERR_ITER_LIMIT, "autotune_batch_alpha: no alpha solved every instance")
    return {"alpha": min(ms, key=ms.get), "device_ms": ms}


def _bucket(n: int) -> int:
    return min(la.LA_ALPHA_BUCKETS - 1, max(0, int(n).bit_length() - 1))


def _time(costs, offsets, ns, opt, reps):
    import torch
    B = int(ns.numel())
    total = int(ns.sum().item())
    match = torch.empty(max(1, total), dtype=torch.int32, device=costs.device)
    out = torch.empty(max(1, B), dtype=torch.int64, device=costs.device)
    best = None
    for _ in range(reps):
        st = la.la_batch_stats()
        rc = la.la_solve_batched_ex(costs, offsets, ns, B, opt, None, match, out, None, st)
        if rc != la.LA_OK:
            raise la.LaError(rc, "autotune")
        best = st.device_ms if best is None else min(best, st.device_ms)
    return best


def autotune_batched(costs, offsets, ns, *, alphas=DEFAULT_ALPHAS, shapes=DEFAULT_SHAPES,
                     per_bucket: int = 0, reps: int = 2, seed: int = 0) -> dict:
    """Tune on CUDA tensors (int32 costs, int64 offsets, int32 ns).

    Each bucket's alpha is timed on that bucket's instances (all of them, or
    a sample of ``per_bucket`` when it is > 0): a bucket's sub-batch must be
    large enough to fill the GPU for its timing to reflect throughput. The
    CTA shape is then timed on the union of the samples with the tuned alphas.
    """
    import numpy as np
    import torch

    ns_h = ns.cpu().numpy()
    off_h = offsets.cpu().numpy()
    max_n = int(ns_h.max()) if ns_h.size else 1
    rng = np.random.default_rng(seed)
    buckets = {}
    for i, n in enumerate(ns_h):
        buckets.setdefault(_bucket(int(n)), []).append(i)
    alpha_tab = [0] * la.LA_ALPHA_BUCKETS
    timings = {"alpha": {}, "block": {}}
    sample_all = []
    for b, idx in sorted(buckets.items()):
        idx = np.array(idx)
        if per_bucket > 0 and idx.size > per_bucket:
            idx = np.sort(rng.choice(idx, per_bucket, replace=False))
        sample_all.extend(idx.tolist())
        sub_off = torch.from_numpy(off_h[idx]).to(costs.device)
        sub_ns = torch.from_numpy(ns_h[idx]).to(costs.device)
        res = {}
        for a in alphas:
            opt = la.batch_options(block_threads=512, slots=4, max_n=max_n, alpha=int(a), no_graph=True,
                                   profile=True)
            res[int(a)] = _time(costs, sub_off, sub_ns, opt, reps)
        alpha_tab[b] = min(res, key=res.get)
        timings["alpha"][b] = res
    idx = np.array(sorted(sample_all))
    sub_off = torch.from_numpy(off_h[idx]).to(costs.device)
    sub_ns = torch.from_numpy(ns_h[idx]).to(costs.device)
    for blk, slots in shapes:
        opt = la.batch_options(block_threads=int(blk), slots=int(slots), max_n=max_n, alpha=alpha_tab,
                               no_graph=True, profile=True)
        timings["block"][(int(blk), int(slots))] = _time(costs, sub_off, sub_ns, opt, reps)
    block, slots = min(timings["block"], key=timings["block"].get)
    return {"block_threads": int(block), "slots": int(slots), "max_n": max_n, "alpha": [int(a) for a in alpha_tab],
            "timings_ms": {"alpha": {str(k): v for k, v in timings["alpha"].items()},
                           "shape": {f"{b}x{s}": v for (b, s), v in timings["block"].items()}}}


def options_from_table(table: dict, **extra) -> "la.la_batch_options":
    return la.batch_options(block_threads=table["block_threads"], slots=table.get("slots", 0),
                            max_n=table["max_n"], alpha=table["alpha"], **extra)


def save_table(path: str, table: dict) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1)


def load_table(path: str) -> dict:
    with open(path) as f:
        return json.load(f)
