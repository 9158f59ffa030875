"""Training, calibration and evaluation of the learned price predictor.

The training data are geometric (optical-flow-like) instances with n
uniform in [256, 1024], solved exactly by the plain cold-start batched
solver. Optimal duals are not unique (the dual optimum is a polytope, and
where the auction's final prices land in it depends on the bidding order),
so the targets are the canonical duals of ``la_dual_certificate``: the
largest potential v <= 0 tight on the optimal matching. Targets are centred
and in units of the instance scale T: t_j = (v_j - mean v) / T. Features come
from ``la_features``;
every forward, backward and Adam step runs in the library's kernels
(``la_predictor_train_step``). PyTorch only holds device memory.

Calibration: on held-out instances, the 95th percentile over instances of
max_j |(y_j - mean y) - t_j| (in units of T) becomes the header's eps0
factor q, so that a warm solve starts at eps0 = ceil((n+1) T q).

Command line (GPU): ``python -m paper_1110_6231_gb300.learn --out PATH``.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

import numpy as np

import paper_1110_6231_gb300 as la
from paper_1110_6231_gb300 import synth

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(PKG, "weights", "set_encoder_geometric.f32")


def geometric_batch_gpu(sizes, seeds, device):
    """Packed geometric instances: points from ``synth`` (seeded), costs
    rint(1e4 |a_i - b_j|^2) formed on the device."""
    import torch
    mats = []
    for n, s in zip(sizes, seeds):
        a, _, b = synth.geometric_points(int(n), int(s))
        A = torch.from_numpy(a).to(device)
        Bm = torch.from_numpy(b).to(device)
        dx = A[:, 0][:, None] - Bm[:, 0][None, :]
        dy = A[:, 1][:, None] - Bm[:, 1][None, :]
        mats.append(torch.round((dx * dx + dy * dy) * 1.0e4).to(torch.int32).reshape(-1))
    flat = torch.cat(mats)
    ns = torch.tensor(np.asarray(sizes, dtype=np.int32), device=device)
    sq = np.asarray(sizes, dtype=np.int64) ** 2
    off = np.zeros(len(sizes), dtype=np.int64)
    off[1:] = np.cumsum(sq)[:-1]
    return flat, torch.from_numpy(off).to(device), ns


def build_dataset(count, seed0, device, chunk=500, n_lo=256, n_hi=1024, log=print):
    """Features, targets and segment offsets of ``count`` solved instances."""
    import torch
    rng = np.random.default_rng(seed0)
    feats, targets, sizes_all = [], [], []
    t0 = time.time()
    for c0 in range(0, count, chunk):
        m = min(chunk, count - c0)
        sizes = rng.integers(n_lo, n_hi + 1, size=m)
        seeds = seed0 + c0 + np.arange(m)
        flat, off, ns = geometric_batch_gpu(sizes, seeds, device)
        sol = la.solve_batched(flat, off, ns, options=la.batch_options(max_n=n_hi))
        moff = 0
        vbuf = torch.empty(n_hi, dtype=torch.int64, device=device)
        for i in range(m):
            n = int(sizes[i])
            C = flat[int(off[i]):int(off[i]) + n * n]
            f = torch.empty((n, la.LA_PRED_FEATURES_PADDED), dtype=torch.float32, device=device)
            inst = torch.empty(2, dtype=torch.float32, device=device)
            rc = la.la_features(C, n, None, f, inst)
            if rc != la.LA_OK:
                raise la.LaError(rc, "la_features")
            rc = la.la_dual_certificate(C, n, sol.match[moff:moff + n], None, None, vbuf)
            if rc != la.LA_OK:
                raise la.LaError(rc, "la_dual_certificate")
            v = vbuf[:n].double()
            T = float(inst[0].item())
            t = ((v - v.mean()) / T).float()
            feats.append(f)
            targets.append(t)
            moff += n
        sizes_all.append(sizes)
        if log:
            log(f"dataset {c0 + m}/{count} ({time.time() - t0:.1f}s, batch solve rc={sol.stats['rc']})")
    sizes = np.concatenate(sizes_all)
    seg = np.zeros(len(sizes) + 1, dtype=np.int64)
    seg[1:] = np.cumsum(sizes)
    return torch.cat(feats), torch.cat(targets), seg


def init_params(seed=0):
    """He-style random initial weights with the header filled in."""
    rng = np.random.default_rng(seed)
    P = np.zeros(la.LA_PRED_PARAMS, dtype=np.float32)
    F, H, NF = la.LA_PRED_FEATURES_PADDED, la.LA_PRED_WIDTH, la.LA_PRED_FEATURES
    P[:5] = [la.LA_PRED_MAGIC, 1.0, F, H, 0.0]
    o = la.LA_PRED_HEADER
    W1 = np.zeros((F, H), np.float32)
    W1[:NF] = rng.normal(0, np.sqrt(2.0 / NF), (NF, H))
    P[o:o + F * H] = W1.ravel()
    o += F * H + H
    P[o:o + 2 * H * H] = rng.normal(0, np.sqrt(2.0 / (2 * H)), 2 * H * H)
    o += 2 * H * H
    P[o:o + H] = 0.01
    o += H
    W3 = np.zeros((H, 8), np.float32)
    W3[:, 0] = rng.normal(0, np.sqrt(1.0 / H), H)
    P[o:o + H * 8] = W3.ravel()
    return P


def train(feats, targets, seg, *, steps=3000, batch=64, lr=2e-3, seed=0, device="cuda", log=print):
    import torch
    P = torch.from_numpy(init_params(seed)).to(device)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    rng = np.random.default_rng(seed)
    I_total = len(seg) - 1
    history = []
    loss = ctypes.c_float(0.0)
    for step in range(1, steps + 1):
        idx = np.sort(rng.choice(I_total, size=min(batch, I_total), replace=False))
        rows = np.concatenate([np.arange(seg[i], seg[i + 1]) for i in idx])
        sizes = seg[idx + 1] - seg[idx]
        s = np.zeros(len(idx) + 1, dtype=np.int32)
        s[1:] = np.cumsum(sizes)
        r = torch.from_numpy(rows).to(device)
        f = feats.index_select(0, r).contiguous()
        t = targets.index_select(0, r).contiguous()
        sg = torch.from_numpy(s).to(device)
        cur = lr * 0.5 * (1 + np.cos(np.pi * (step - 1) / steps))
        rc = la.la_predictor_train_step(P, m, v, f, t, sg, len(idx), len(rows), step, cur, 0.0, None,
                                        None, ctypes.byref(loss))
        if rc != la.LA_OK:
            raise la.LaError(rc, "la_predictor_train_step")
        history.append(float(loss.value))
        if log and (step % 250 == 0 or step == 1):
            log(f"step {step} loss {np.mean(history[-250:]):.5f} lr {cur:.2e}")
    return P, history


def errors(P, feats, targets, seg, device="cuda"):
    """Per instance: max_j |(y_j - mean y) - t_j| (units of T)."""
    import torch
    N = feats.shape[0]
    y = torch.empty(N, dtype=torch.float32, device=device)
    sg = torch.from_numpy(np.asarray(seg, dtype=np.int32)).to(device)
    rc = la.la_predictor_forward(P, feats, sg, len(seg) - 1, N, None, y)
    if rc != la.LA_OK:
        raise la.LaError(rc, "la_predictor_forward")
    y = y.cpu().numpy().astype(np.float64)
    t = targets.cpu().numpy().astype(np.float64)
    out = []
    for i in range(len(seg) - 1):
        a, b = seg[i], seg[i + 1]
        d = (y[a:b] - y[a:b].mean()) - (t[a:b] - t[a:b].mean())
        out.append(np.abs(d).max())
    return np.array(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--train", type=int, default=50_000)
    ap.add_argument("--holdout", type=int, default=500)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--quantile", type=float, default=95.0)
    args = ap.parse_args()
    import torch
    dev = torch.device("cuda")
    la.lib()
    t0 = time.time()
    feats, targets, seg = build_dataset(args.train, 1_000_000, dev)
    hf, ht, hs = build_dataset(args.holdout, 3_000_000, dev)
    t1 = time.time()
    P, hist = train(feats, targets, seg, steps=args.steps, device=dev)
    t2 = time.time()
    err = errors(P, hf, ht, hs, dev)
    q = float(np.percentile(err, args.quantile))
    P[4] = q
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    P.cpu().numpy().astype(np.float32).tofile(args.out)
    meta = dict(train_instances=args.train, holdout_instances=args.holdout, steps=args.steps,
                final_loss=float(np.mean(hist[-250:])), first_loss=float(hist[0]),
                eps_factor_q=q, holdout_err_median=float(np.median(err)),
                holdout_err_max=float(err.max()), data_s=t1 - t0, train_s=t2 - t1,
                train_seeds="1000000 + i", holdout_seeds="3000000 + i", n_range=[256, 1024])
    with open(args.out + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
