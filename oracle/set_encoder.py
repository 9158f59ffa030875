"""CPU oracle of the learned price predictor (test infrastructure only).

Plain numpy in float64, written from the predictor's definition. The paper
has no learned component; its only contact with the paper is that any start
prices are admissible (Sect. 5.2, Algorithm 5.2's refine initialisation), so
this oracle pins the network's arithmetic, not a result of the paper.

* ``features(C)``          -- the 8 per-column statistics (padded to 16) and T.
* ``forward(P, X, seg)``   -- the set encoder's outputs y.
* ``loss_grad(P, X, t, seg)`` -- loss L = (1/I) sum_i (1/n_i) sum_j
  (d_j - mean_i d)^2 with d = y - t (the per-instance variance of the
  error, blind to a shift of y or t, as prices are) and dL/dP by
  hand-written backpropagation.
* ``bf16(x)``              -- round to bfloat16 (nearest even), to emulate the
  GPU's tensor-core operands when a tight comparison is wanted.

Pinned in tests by central finite differences of the loss (independent of
the backward code), by the loss's invariance to a per-instance shift of y,
and by hand-checked features of small matrices.
"""

from __future__ import annotations

import numpy as np

F = 16          # padded feature count
NF = 8          # real features
H = 128
HEADER = 16
OFF_W1 = HEADER
OFF_B1 = OFF_W1 + F * H
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + 2 * H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H * 8
NPARAM = OFF_B3 + 8
MAGIC = 4242.0


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return (P[OFF_W1:OFF_B1].reshape(F, H), P[OFF_B1:OFF_W2], P[OFF_W2:OFF_B2].reshape(2 * H, H),
            P[OFF_B2:OFF_W3], P[OFF_W3:OFF_B3].reshape(H, 8), P[OFF_B3:OFF_B3 + 8])


def pack(W1, b1, W2, b2, W3, b3, eps_factor=0.0):
    P = np.zeros(NPARAM, dtype=np.float64)
    P[0], P[1], P[2], P[3], P[4] = MAGIC, 1.0, F, H, eps_factor
    P[OFF_W1:OFF_B1] = np.ravel(W1)
    P[OFF_B1:OFF_W2] = b1
    P[OFF_W2:OFF_B2] = np.ravel(W2)
    P[OFF_B2:OFF_W3] = b2
    P[OFF_W3:OFF_B3] = np.ravel(W3)
    P[OFF_B3:OFF_B3 + 8] = b3
    return P


def bf16(x):
    """Round float values to bfloat16 (round to nearest, ties to even)."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(C):
    """Per-column features of an n x n integer matrix, and T.

    For column j: a = min_i C[i,j], b = second smallest C[i,j] (b = a if
    n = 1); with row minima u_i = min_j C[i,j]: q = min_i (C[i,j] - u_i) and
    its second smallest; cnt = number of rows whose (lowest-index) minimum
    is column j; m = mean_i C[i,j]. T = 1 + mean_j (b - a). Features:
    (a - mean a)/T, (b - a)/T, (q - mean q)/T, (q2 - q)/T, log(1 + cnt),
    (m - mean m)/(std m + 1), log(T)/10, log(n)/10.
    """
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    s = np.sort(C, axis=0)
    a = s[0]
    b = s[1] if n > 1 else s[0]
    u = C.min(axis=1)
    R = np.sort(C - u[:, None], axis=0)
    q = R[0]
    q2 = R[1] if n > 1 else R[0]
    cnt = np.bincount(np.argmin(C, axis=1), minlength=n)
    m = C.mean(axis=0)
    T = 1.0 + np.mean(b - a)
    X = np.zeros((n, F))
    X[:, 0] = (a - a.mean()) / T
    X[:, 1] = (b - a) / T
    X[:, 2] = (q - q.mean()) / T
    X[:, 3] = (q2 - q) / T
    X[:, 4] = np.log1p(cnt)
    X[:, 5] = (m - m.mean()) / (np.sqrt(np.mean((m - m.mean()) ** 2)) + 1.0)
    X[:, 6] = np.log(T) / 10.0
    X[:, 7] = np.log(n) / 10.0
    return X, T


def _q(x, quant):
    return bf16(x) if quant else np.asarray(x, dtype=np.float64)


def forward(P, X, seg, quant=False, cache=False):
    """Outputs y (one per feature row). ``quant`` rounds every matrix
    product's operands to bfloat16, as the GPU's tensor cores see them."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    X = np.asarray(X, dtype=np.float64)
    seg = np.asarray(seg)
    H1 = np.maximum(_q(X, quant) @ _q(W1, quant) + b1, 0.0)
    I = len(seg) - 1
    ctx = np.zeros((I, H))
    rowseg = np.zeros(X.shape[0], dtype=np.int64)
    for i in range(I):
        r0, r1 = seg[i], seg[i + 1]
        rowseg[r0:r1] = i
        if r1 > r0:
            ctx[i] = H1[r0:r1].mean(axis=0)
    Z = np.concatenate([H1, ctx[rowseg]], axis=1)
    H2 = np.maximum(_q(Z, quant) @ _q(W2, quant) + b2, 0.0)
    Y = _q(H2, quant) @ _q(W3, quant) + b3
    y = Y[:, 0]
    if cache:
        return y, dict(X=X, H1=H1, ctx=ctx, Z=Z, H2=H2, rowseg=rowseg)
    return y


def loss(P, X, t, seg, quant=False):
    y = forward(P, X, seg, quant)
    seg = np.asarray(seg)
    I = len(seg) - 1
    L = 0.0
    for i in range(I):
        r0, r1 = seg[i], seg[i + 1]
        if r1 > r0:
            d = y[r0:r1] - t[r0:r1]
            L += np.mean((d - d.mean()) ** 2)
    return L / I


def loss_grad(P, X, t, seg, quant=False):
    """Loss and its gradient with respect to every parameter (header = 0)."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    y, c = forward(P, X, seg, quant, cache=True)
    seg = np.asarray(seg)
    t = np.asarray(t, dtype=np.float64)
    I = len(seg) - 1
    N = X.shape[0]
    dy = np.zeros(N)
    L = 0.0
    for i in range(I):
        r0, r1 = seg[i], seg[i + 1]
        n = r1 - r0
        if n == 0:
            continue
        d = y[r0:r1] - t[r0:r1]
        e = d - d.mean()
        L += np.mean(e * e)
        # d/dy_j of (1/n) sum_k (d_k - mean d)^2 = (2/n) e_j
        dy[r0:r1] = 2.0 * e / (I * n)
    L /= I
    H1, Z, H2, rowseg = c["H1"], c["Z"], c["H2"], c["rowseg"]
    # every matrix product below rounds its operands when ``quant`` is set
    dW3 = np.zeros((H, 8))
    dW3[:, 0] = _q(H2, quant).T @ _q(dy, quant)
    db3 = np.zeros(8)
    db3[0] = dy.sum()
    dH2 = np.outer(dy, W3[:, 0]) * (H2 > 0)
    dW2 = _q(Z, quant).T @ _q(dH2, quant)
    db2 = dH2.sum(axis=0)
    dZ = _q(dH2, quant) @ _q(W2, quant).T
    dH1 = dZ[:, :H].copy()
    for i in range(I):
        r0, r1 = seg[i], seg[i + 1]
        if r1 > r0:
            dH1[r0:r1] += dZ[r0:r1, H:].sum(axis=0) / (r1 - r0)
    dH1 *= (H1 > 0)
    dW1 = _q(c["X"], quant).T @ _q(dH1, quant)
    db1 = dH1.sum(axis=0)
    g = pack(dW1, db1, dW2, db2, dW3, db3)
    g[:HEADER] = 0.0
    return L, g


def init_params(seed=0, eps_factor=0.0):
    """He-style random initial weights."""
    rng = np.random.default_rng(seed)
    W1 = np.zeros((F, H))
    W1[:NF] = rng.normal(0.0, np.sqrt(2.0 / NF), size=(NF, H))
    W2 = rng.normal(0.0, np.sqrt(2.0 / (2 * H)), size=(2 * H, H))
    W3 = np.zeros((H, 8))
    W3[:, 0] = rng.normal(0.0, np.sqrt(1.0 / H), size=H)
    return pack(W1, np.zeros(H), W2, np.full(H, 0.01), W3, np.zeros(8), eps_factor)
