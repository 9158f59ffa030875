"""Seeded synthetic assignment instances.

This module only draws inputs. It holds none of the solver's arithmetic, and
both the CUDA path (through the tests and ``bench.py``) and the CPU oracle
consume the int32 matrices it returns, so the two sides always see the same
bytes.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value ``i`` of a stream is ``mix64(key + (i + 1) * GAMMA)``. Every
transcendental function the generators need (``log``, ``exp``, ``cos``,
``sin``) is evaluated here from its power series with IEEE-754 ``+ - * /``
and ``sqrt`` only, one numpy ufunc per operation (no fused multiply-add), so
the same seed gives the same matrix bit for bit on x86-64 and on AArch64.

Workload shapes follow the paper's problem statement (Sect. 3 and Sect. 5:
complete bipartite graphs ``|X| = |Y| = n`` with integer edge costs) and its
motivating application, optical flow by assignment (Sect. 1):

* ``uniform_costs``   -- i.i.d. integer costs, uniform on ``[lo, hi]``.
* ``geometric_costs`` -- points ``a_i`` uniform in the unit square, targets
  ``b_j = a_{pi(j)} + N(0, sigma^2)`` per coordinate, cost
  ``round_half_even(scale * |a_i - b_j|^2)``.
* ``batch``           -- many independent instances of uneven size,
  ``n = floor(exp(U(ln lo, ln hi)))``, half uniform and half geometric.
* ``sparse_uniform``, ``sparse_geometric`` -- sparse bipartite graphs (the
  paper's implementation takes arbitrary bipartite graphs, Sect. 1 and
  Sect. 6) in CSR form ``(row_ptr, cols, costs)``, each with a planted
  perfect matching: random arcs with uniform costs, and the optical-flow
  points linked to the targets in their 3 x 3 grid neighbourhood.
* ``grid_cut`` -- max-flow instances (the paper's Sect. 4 problem) in the form
  of graph-cut segmentation: a 4-connected H x W grid with source and sink
  arcs, built from a noisy image of bright disks on a dark background;
  ``grid_crossing`` -- the same grid with source arcs on the left column and
  sink arcs on the right one, so that every unit of flow crosses the grid.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "u64_stream",
    "uniform_ints",
    "uniform_doubles",
    "normal_pairs",
    "uniform_costs",
    "uniform_costs_torch",
    "geometric_costs",
    "batch_sizes",
    "batch",
    "instance",
    "sparse_uniform",
    "sparse_geometric",
    "sparse_instance",
    "grid_cut",
    "grid_crossing",
    "GRID_WORKLOADS",
    "grid_instance",
    "WORKLOADS",
    "SPARSE_WORKLOADS",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags keep the draws of one instance independent of each other
_TAG_UNIFORM = 1
_TAG_POINTS = 2
_TAG_PERM = 3
_TAG_JITTER = 4
_TAG_SIZES = 5
_TAG_ARCS = 6
_TAG_ARC_COSTS = 7
_TAG_BLOBS = 8
_TAG_PIXEL_NOISE = 9


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64_stream(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` 64-bit words of stream ``(seed, tag)``, from index ``start``."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed * 0x100 + tag) & 0xFFFFFFFFFFFFFFFF],
                              dtype=np.uint64) * _GAMMA)[0]
        ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GAMMA)


def uniform_ints(seed: int, tag: int, count: int, lo: int, hi: int,
                 start: int = 0) -> np.ndarray:
    """Integers uniform on ``[lo, hi]`` (inclusive) by multiply-shift.

    The range ``hi - lo + 1`` must be at most ``2**32``; the bias of the
    multiply-shift map is below ``range / 2**32``.
    """
    r = hi - lo + 1
    if not (1 <= r <= 1 << 32):
        raise ValueError("range must be in [1, 2**32]")
    z = u64_stream(seed, tag, count, start) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return (np.int64(lo) + ((z * np.uint64(r)) >> np.uint64(32)).astype(np.int64))


def _i64(v: int) -> int:
    """The int64 with the bit pattern of the 64-bit word ``v``."""
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _t_srl(x, k: int):
    """Logical right shift of an int64 tensor (``>>`` is arithmetic)."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _t_mix64(z):
    z = (z ^ _t_srl(z, 30)) * _i64(int(_M1))
    z = (z ^ _t_srl(z, 27)) * _i64(int(_M2))
    return z ^ _t_srl(z, 31)


def uniform_costs_torch(n: int, lo: int, hi: int, seed: int, device="cpu"):
    """``uniform_costs(n, lo, hi, seed)`` drawn with torch on ``device``: the
    same SplitMix64 stream and multiply-shift map in int64 arithmetic (which
    wraps modulo 2^64 like the uint64 one), so the int32 result is equal bit
    for bit. Many large instances can be drawn on the GPU in milliseconds."""
    import torch
    r = hi - lo + 1
    if n < 0 or not (1 <= r <= 1 << 32) or not (-(1 << 31) <= lo <= hi < (1 << 31)):
        raise ValueError("bad size or range")
    with np.errstate(over="ignore"):
        key = int(_mix64(np.array([(seed * 0x100 + _TAG_UNIFORM) & 0xFFFFFFFFFFFFFFFF],
                                  dtype=np.uint64) * _GAMMA)[0])
    ctr = torch.arange(1, n * n + 1, dtype=torch.int64, device=device)
    z = _t_mix64(ctr * _i64(int(_GAMMA)) + _i64(key))
    z = _t_srl(z, 32)
    v = _t_srl(z * r, 32) + lo
    return v.to(torch.int32).view(n, n)


def uniform_doubles(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles uniform on ``[0, 1)`` with 53 random bits."""
    z = u64_stream(seed, tag, count, start) >> np.uint64(11)
    return z.astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------- elementary
# functions from their series, so that results do not depend on the libm or
# on numpy's SIMD kernels of the machine.

_LN2 = 0.6931471805599453
_TWO_PI = 6.283185307179586
_SQRT_HALF = 0.7071067811865476


def _ln(x: np.ndarray) -> np.ndarray:
    """Natural log for x > 0: x = m 2^e, ln m = 2 artanh((m-1)/(m+1))."""
    m, e = np.frexp(x)
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    acc = np.full_like(s, 1.0 / 29.0)
    for k in range(13, -1, -1):
        acc = acc * s2
        acc = acc + (1.0 / (2 * k + 1))
    return e * _LN2 + 2.0 * (s * acc)


def _exp(x: np.ndarray) -> np.ndarray:
    """exp(x) = 2^k exp(r), r = x - k ln 2, |r| <= ln2 / 2."""
    k = np.rint(x * (1.0 / _LN2))
    r = x - k * _LN2
    acc = np.full_like(r, 1.0 / math.factorial(22))
    for j in range(21, -1, -1):
        acc = acc * r
        acc = acc + (1.0 / math.factorial(j))
    return np.ldexp(acc, k.astype(np.int32))


def _cos_sin_turns(t: np.ndarray):
    """cos and sin of 2 pi t for t in [0, 1), reduced to |angle| <= pi / 4."""
    q = np.rint(t * 4.0)
    f = t - q * 0.25                       # exact
    a = f * _TWO_PI
    a2 = a * a
    c = np.full_like(a, 1.0 / math.factorial(20))
    for j in range(18, -1, -2):
        c = c * a2
        c = c + ((-1.0) ** (j // 2)) / math.factorial(j)
    s = np.full_like(a, -1.0 / math.factorial(19))
    for j in range(17, 0, -2):
        s = s * a2
        s = s + ((-1.0) ** ((j - 1) // 2)) / math.factorial(j)
    s = s * a
    quad = (q.astype(np.int64)) & 3
    cos = np.select([quad == 0, quad == 1, quad == 2], [c, -s, -c], s)
    sin = np.select([quad == 0, quad == 1, quad == 2], [s, c, -s], -c)
    return cos, sin


def normal_pairs(seed: int, tag: int, count: int):
    """``2 * count`` standard normal deviates by the Box-Muller transform
    (Box and Muller, Ann. Math. Stat. 29, 1958), returned as two arrays."""
    u = uniform_doubles(seed, tag, 2 * count)
    u1 = 1.0 - u[0::2]                     # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * _ln(u1))
    c, s = _cos_sin_turns(u2)
    return r * c, r * s


# ---------------------------------------------------------------- workloads

def uniform_costs(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n x n int32 costs, i.i.d. uniform on ``[lo, hi]``, row-major."""
    if n < 0:
        raise ValueError("n must be >= 0")
    if not (-(1 << 31) <= lo <= hi < (1 << 31)):
        raise ValueError("costs must fit int32")
    v = uniform_ints(seed, _TAG_UNIFORM, n * n, lo, hi)
    return v.astype(np.int32).reshape(n, n)


def _permutation(n: int, seed: int) -> np.ndarray:
    keys = u64_stream(seed, _TAG_PERM, n)
    return np.argsort(keys, kind="stable").astype(np.int64)


def geometric_points(n: int, seed: int, sigma: float = 0.01):
    """Source points ``a`` (n x 2), permutation ``pi`` and targets ``b``."""
    a = uniform_doubles(seed, _TAG_POINTS, 2 * n).reshape(n, 2)
    pi = _permutation(n, seed)
    zx, zy = normal_pairs(seed, _TAG_JITTER, n)
    b = np.empty_like(a)
    b[:, 0] = a[pi, 0] + sigma * zx
    b[:, 1] = a[pi, 1] + sigma * zy
    return a, pi, b


def geometric_costs(n: int, seed: int, sigma: float = 0.01,
                    scale: float = 1.0e4, block: int = 1024) -> np.ndarray:
    """Optical-flow-like n x n int32 costs: ``rint(scale * |a_i - b_j|^2)``."""
    if n < 0:
        raise ValueError("n must be >= 0")
    a, _, b = geometric_points(n, seed, sigma)
    out = np.empty((n, n), dtype=np.int32)
    bx = b[:, 0][None, :]
    by = b[:, 1][None, :]
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        dx = a[r0:r1, 0][:, None] - bx
        dy = a[r0:r1, 1][:, None] - by
        d2 = dx * dx + dy * dy
        out[r0:r1] = np.rint(d2 * scale).astype(np.int32)
    return out


def batch_sizes(count: int, seed: int, lo: int = 16, hi: int = 1024) -> np.ndarray:
    """``n = floor(exp(U(ln lo, ln hi)))`` clamped to ``[lo, hi]``."""
    u = uniform_doubles(seed, _TAG_SIZES, count)
    llo, lhi = _ln(np.array([float(lo)]))[0], _ln(np.array([float(hi)]))[0]
    n = np.floor(_exp(llo + u * (lhi - llo))).astype(np.int64)
    return np.clip(n, lo, hi).astype(np.int32)


def batch(count: int, seed: int, lo: int = 16, hi: int = 1024,
          cost_hi: int = 10_000):
    """``count`` independent instances packed back to back.

    Even-numbered instances are uniform on ``[0, cost_hi]``; odd-numbered ones
    are geometric. Instance ``i`` draws from seed ``seed * 1_000_003 + i``.
    Returns ``(costs_flat int32, offsets int64, ns int32)`` where instance
    ``i`` is ``costs_flat[offsets[i] : offsets[i] + ns[i]**2]`` (row-major).
    """
    ns = batch_sizes(count, seed, lo, hi)
    sizes = ns.astype(np.int64) ** 2
    offsets = np.zeros(count, dtype=np.int64)
    if count > 1:
        offsets[1:] = np.cumsum(sizes)[:-1]
    flat = np.empty(int(sizes.sum()), dtype=np.int32)
    for i in range(count):
        s = seed * 1_000_003 + i
        n = int(ns[i])
        c = uniform_costs(n, 0, cost_hi, s) if i % 2 == 0 else geometric_costs(n, s)
        flat[offsets[i]:offsets[i] + n * n] = c.ravel()
    return flat, offsets, ns


# Named workloads: the sizes, cost ranges and structure of the dense
# assignment instances this library is measured on.
WORKLOADS = {
    "uniform-n256-c1000": dict(kind="uniform", n=256, lo=0, hi=1000),
    "uniform-n4096-c2^20": dict(kind="uniform", n=4096, lo=0, hi=(1 << 20) - 1),
    "geometric-n8192": dict(kind="geometric", n=8192),
}


def instance(name: str, seed: int, n: int | None = None) -> np.ndarray:
    """One instance of a named workload (optionally at another size ``n``)."""
    w = WORKLOADS[name]
    nn = w["n"] if n is None else n
    if w["kind"] == "uniform":
        return uniform_costs(nn, w["lo"], w["hi"], seed)
    return geometric_costs(nn, seed)


# ---------------------------------------------------------------- sparse graphs

def _csr_from_pairs(n: int, rows: np.ndarray, cols: np.ndarray):
    """Sorted, duplicate-free arcs (row-major order) and their row offsets."""
    key = np.unique(rows.astype(np.int64) * n + cols.astype(np.int64))
    r = (key // n).astype(np.int64)
    c = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    if row_ptr[-1] >= (1 << 31):
        raise ValueError("too many arcs for int32 offsets")
    return row_ptr.astype(np.int32), c, r


def sparse_uniform(n: int, degree: int, seed: int, lo: int = 0, hi: int = 10_000):
    """Row x has arcs to ``degree`` uniform random columns and to its planted
    partner ``pi(x)`` (duplicates merged), costs uniform on ``[lo, hi]``.
    Returns ``(row_ptr, cols, costs)`` (int32)."""
    if n < 0 or degree < 0:
        raise ValueError("n and degree must be >= 0")
    pi = _permutation(n, seed)
    rnd = uniform_ints(seed, _TAG_ARCS, n * degree, 0, max(n - 1, 0)) if n else np.zeros(0, np.int64)
    rows = np.concatenate([np.arange(n, dtype=np.int64), np.repeat(np.arange(n, dtype=np.int64), degree)])
    cols = np.concatenate([pi, rnd.astype(np.int64)])
    row_ptr, c, _ = _csr_from_pairs(n, rows, cols)
    costs = uniform_ints(seed, _TAG_ARC_COSTS, c.size, lo, hi).astype(np.int32)
    return row_ptr, c, costs


def sparse_geometric(n: int, seed: int, sigma: float = 0.01, scale: float = 1.0e3):
    """Optical-flow-like sparse graph: the points of ``geometric_points`` on
    a G x G grid (G = floor(sqrt(n / 4)), about four targets per cell); row
    i has arcs to every target b_j in the 3 x 3 cells around a_i, and to its
    true partner (the j with pi(j) = i), at cost
    ``rint(scale * (G |a_i - b_j|)^2)`` (distances in units of a cell).
    Returns ``(row_ptr, cols, costs)`` (int32)."""
    if n < 0:
        raise ValueError("n must be >= 0")
    a, pi, b = geometric_points(n, seed, sigma)
    G = max(1, math.isqrt(n // 4))

    def cell(p):
        q = np.floor(np.clip(p, 0.0, 1.0) * G).astype(np.int64)
        return np.minimum(q, G - 1)

    bcx, bcy = cell(b[:, 0]), cell(b[:, 1])
    bcell = bcy * G + bcx
    order = np.argsort(bcell, kind="stable")
    counts = np.bincount(bcell, minlength=G * G)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    acx, acy = cell(a[:, 0]), cell(a[:, 1])
    rows_l, cols_l = [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            nx, ny = acx + dx, acy + dy
            ok = (nx >= 0) & (nx < G) & (ny >= 0) & (ny < G)
            rr = np.nonzero(ok)[0]
            cc = (ny[rr] * G + nx[rr])
            k = counts[cc]
            rep = np.repeat(rr, k)
            first = np.repeat(starts[cc], k)
            within = np.arange(rep.size) - np.repeat(np.cumsum(k) - k, k)
            rows_l.append(rep)
            cols_l.append(order[first + within])
    inv = np.empty(n, dtype=np.int64)
    inv[pi] = np.arange(n, dtype=np.int64)
    rows_l.append(np.arange(n, dtype=np.int64))
    cols_l.append(inv)
    row_ptr, c, r = _csr_from_pairs(n, np.concatenate(rows_l), np.concatenate(cols_l))
    dx = (a[r, 0] - b[c, 0]) * G
    dy = (a[r, 1] - b[c, 1]) * G
    costs = np.rint((dx * dx + dy * dy) * scale).astype(np.int32)
    return row_ptr, c, costs


# Named sparse workloads (n, kind, degree).
SPARSE_WORKLOADS = {
    "sparse-uniform-n65536-d32": dict(kind="uniform", n=65536, degree=32),
    "sparse-geometric-n65536": dict(kind="geometric", n=65536),
}


def sparse_instance(name: str, seed: int, n: int | None = None):
    w = SPARSE_WORKLOADS[name]
    n = w["n"] if n is None else n
    if w["kind"] == "uniform":
        return sparse_uniform(n, w["degree"], seed)
    return sparse_geometric(n, seed)


# ---------------------------------------------------------------- grid max-flow

def grid_cut(H: int, W: int, seed: int, disks: int = 12, sigma_noise: float = 0.12,
             data_scale: float = 1000.0, smooth: float = 300.0, sigma_edge: float = 0.1):
    """A graph-cut segmentation instance on an H x W 4-connected grid.

    The image: intensity 0.2, and 0.8 inside ``disks`` disks (centres uniform,
    radii uniform in [0.03, 0.15] min(H, W)), plus N(0, sigma_noise^2) noise.
    Data terms: s -> (i, j) costs ``rint(data_scale (I - 0.2)^2)`` (taking the
    pixel to the background side cuts it) and (i, j) -> t costs
    ``rint(data_scale (I - 0.8)^2)``. Smoothness: the arc to each neighbour
    costs ``rint(smooth exp(-(I_u - I_v)^2 / (2 sigma_edge^2)))`` both ways;
    arcs that would leave the grid are 0.

    Returns ``(cap, src, snk)``: int32 arrays [4][H][W], [H][W], [H][W], with
    directions 0: (i, j+1), 1: (i, j-1), 2: (i+1, j), 3: (i-1, j).
    """
    if H < 1 or W < 1:
        raise ValueError("H and W must be >= 1")
    d = uniform_doubles(seed, _TAG_BLOBS, 3 * disks).reshape(disks, 3)
    side = float(min(H, W))
    cy, cx = d[:, 0] * H, d[:, 1] * W
    r = (0.03 + 0.12 * d[:, 2]) * side
    ii = np.arange(H, dtype=np.float64)[:, None] + 0.5
    jj = np.arange(W, dtype=np.float64)[None, :] + 0.5
    inside = np.zeros((H, W), dtype=bool)
    for k in range(disks):
        dy = ii - cy[k]
        dx = jj - cx[k]
        inside |= dy * dy + dx * dx <= r[k] * r[k]
    zx, _ = normal_pairs(seed, _TAG_PIXEL_NOISE, H * W)
    img = np.where(inside, 0.8, 0.2) + sigma_noise * zx.reshape(H, W)
    src = np.rint(data_scale * (img - 0.2) * (img - 0.2)).astype(np.int32)
    snk = np.rint(data_scale * (img - 0.8) * (img - 0.8)).astype(np.int32)
    cap = np.zeros((4, H, W), dtype=np.int32)
    inv = -1.0 / (2.0 * sigma_edge * sigma_edge)
    if W > 1:
        dh = img[:, 1:] - img[:, :-1]
        w = np.rint(smooth * _exp(dh * dh * inv)).astype(np.int32)
        cap[0, :, :-1] = w
        cap[1, :, 1:] = w
    if H > 1:
        dv = img[1:, :] - img[:-1, :]
        w = np.rint(smooth * _exp(dv * dv * inv)).astype(np.int32)
        cap[2, :-1, :] = w
        cap[3, 1:, :] = w
    return cap, src, snk


_TAG_GRID_CAPS = 10


def grid_crossing(H: int, W: int, seed: int, hi: int = 100):
    """A max-flow instance whose flow must cross the grid: source arcs only
    into column 0 and sink arcs only out of column W - 1 (capacity 100 hi
    each), neighbour arcs with independent capacities uniform on [1, hi].
    Augmenting paths are at least W - 1 arcs long. Returns ``(cap, src, snk)``
    as ``grid_cut`` does."""
    if H < 1 or W < 1:
        raise ValueError("H and W must be >= 1")
    cap = uniform_ints(seed, _TAG_GRID_CAPS, 4 * H * W, 1, hi).astype(np.int32).reshape(4, H, W)
    cap[0, :, -1] = 0
    cap[1, :, 0] = 0
    cap[2, -1, :] = 0
    cap[3, 0, :] = 0
    src = np.zeros((H, W), dtype=np.int32)
    snk = np.zeros((H, W), dtype=np.int32)
    src[:, 0] = 100 * hi
    snk[:, -1] = 100 * hi
    return cap, src, snk


GRID_WORKLOADS = {
    "gridcut-1024x1024": dict(kind="cut", H=1024, W=1024),
    "gridcut-256x256": dict(kind="cut", H=256, W=256),
    "gridcross-512x512": dict(kind="cross", H=512, W=512),
}


def grid_instance(name: str, seed: int):
    w = GRID_WORKLOADS[name]
    if w["kind"] == "cross":
        return grid_crossing(w["H"], w["W"], seed)
    return grid_cut(w["H"], w["W"], seed)
