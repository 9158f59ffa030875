"""CPU oracle for the assignment problem and maximum flow (test
infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
import this package. It shares no code with the CUDA path in
``paper_1110_6231_gb300``; the two meet only in the seeded inputs of
``paper_1110_6231_gb300.synth``.

The arithmetic lives in ``oracle.c`` (plain C, exact int64); this module
builds it with gcc on first use and marshals numpy arrays. Functions:

* ``brute_force(C)``      -- min over all n! permutations (n <= 10).
* ``hungarian(C)``        -- shortest-augmenting-path Hungarian method with
  integer duals ``u, v`` (Kuhn 1955 / Munkres 1957; not from the paper).
* ``cost_scaling_arcfix(C, ...)`` -- the same with the arc fixing of Sect.
  5.2 (arcs whose reduced cost exceeds 2 n eps after a phase are deleted).
* ``cost_scaling(C, ...)`` -- the paper's sequential cost scaling: Algorithm
  5.0's epsilon loop, Algorithm 5.2's refine initialisation and Algorithm 5.4's
  push/relabel taken as the Goldberg-Kennedy double push, on costs scaled by
  n + 1.
* ``check_matching``, ``check_duals``, ``check_eps_cs`` -- certificates.
* ``certify_optimal(C, match)`` -- optimality of any claimed matching with no
  duals given (Klein's negative-cycle criterion by Bellman-Ford), at any n.
* ``sparse_brute_force``, ``sparse_ssp`` and ``sparse_check_*`` -- the same
  problem on a sparse bipartite graph given by its arcs in CSR form
  (``row_ptr, cols, costs``); ``INFEASIBLE`` when it has no perfect matching.
* ``min_cut_brute``, ``maxflow_dinic``, ``cut_capacity`` -- maximum s-t flow
  (the paper's Sect. 4 problem) on a directed graph given by its arcs, and
  ``grid_arcs`` for the 4-connected grid graphs with terminal arcs.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, INVARIANT, OVERFLOW, NOMEM, INFEASIBLE = 0, 1, 2, 3, 4, 5


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.or_brute_force.argtypes = [P, i32, P, P]
            lib.or_hungarian.argtypes = [P, i32, P, P, P, P]
            lib.or_cost_scaling.argtypes = [P, i32, i32, i64, P, i64, i32, P, P, P, P]
            lib.or_cost_scaling_arcfix.argtypes = [P, i32, i32, i64, P, P, P, P, P, P]
            lib.or_check_matching.argtypes = [P, i32, P, i64]
            lib.or_check_duals.argtypes = [P, i32, P, P, P]
            lib.or_check_eps_cs.argtypes = [P, i32, P, P, i64]
            lib.or_certify_optimal.argtypes = [P, i32, P, P, P]
            lib.or_sparse_brute_force.argtypes = [i32, P, P, P, P, P]
            lib.or_sparse_ssp.argtypes = [i32, P, P, P, P, P, P, P]
            lib.or_sparse_check_matching.argtypes = [i32, P, P, P, P, i64]
            lib.or_sparse_check_duals.argtypes = [i32, P, P, P, P, P, P]
            lib.or_sparse_check_eps_cs.argtypes = [i32, P, P, P, P, P, i64]
            lib.or_min_cut_brute.argtypes = [i32, i32, P, P, P, i32, i32, P, P]
            lib.or_maxflow_dinic.argtypes = [i32, i32, P, P, P, i32, i32, P, P]
            lib.or_cut_capacity.argtypes = [i32, i32, P, P, P, i32, i32, P, P]
            for f in (lib.or_brute_force, lib.or_hungarian, lib.or_cost_scaling,
                      lib.or_check_matching, lib.or_check_duals, lib.or_check_eps_cs,
                      lib.or_certify_optimal,
                      lib.or_sparse_brute_force, lib.or_sparse_ssp, lib.or_sparse_check_matching,
                      lib.or_sparse_check_duals, lib.or_sparse_check_eps_cs,
                      lib.or_min_cut_brute, lib.or_maxflow_dinic, lib.or_cut_capacity):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _costs(C) -> np.ndarray:
    C = np.ascontiguousarray(C, dtype=np.int32)
    if C.ndim != 2 or C.shape[0] != C.shape[1]:
        raise ValueError("cost matrix must be square")
    return C


def brute_force(C):
    """Exact optimum by enumeration. Returns ``(cost, match)``."""
    C = _costs(C)
    n = C.shape[0]
    match = np.zeros(n, dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    rc = _load().or_brute_force(_ptr(C), n, _ptr(match), _ptr(cost))
    if rc:
        raise OracleError(f"or_brute_force returned {rc}")
    return int(cost[0]), match


def hungarian(C):
    """Exact optimum with integer duals. Returns ``(cost, match, u, v)``."""
    C = _costs(C)
    n = C.shape[0]
    match = np.zeros(n, dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    u = np.zeros(n, dtype=np.int64)
    v = np.zeros(n, dtype=np.int64)
    rc = _load().or_hungarian(_ptr(C), n, _ptr(match), _ptr(cost), _ptr(u), _ptr(v))
    if rc:
        raise OracleError(f"or_hungarian returned {rc}")
    return int(cost[0]), match, u, v


def cost_scaling(C, alpha: int = 10, eps0: int = 0, init_prices=None,
                 final_eps: int = 1, check: bool = False):
    """Sequential cost scaling. Returns ``(cost, match, prices, stats)``.

    ``prices`` are the final column prices in the paper's sign, on costs
    scaled by n + 1; ``stats`` is a dict with ``phases``, ``scans``
    (row scans = double pushes), ``displaced`` and ``eps_first``.
    """
    C = _costs(C)
    n = C.shape[0]
    match = np.zeros(n, dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    prices = np.zeros(n, dtype=np.int64)
    stats = np.zeros(4, dtype=np.int64)
    ip = None if init_prices is None else np.ascontiguousarray(init_prices, dtype=np.int64)
    rc = _load().or_cost_scaling(_ptr(C), n, int(alpha), int(eps0), _ptr(ip),
                                 int(final_eps), int(bool(check)), _ptr(match),
                                 _ptr(cost), _ptr(prices), _ptr(stats))
    if rc:
        raise OracleError(f"or_cost_scaling returned {rc}")
    st = dict(phases=int(stats[0]), scans=int(stats[1]), displaced=int(stats[2]),
              eps_first=int(stats[3]))
    return int(cost[0]), match, prices, st


def cost_scaling_arcfix(C, alpha: int = 10, eps0: int = 0, init_prices=None):
    """Sequential cost scaling with the arc fixing of Sect. 5.2: after every
    phase but the last, arcs with reduced cost above 2 n eps are deleted.
    Returns ``(cost, match, prices, fixed, stats)``; ``fixed`` is an n x n
    bool array of the deleted arcs, ``stats`` adds ``deleted`` to the keys of
    ``cost_scaling``'s."""
    C = _costs(C)
    n = C.shape[0]
    match = np.zeros(n, dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    prices = np.zeros(n, dtype=np.int64)
    fixed = np.zeros((n, n), dtype=np.uint8)
    stats = np.zeros(5, dtype=np.int64)
    ip = None if init_prices is None else np.ascontiguousarray(init_prices, dtype=np.int64)
    rc = _load().or_cost_scaling_arcfix(_ptr(C), n, int(alpha), int(eps0), _ptr(ip), _ptr(match),
                                        _ptr(cost), _ptr(prices), _ptr(fixed), _ptr(stats))
    if rc:
        raise OracleError(f"or_cost_scaling_arcfix returned {rc}")
    st = dict(phases=int(stats[0]), scans=int(stats[1]), displaced=int(stats[2]),
              eps_first=int(stats[3]), deleted=int(stats[4]))
    return int(cost[0]), match, prices, fixed.astype(bool), st


def check_matching(C, match, claimed_cost) -> int:
    C = _costs(C)
    m = np.ascontiguousarray(match, dtype=np.int32)
    return _load().or_check_matching(_ptr(C), C.shape[0], _ptr(m), int(claimed_cost))


def check_duals(C, match, u, v) -> int:
    C = _costs(C)
    m = np.ascontiguousarray(match, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    return _load().or_check_duals(_ptr(C), C.shape[0], _ptr(m), _ptr(u), _ptr(v))


def check_eps_cs(C, match, prices, eps: int = 1) -> int:
    C = _costs(C)
    m = np.ascontiguousarray(match, dtype=np.int32)
    p = np.ascontiguousarray(prices, dtype=np.int64)
    return _load().or_check_eps_cs(_ptr(C), C.shape[0], _ptr(m), _ptr(p), int(eps))


def certify_optimal(C, match):
    """Optimality of a perfect matching by the negative-cycle criterion
    (Bellman-Ford on the alternating-cycle graph over the columns). Returns
    ``(rc, u, v)``: rc 0 = optimal, with exact LP duals ``u, v`` tight on the
    matching; 10 = not a permutation; 16 = a cheaper matching exists."""
    C = _costs(C)
    n = C.shape[0]
    m = np.ascontiguousarray(match, dtype=np.int32)
    if m.shape != (n,):
        raise ValueError("match must hold one column per row")
    u = np.zeros(n, dtype=np.int64)
    v = np.zeros(n, dtype=np.int64)
    rc = _load().or_certify_optimal(_ptr(C), n, _ptr(m), _ptr(u), _ptr(v))
    return rc, u, v


def eps_schedule(Ct: int, alpha: int = 10, eps0: int = 0, final_eps: int = 1):
    """The epsilon of every refine phase: eps <- max(1, eps // alpha), starting
    from eps0 (default C~), until the phase run at eps <= final_eps."""
    eps = eps0 if eps0 > 0 else Ct
    out = []
    while True:
        eps = max(1, eps // alpha)
        out.append(eps)
        if eps <= final_eps:
            return out


# ---------------------------------------------------------------- sparse graphs

class Infeasible(OracleError):
    """The graph has no perfect matching."""


def _csr(row_ptr, cols, costs):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    costs = np.ascontiguousarray(costs, dtype=np.int32)
    if row_ptr.ndim != 1 or row_ptr.size < 1 or cols.shape != costs.shape:
        raise ValueError("bad CSR arrays")
    return row_ptr.size - 1, row_ptr, cols, costs


def sparse_brute_force(row_ptr, cols, costs):
    """Min over permutations made of arcs (n <= 10). Returns ``(cost, match)``;
    raises ``Infeasible`` when there is none."""
    n, rp, cc, cs = _csr(row_ptr, cols, costs)
    match = np.zeros(max(n, 1), dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    rc = _load().or_sparse_brute_force(n, _ptr(rp), _ptr(cc), _ptr(cs), _ptr(match), _ptr(cost))
    if rc == INFEASIBLE:
        raise Infeasible("no perfect matching")
    if rc:
        raise OracleError(f"or_sparse_brute_force returned {rc}")
    return int(cost[0]), match[:n]


def sparse_ssp(row_ptr, cols, costs):
    """Successive shortest paths with integer duals. Returns
    ``(cost, match, u, v)``; raises ``Infeasible`` when the graph has no
    perfect matching."""
    n, rp, cc, cs = _csr(row_ptr, cols, costs)
    match = np.zeros(max(n, 1), dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    u = np.zeros(max(n, 1), dtype=np.int64)
    v = np.zeros(max(n, 1), dtype=np.int64)
    rc = _load().or_sparse_ssp(n, _ptr(rp), _ptr(cc), _ptr(cs), _ptr(match), _ptr(cost), _ptr(u), _ptr(v))
    if rc == INFEASIBLE:
        raise Infeasible("no perfect matching")
    if rc:
        raise OracleError(f"or_sparse_ssp returned {rc}")
    return int(cost[0]), match[:n], u[:n], v[:n]


def sparse_check_matching(row_ptr, cols, costs, match, claimed_cost) -> int:
    n, rp, cc, cs = _csr(row_ptr, cols, costs)
    m = np.ascontiguousarray(match, dtype=np.int32)
    return _load().or_sparse_check_matching(n, _ptr(rp), _ptr(cc), _ptr(cs), _ptr(m), int(claimed_cost))


def sparse_check_duals(row_ptr, cols, costs, match, u, v) -> int:
    n, rp, cc, cs = _csr(row_ptr, cols, costs)
    m = np.ascontiguousarray(match, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    return _load().or_sparse_check_duals(n, _ptr(rp), _ptr(cc), _ptr(cs), _ptr(m), _ptr(u), _ptr(v))


def sparse_check_eps_cs(row_ptr, cols, costs, match, prices, eps: int = 1) -> int:
    n, rp, cc, cs = _csr(row_ptr, cols, costs)
    m = np.ascontiguousarray(match, dtype=np.int32)
    p = np.ascontiguousarray(prices, dtype=np.int64)
    return _load().or_sparse_check_eps_cs(n, _ptr(rp), _ptr(cc), _ptr(cs), _ptr(m), _ptr(p), int(eps))


# ---------------------------------------------------------------- maximum flow

def _arcs(tail, head, cap):
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    cap = np.ascontiguousarray(cap, dtype=np.int64)
    if not (tail.shape == head.shape == cap.shape) or tail.ndim != 1:
        raise ValueError("tail, head and cap must be 1-D arrays of one length")
    return tail, head, cap


def min_cut_brute(nn, tail, head, cap, s, t):
    """Minimum s-t cut by enumeration (nn <= 20). Returns ``(value, side)``."""
    tail, head, cap = _arcs(tail, head, cap)
    value = np.zeros(1, dtype=np.int64)
    side = np.zeros(nn, dtype=np.uint8)
    rc = _load().or_min_cut_brute(int(nn), tail.size, _ptr(tail), _ptr(head), _ptr(cap), int(s), int(t),
                                  _ptr(value), _ptr(side))
    if rc:
        raise OracleError(f"or_min_cut_brute returned {rc}")
    return int(value[0]), side


def maxflow_dinic(nn, tail, head, cap, s, t):
    """Maximum flow value and the source side of a minimum cut (Dinic)."""
    tail, head, cap = _arcs(tail, head, cap)
    value = np.zeros(1, dtype=np.int64)
    side = np.zeros(nn, dtype=np.uint8)
    rc = _load().or_maxflow_dinic(int(nn), tail.size, _ptr(tail), _ptr(head), _ptr(cap), int(s), int(t),
                                  _ptr(value), _ptr(side))
    if rc:
        raise OracleError(f"or_maxflow_dinic returned {rc}")
    return int(value[0]), side


def cut_capacity(nn, tail, head, cap, s, t, side) -> int:
    tail, head, cap = _arcs(tail, head, cap)
    side = np.ascontiguousarray(side, dtype=np.uint8)
    value = np.zeros(1, dtype=np.int64)
    rc = _load().or_cut_capacity(int(nn), tail.size, _ptr(tail), _ptr(head), _ptr(cap), int(s), int(t),
                                 _ptr(side), _ptr(value))
    if rc:
        raise OracleError(f"or_cut_capacity returned {rc}")
    return int(value[0])


def grid_arcs(cap, src, snk):
    """Arcs of a 4-connected H x W grid graph with terminals: node i*W + j is
    pixel (i, j), s = H*W, t = H*W + 1. ``cap[d][i][j]`` is the capacity of
    the arc from (i, j) to its neighbour in direction d (0: (i, j+1),
    1: (i, j-1), 2: (i+1, j), 3: (i-1, j)); ``src`` / ``snk`` the capacities
    s -> (i, j) and (i, j) -> t. Returns ``(nn, tail, head, cap, s, t)``."""
    cap = np.asarray(cap, dtype=np.int64)
    src = np.asarray(src, dtype=np.int64)
    snk = np.asarray(snk, dtype=np.int64)
    _, H, W = cap.shape
    N = H * W
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    u = (ii * W + jj).ravel()
    tails, heads, caps = [], [], []
    for d, (di, dj) in enumerate(((0, 1), (0, -1), (1, 0), (-1, 0))):
        ni, nj = (ii + di).ravel(), (jj + dj).ravel()
        ok = (ni >= 0) & (ni < H) & (nj >= 0) & (nj < W)
        tails.append(u[ok])
        heads.append((ni * W + nj)[ok])
        caps.append(cap[d].ravel()[ok])
    tails += [np.full(N, N), u]
    heads += [u, np.full(N, N + 1)]
    caps += [src.ravel(), snk.ravel()]
    return N + 2, np.concatenate(tails), np.concatenate(heads), np.concatenate(caps), N, N + 1
