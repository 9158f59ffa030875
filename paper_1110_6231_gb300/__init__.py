"""GB300 dense assignment solver: Python binding of ``libla.so``.

The binding only marshals arguments: tensors become raw device pointers,
the current torch stream becomes the ``cudaStream_t``, and every step of the
solve runs in the library's CUDA kernels. There is no CPU fallback: if
``libla.so`` has not been built (``__graft_entry__.build()`` or
``python -m paper_1110_6231_gb300.build``), every call raises.

Low-level functions keep the C names and argument order of ``include/la.h``
(``la_solve``, ``la_solve_ex``, ``la_status_string``, ...). ``solve`` is the
convenience wrapper most callers want.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libla.so")

LA_OK = 0
LA_ERR_INVALID = 1
LA_ERR_CUDA = 2
LA_ERR_OVERFLOW = 3
LA_ERR_ITER_LIMIT = 4
LA_ERR_NOMEM = 5
LA_ERR_INTERNAL = 6
LA_ERR_TOO_LARGE = 7
LA_ERR_INFEASIBLE = 8
LA_MAX_N = (1 << 20) - 1
LA_NOALLOC_MAX_N = 16384
LA_FLAG_NO_CANDIDATE_LISTS = 1
LA_FLAG_CHECK_PHASES = 2
LA_FLAG_NO_ARC_FIXING = 4
LA_FLAG_NO_SMALL_KERNEL = 8
LA_FLAG_TAIL_PRICE_UPDATE = 16
LA_FLAG_NO_TEAM_REFINE = 32


class la_options(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_int32),
        ("eps0", ctypes.c_int64),
        ("init_prices", ctypes.c_void_p),
        ("prices_out", ctypes.c_void_p),
        ("scan_budget", ctypes.c_int64),
        ("profile", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("tail_threshold", ctypes.c_int32),
        ("price_updates", ctypes.c_int32),
        ("phase_cutoff", ctypes.c_int32),
        ("team_threshold", ctypes.c_int32),
        ("tail_updates", ctypes.c_int32),
        ("alpha_fine", ctypes.c_int32),
    ]


class la_stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("phases", ctypes.c_int64),
        ("scans", ctypes.c_int64),
        ("wins", ctypes.c_int64),
        ("displaced", ctypes.c_int64),
        ("eps_first", ctypes.c_int64),
        ("scaled_range", ctypes.c_int64),
        ("wide", ctypes.c_int32),
        ("vector_loads", ctypes.c_int32),
        ("launches", ctypes.c_int64),
        ("refine_launches", ctypes.c_int64),
        ("refine_ms", ctypes.c_double),
        ("max_chain", ctypes.c_int64),
        ("phase_scans", ctypes.c_int64 * 32),
        ("phase_ms", ctypes.c_double * 32),
        ("full_scans", ctypes.c_int64),
        ("list_scans", ctypes.c_int64),
        ("tail_scans", ctypes.c_int64),
        ("tail_phases", ctypes.c_int32),
        ("price_updates", ctypes.c_int64),
        ("price_update_sweeps", ctypes.c_int64),
        ("price_update_levels", ctypes.c_int64),
        ("list_entries", ctypes.c_int32),
        ("tail_ms", ctypes.c_double),
        ("tail_full_scans", ctypes.c_int64),
        ("tail_giveups", ctypes.c_int32),
        ("checked_phases", ctypes.c_int32),
        ("check_violations", ctypes.c_int64),
        ("stop_phase", ctypes.c_int32),
        ("stop_eps", ctypes.c_int64),
        ("phase_tail_ms", ctypes.c_double * 32),
        ("phase_full_scans", ctypes.c_int64 * 32),
        ("phase_tail_scans", ctypes.c_int64 * 32),
        ("phase_fixed_rows", ctypes.c_int64 * 32),
        ("fixed_rows", ctypes.c_int64),
        ("fixed_arcs", ctypes.c_int64),
        ("sweep_ms", ctypes.c_double),
        ("sweep_scans", ctypes.c_int64),
        ("sweep_full_scans", ctypes.c_int64),
        ("small_kernel", ctypes.c_int32),
        ("tail_price_update_ms", ctypes.c_double),
        ("team_phases", ctypes.c_int32),
        ("team_scans", ctypes.c_int64),
        ("team_full_scans", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if name.startswith("phase_"):
                v = list(v)[: max(0, min(32, int(self.phases)))]
            d[name] = v
        return d


LA_ALPHA_BUCKETS = 16
LA_BATCH_MAX_N = 8192
LA_PRED_FEATURES = 8
LA_PRED_FEATURES_PADDED = 16
LA_PRED_WIDTH = 128
LA_PRED_HEADER = 16
LA_PRED_PARAMS = 36120
LA_PRED_MAGIC = 4242.0


class la_batch_options(ctypes.Structure):
    _fields_ = [
        ("block_threads", ctypes.c_int32),
        ("max_n", ctypes.c_int32),
        ("alpha", ctypes.c_int32 * LA_ALPHA_BUCKETS),
        ("budget_factor", ctypes.c_int32),
        ("no_graph", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("prices_out", ctypes.c_void_p),
        ("slots", ctypes.c_int32),
        ("lists", ctypes.c_int32),
    ]


class la_batch_stats(ctypes.Structure):
    _fields_ = [
        ("instances", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("scans", ctypes.c_int64),
        ("scan_bytes", ctypes.c_int64),
        ("wins", ctypes.c_int64),
        ("displaced", ctypes.c_int64),
        ("phases", ctypes.c_int64),
        ("max_n", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("graph", ctypes.c_int32),
        ("device_ms", ctypes.c_double),
        ("slots", ctypes.c_int32),
        ("lists", ctypes.c_int32),
        ("full_scans", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class la_maxflow_options(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int32), ("max_rounds", ctypes.c_int32)]


class la_maxflow_stats(ctypes.Structure):
    _fields_ = [
        ("flow", ctypes.c_int64),
        ("excess_total", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("global_relabels", ctypes.c_int64),
        ("relabel_sweeps", ctypes.c_int64),
        ("launches", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class LaError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {la_status_string(status)}" if where else la_status_string(status))


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded ``libla.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -m paper_1110_6231_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.la_solve.argtypes = [P, i32, P, P, P]
            L.la_solve_ex.argtypes = [P, i32, P, P, P, P, P]
            L.la_debug_price_update.argtypes = [P, i32, P, P, i64, P, P, P, i32]
            L.la_solve_noalloc.argtypes = [P, i32, P, P, P]
            L.la_solve_sparse.argtypes = [P, P, P, i32, i32, P, P, P]
            L.la_solve_sparse_ex.argtypes = [P, P, P, i32, i32, P, P, P, P, P]
            L.la_maxflow_grid.argtypes = [P, P, P, i32, i32, P, P, P]
            L.la_maxflow_grid_ex.argtypes = [P, P, P, i32, i32, P, P, P, P, P]
            L.la_solve_batched.argtypes = [P, P, P, i32, P, P, P]
            L.la_solve_batched_ex.argtypes = [P, P, P, i32, P, P, P, P, P, P]
            L.la_predictor_param_count.argtypes = []
            L.la_predictor_param_count.restype = i32
            L.la_features.argtypes = [P, i32, P, P, P]
            L.la_predictor_forward.argtypes = [P, P, P, i32, i32, P, P]
            L.la_predictor_train_step.argtypes = [P, P, P, P, P, P, i32, i32, i32, ctypes.c_float,
                                                  ctypes.c_float, P, P, P]
            L.la_predict_prices.argtypes = [P, i32, P, P, P]
            L.la_predict_prices_ex.argtypes = [P, i32, P, P, P, P]
            L.la_solve_warm.argtypes = [P, i32, P, P, P, P, P]
            L.la_dual_certificate.argtypes = [P, i32, P, P, P, P]
            L.la_dual_certificate.restype = ctypes.c_int
            L.la_probe_read.argtypes = [P, ctypes.c_size_t, i32, P, ctypes.POINTER(ctypes.c_float)]
            L.la_probe_read.restype = ctypes.c_int
            for f in (L.la_features, L.la_predictor_forward, L.la_predictor_train_step,
                      L.la_predict_prices, L.la_predict_prices_ex, L.la_solve_warm):
                f.restype = ctypes.c_int
            L.la_status_string.argtypes = [ctypes.c_int]
            L.la_status_string.restype = ctypes.c_char_p
            L.la_release_workspace.argtypes = []
            L.la_version.argtypes = []
            L.la_version.restype = i32
            for f in (L.la_solve, L.la_solve_ex, L.la_solve_noalloc, L.la_release_workspace,
                      L.la_solve_batched, L.la_solve_batched_ex, L.la_solve_sparse, L.la_solve_sparse_ex,
                      L.la_maxflow_grid, L.la_maxflow_grid_ex):
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(x):
    """A device pointer from a tensor, an int address, or None (NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------- C names

def la_solve(cost, n, stream, match_out, cost_out) -> int:
    return lib().la_solve(_ptr(cost), int(n), _stream(stream), _ptr(match_out), _ptr(cost_out))


def la_solve_ex(cost, n, opt, stream, match_out, cost_out, stats_out) -> int:
    return lib().la_solve_ex(_ptr(cost), int(n), None if opt is None else ctypes.byref(opt),
                             _stream(stream), _ptr(match_out), _ptr(cost_out),
                             None if stats_out is None else ctypes.byref(stats_out))


def la_debug_price_update(cost, n, prices, row_match, eps, stream, labels_out, prices_out, kernel=0) -> int:
    return lib().la_debug_price_update(_ptr(cost), int(n), _ptr(prices), _ptr(row_match), int(eps),
                                       _stream(stream), _ptr(labels_out), _ptr(prices_out), int(kernel))


def la_solve_noalloc(cost, n, stream, match_out, cost_out) -> int:
    """la_solve without any allocation: scratch is a fixed device array of the
    library (n <= LA_NOALLOC_MAX_N), for callers that cannot allocate."""
    return lib().la_solve_noalloc(_ptr(cost), int(n), _stream(stream), _ptr(match_out), _ptr(cost_out))


def la_solve_sparse(row_ptr, cols, costs, n, nnz, stream, match_out, cost_out) -> int:
    return lib().la_solve_sparse(_ptr(row_ptr), _ptr(cols), _ptr(costs), int(n), int(nnz), _stream(stream),
                                 _ptr(match_out), _ptr(cost_out))


def la_solve_sparse_ex(row_ptr, cols, costs, n, nnz, opt, stream, match_out, cost_out, stats_out) -> int:
    return lib().la_solve_sparse_ex(_ptr(row_ptr), _ptr(cols), _ptr(costs), int(n), int(nnz),
                                    None if opt is None else ctypes.byref(opt), _stream(stream),
                                    _ptr(match_out), _ptr(cost_out),
                                    None if stats_out is None else ctypes.byref(stats_out))


def la_maxflow_grid(cap, src, snk, H, W, stream, flow_out, cut_out) -> int:
    return lib().la_maxflow_grid(_ptr(cap), _ptr(src), _ptr(snk), int(H), int(W), _stream(stream),
                                 _ptr(flow_out), _ptr(cut_out))


def la_maxflow_grid_ex(cap, src, snk, H, W, opt, stream, flow_out, cut_out, stats_out) -> int:
    return lib().la_maxflow_grid_ex(_ptr(cap), _ptr(src), _ptr(snk), int(H), int(W),
                                    None if opt is None else ctypes.byref(opt), _stream(stream),
                                    _ptr(flow_out), _ptr(cut_out),
                                    None if stats_out is None else ctypes.byref(stats_out))


def la_solve_batched(cost, offsets, ns, B, stream, match_out, cost_out) -> int:
    return lib().la_solve_batched(_ptr(cost), _ptr(offsets), _ptr(ns), int(B), _stream(stream),
                                  _ptr(match_out), _ptr(cost_out))


def la_solve_batched_ex(cost, offsets, ns, B, opt, stream, match_out, cost_out, status_out,
                        stats_out) -> int:
    return lib().la_solve_batched_ex(_ptr(cost), _ptr(offsets), _ptr(ns), int(B),
                                     None if opt is None else ctypes.byref(opt), _stream(stream),
                                     _ptr(match_out), _ptr(cost_out), _ptr(status_out),
                                     None if stats_out is None else ctypes.byref(stats_out))


def la_features(cost, n, stream, feats_out, inst_out) -> int:
    return lib().la_features(_ptr(cost), int(n), _stream(stream), _ptr(feats_out), _ptr(inst_out))


def la_predictor_forward(params, feats, seg, I, N, stream, y_out) -> int:
    return lib().la_predictor_forward(_ptr(params), _ptr(feats), _ptr(seg), int(I), int(N),
                                      _stream(stream), _ptr(y_out))


def la_predictor_train_step(params, adam_m, adam_v, feats, targets, seg, I, N, step, lr,
                            weight_decay, stream, grad_out, loss_out) -> int:
    return lib().la_predictor_train_step(_ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(feats),
                                         _ptr(targets), _ptr(seg), int(I), int(N), int(step),
                                         float(lr), float(weight_decay), _stream(stream),
                                         _ptr(grad_out), loss_out)


def la_predict_prices(cost, n, weights, stream, prices_out) -> int:
    return lib().la_predict_prices(_ptr(cost), int(n), _ptr(weights), _stream(stream), _ptr(prices_out))


def la_predict_prices_ex(cost, n, weights, stream, prices_out, eps0_out) -> int:
    return lib().la_predict_prices_ex(_ptr(cost), int(n), _ptr(weights), _stream(stream),
                                      _ptr(prices_out), eps0_out)


def la_solve_warm(cost, n, weights, stream, match_out, cost_out, stats_out) -> int:
    return lib().la_solve_warm(_ptr(cost), int(n), _ptr(weights), _stream(stream), _ptr(match_out),
                               _ptr(cost_out), None if stats_out is None else ctypes.byref(stats_out))


def la_dual_certificate(cost, n, match, stream, u_out, v_out) -> int:
    return lib().la_dual_certificate(_ptr(cost), int(n), _ptr(match), _stream(stream), _ptr(u_out),
                                     _ptr(v_out))


def dual_certificate(C, match, *, stream=None):
    """Exact integer duals (u, v) (int64 CUDA tensors, cost units) proving
    ``match`` optimal for the int32 CUDA matrix ``C``."""
    import torch
    n = C.shape[0]
    u = torch.empty(max(1, n), dtype=torch.int64, device=C.device)
    v = torch.empty(max(1, n), dtype=torch.int64, device=C.device)
    rc = la_dual_certificate(C.contiguous(), n, match.contiguous(), stream, u, v)
    if rc != LA_OK:
        raise LaError(rc, "la_dual_certificate")
    return u[:n], v[:n]


def la_probe_read(buf, nbytes, reps, stream, ms_out) -> int:
    return lib().la_probe_read(_ptr(buf), int(nbytes), int(reps), _stream(stream), ms_out)


def probe_read_gbps(buf, reps: int, *, stream=None) -> float:
    """Read rate (GB/s) of ``reps`` passes over the CUDA tensor ``buf`` in one
    launch of the library's probe kernel (128-bit loads cached at L2 only):
    the L2 rate when ``buf`` fits in L2, the HBM rate when it is far larger."""
    nbytes = buf.numel() * buf.element_size()
    ms = ctypes.c_float(0.0)
    rc = la_probe_read(buf, nbytes, reps, stream, ctypes.byref(ms))
    if rc != LA_OK:
        raise LaError(rc, "la_probe_read")
    return nbytes * reps / (ms.value * 1e-3) / 1e9


def la_status_string(status: int) -> str:
    return lib().la_status_string(int(status)).decode()


def la_release_workspace() -> int:
    return lib().la_release_workspace()


def la_version() -> int:
    return lib().la_version()


# ------------------------------------------------------------- convenience

@dataclass
class Solution:
    cost: int            # exact optimal total cost
    match: object        # torch.int32 [n] on the device: row x -> column
    stats: dict          # la_stats counters
    prices: object = None  # torch.int64 [n] final column prices (if asked)


def solve(C, *, alpha: int = 0, eps0: int = 0, init_prices=None, want_prices: bool = False,
          scan_budget: int = 0, profile: bool = False, block_threads: int = 0,
          flags: int = 0, tail_threshold: int = 0, price_updates: int = 0, phase_cutoff: int = 0, team_threshold: int = 0,
          tail_updates: int = 0, alpha_fine: int = 0,
          stream=None, check: bool = True) -> Solution:
    """Exact minimum-cost assignment of a square int32 CUDA tensor ``C``.

    ``init_prices`` (int64 CUDA tensor, paper sign, units of (n+1) C) warm
    starts the solve. Raises ``LaError`` on a non-OK status when ``check``.
    """
    import torch
    if C.dim() != 2 or C.shape[0] != C.shape[1]:
        raise ValueError("cost matrix must be square")
    if C.dtype != torch.int32 or not C.is_cuda:
        raise ValueError("cost matrix must be an int32 CUDA tensor")
    C = C.contiguous()
    n = C.shape[0]
    dev = C.device
    match = torch.empty(n, dtype=torch.int32, device=dev)
    cost = torch.empty(1, dtype=torch.int64, device=dev)
    prices = torch.empty(n, dtype=torch.int64, device=dev) if want_prices else None
    opt = la_options()
    opt.alpha = alpha
    opt.eps0 = eps0
    if init_prices is not None:
        if init_prices.dtype != torch.int64 or init_prices.numel() != n or not init_prices.is_cuda:
            raise ValueError("init_prices must be an int64 CUDA tensor of length n")
        init_prices = init_prices.contiguous()
    opt.init_prices = _ptr(init_prices)
    opt.prices_out = _ptr(prices)
    opt.scan_budget = scan_budget
    opt.profile = int(bool(profile))
    opt.block_threads = block_threads
    opt.flags = flags
    opt.tail_threshold = tail_threshold
    opt.price_updates = price_updates
    opt.phase_cutoff = phase_cutoff
    opt.team_threshold = team_threshold
    opt.tail_updates = tail_updates
    opt.alpha_fine = alpha_fine
    st = la_stats()
    with torch.cuda.device(dev):
        rc = la_solve_ex(C, n, opt, stream, match, cost, st)
    if rc != LA_OK and check:
        raise LaError(rc, "la_solve_ex")
    return Solution(cost=int(cost.item()) if rc == LA_OK else None, match=match,
                    stats=dict(st.as_dict(), status=rc), prices=prices)


def solve_sparse(row_ptr, cols, costs, *, alpha: int = 0, eps0: int = 0, want_prices: bool = False,
                 scan_budget: int = 0, profile: bool = False, stream=None, check: bool = True) -> Solution:
    """Exact minimum-cost perfect matching of a sparse bipartite graph given
    by int32 CUDA tensors in CSR form (``row_ptr`` of length n + 1, ``cols``
    and ``costs`` of length nnz). Raises ``LaError`` on a non-OK status when
    ``check`` (``LA_ERR_INFEASIBLE`` when there is no perfect matching)."""
    import torch
    for t in (row_ptr, cols, costs):
        if t.dtype != torch.int32 or not t.is_cuda or t.dim() != 1:
            raise ValueError("row_ptr, cols and costs must be 1-D int32 CUDA tensors")
    if cols.numel() != costs.numel():
        raise ValueError("cols and costs must have the same length")
    row_ptr, cols, costs = row_ptr.contiguous(), cols.contiguous(), costs.contiguous()
    n = row_ptr.numel() - 1
    if n < 0:
        raise ValueError("row_ptr must have n + 1 entries")
    dev = row_ptr.device
    match = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cost = torch.empty(1, dtype=torch.int64, device=dev)
    prices = torch.empty(max(n, 1), dtype=torch.int64, device=dev) if want_prices else None
    opt = la_options()
    opt.alpha = alpha
    opt.eps0 = eps0
    opt.prices_out = _ptr(prices)
    opt.scan_budget = scan_budget
    opt.profile = int(bool(profile))
    st = la_stats()
    with torch.cuda.device(dev):
        rc = la_solve_sparse_ex(row_ptr, cols, costs, n, cols.numel(), opt, stream, match, cost, st)
    if rc != LA_OK and check:
        raise LaError(rc, "la_solve_sparse_ex")
    return Solution(cost=int(cost.item()) if rc == LA_OK else None, match=match[:n],
                    stats=dict(st.as_dict(), status=rc), prices=None if prices is None else prices[:n])


@dataclass
class MaxFlow:
    flow: int          # the maximum flow value
    cut: object        # torch.uint8 [H, W]: 1 = source side of a minimum cut
    stats: dict


def maxflow_grid(cap, src, snk, *, cycle: int = 0, max_rounds: int = 0, stream=None,
                 check: bool = True) -> MaxFlow:
    """Maximum flow and a minimum cut of a 4-connected grid graph given by
    int32 CUDA tensors ``cap`` [4, H, W], ``src`` and ``snk`` [H, W]."""
    import torch
    if cap.dim() != 3 or cap.shape[0] != 4 or tuple(src.shape) != tuple(cap.shape[1:]) \
            or tuple(snk.shape) != tuple(cap.shape[1:]):
        raise ValueError("cap must be [4, H, W], src and snk [H, W]")
    for t in (cap, src, snk):
        if t.dtype != torch.int32 or not t.is_cuda:
            raise ValueError("capacities must be int32 CUDA tensors")
    cap, src, snk = cap.contiguous(), src.contiguous(), snk.contiguous()
    H, W = int(cap.shape[1]), int(cap.shape[2])
    flow = torch.empty(1, dtype=torch.int64, device=cap.device)
    cut = torch.empty((H, W), dtype=torch.uint8, device=cap.device)
    opt = la_maxflow_options()
    opt.cycle = cycle
    opt.max_rounds = max_rounds
    st = la_maxflow_stats()
    with torch.cuda.device(cap.device):
        rc = la_maxflow_grid_ex(cap, src, snk, H, W, opt, stream, flow, cut, st)
    if rc != LA_OK and check:
        raise LaError(rc, "la_maxflow_grid_ex")
    return MaxFlow(flow=int(flow.item()) if rc == LA_OK else None, cut=cut, stats=dict(st.as_dict(), status=rc))


@dataclass
class BatchSolution:
    costs: object      # torch.int64 [B] exact optimal cost per instance
    match: object      # torch.int32 [sum n] packed matchings (instance i at prefix sum of n)
    status: object     # torch.int32 [B] la_status per instance
    stats: dict


def batch_options(block_threads: int = 0, max_n: int = 0, alpha=None, budget_factor: int = 0,
                  no_graph: bool = False, profile: bool = False, prices_out=None,
                  slots: int = 0, lists: int = 0) -> la_batch_options:
    """Build la_batch_options; ``alpha`` is an int or a per-bucket list
    (bucket k holds 2^k <= n < 2^(k+1)); ``lists`` > 0 turns candidate lists
    on, < 0 off, 0 leaves the choice to the library (on for large n)."""
    o = la_batch_options()
    o.block_threads = block_threads
    o.max_n = max_n
    if alpha is not None:
        vals = [alpha] * LA_ALPHA_BUCKETS if isinstance(alpha, int) else list(alpha)
        for k, a in enumerate(vals[:LA_ALPHA_BUCKETS]):
            o.alpha[k] = int(a)
    o.budget_factor = budget_factor
    o.no_graph = int(bool(no_graph))
    o.profile = int(bool(profile))
    o.prices_out = _ptr(prices_out)
    o.slots = slots
    o.lists = lists
    return o


def solve_batched(costs, offsets, ns, *, options: la_batch_options = None, stream=None,
                  check: bool = True) -> BatchSolution:
    """Solve B packed instances (int32 costs, int64 offsets, int32 sizes; all
    CUDA tensors) in one persistent launch."""
    import torch
    B = int(ns.numel())
    for t, dt in ((costs, torch.int32), (offsets, torch.int64), (ns, torch.int32)):
        if t.dtype != dt or not t.is_cuda:
            raise ValueError("costs int32, offsets int64 and ns int32 must be CUDA tensors")
    dev = costs.device
    total = int(ns.sum().item()) if B else 0
    match = torch.empty(max(1, total), dtype=torch.int32, device=dev)
    out = torch.empty(max(1, B), dtype=torch.int64, device=dev)
    status = torch.empty(max(1, B), dtype=torch.int32, device=dev)
    st = la_batch_stats()
    with torch.cuda.device(dev):
        rc = la_solve_batched_ex(costs, offsets, ns, B, options, stream, match, out, status, st)
    if rc != LA_OK and check:
        raise LaError(rc, "la_solve_batched_ex")
    return BatchSolution(costs=out[:B], match=match[:total], status=status[:B],
                         stats=dict(st.as_dict(), rc=rc))


def solve_warm(C, weights, *, stream=None, check: bool = True) -> Solution:
    """Exact assignment warm-started from the learned price predictor
    (``weights``: float32 CUDA tensor of LA_PRED_PARAMS entries)."""
    import torch
    if C.dim() != 2 or C.shape[0] != C.shape[1] or C.dtype != torch.int32 or not C.is_cuda:
        raise ValueError("cost matrix must be a square int32 CUDA tensor")
    C = C.contiguous()
    n = C.shape[0]
    match = torch.empty(n, dtype=torch.int32, device=C.device)
    cost = torch.empty(1, dtype=torch.int64, device=C.device)
    st = la_stats()
    with torch.cuda.device(C.device):
        rc = la_solve_warm(C, n, weights, stream, match, cost, st)
    if rc != LA_OK and check:
        raise LaError(rc, "la_solve_warm")
    return Solution(cost=int(cost.item()) if rc == LA_OK else None, match=match,
                    stats=dict(st.as_dict(), status=rc))


def predict_prices(C, weights, *, stream=None):
    """Predicted column prices (int64 CUDA tensor, paper sign, scaled units)
    and the calibrated starting eps."""
    import torch
    n = C.shape[0]
    prices = torch.empty(max(1, n), dtype=torch.int64, device=C.device)
    eps0 = ctypes.c_int64(0)
    rc = la_predict_prices_ex(C.contiguous(), n, weights, stream, prices, ctypes.byref(eps0))
    if rc != LA_OK:
        raise LaError(rc, "la_predict_prices_ex")
    return prices[:n], int(eps0.value)
