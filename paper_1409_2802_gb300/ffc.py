"""ctypes binding of libffc (include/ffc.h): argument marshalling only.

Every function here validates nothing beyond tensor placement and dtype,
passes raw device pointers and sizes to the C ABI, and turns the returned
status into a Python value or exception. All arithmetic runs in libffc's
CUDA kernels; there is no CPU fallback: if libffc.so is missing or no GPU is
present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffc.so")

FFC_OK = 0
FFC_E_INVALID = 1
FFC_E_NOMEM = 2
FFC_E_CUDA = 3
FFC_E_TIMEOUT = 4
FFC_E_FARFIELD_TOO_SMALL = 5
FFC_E_SINGULAR = 6
FFC_E_TOL_NOT_REACHED = 7
SOFT_STATUSES = (FFC_OK, FFC_E_FARFIELD_TOO_SMALL, FFC_E_TOL_NOT_REACHED)

GAUSSIAN, LAPLACE, POLYNOMIAL = 0, 1, 2
SAMPLE_UNIFORM, SAMPLE_LEARNED, SAMPLE_DISTANCE, SAMPLE_INV_DISTANCE, SAMPLE_NEAREST = 0, 1, 2, 3, 4
F64, F32 = 0, 1
FP64, MIXED = 0, 1
EVAL_DEFAULT, EVAL_SIMT, EVAL_MMA_SYNC, EVAL_TCGEN05 = 0, 1, 2, 3
EVAL_TCGEN05_TILE0, EVAL_TCGEN05_TILES = 4, 5   # EVAL_TCGEN05_TILE0 + v: tcgen05 tile variant v
SOLVE_DEFAULT, SOLVE_FP64 = 0, 1

EXPORTS = (
    "ffc_last_error", "ffc_version", "ffc_far_field", "ffc_sample_rows", "ffc_eval_block", "ffc_id",
    "ffc_id_error", "ffc_tree_depth", "ffc_build_tree", "ffc_compress_tree", "ffc_tree_result_view",
    "ffc_tree_result_free", "ffc_tree_profile_enable", "ffc_tree_profile_reset", "ffc_tree_profile_get",
    "ffc_id_noalloc", "ffc_features", "ffc_mlp_forward", "ffc_sample_weighted", "ffc_propose_rows",
    "ffc_mlp_loss_grad", "ffc_adam_step", "ffc_leverage", "ffc_leverage_batched", "ffc_set_wait_limit",
    "ffc_skeleton_charges", "ffc_potential", "ffc_tree_apply", "ffc_sample_paper", "ffc_sample_leverage",
    "ffc_spectrum", "ffc_set_eval_path",
)
MLP_PARAMS = 18305
N_FEATURES = 12
MAX_DRAW = 8192
PROFILE_PHASES = ("sample", "eval", "qr", "trsm", "bookkeeping")


class FFCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libffc status {status}: {msg}")
        self.status = status


class c_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("p", ctypes.c_int32), ("h", ctypes.c_double), ("c", ctypes.c_double)]


class c_tree(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("begin_dev", ctypes.c_void_p),
                ("count_dev", ctypes.c_void_p), ("centroid_dev", ctypes.c_void_p), ("radius_dev", ctypes.c_void_p)]


class c_params(ctypes.Structure):
    _fields_ = [("kernel", c_kernel), ("precision", ctypes.c_int32), ("min_level", ctypes.c_int32),
                ("s0", ctypes.c_int32), ("s_max", ctypes.c_int32), ("tol", ctypes.c_double),
                ("xi", ctypes.c_double), ("seed", ctypes.c_uint64), ("sampler", ctypes.c_int32),
                ("pool_rows", ctypes.c_int32), ("proj_dev", ctypes.c_void_p), ("mlp_dev", ctypes.c_void_p),
                ("qr_big_min_s", ctypes.c_int32), ("qr_l2_budget_mb", ctypes.c_int32), ("qr_panel", ctypes.c_int32),
                ("nested", ctypes.c_int32), ("eval_path", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("qr_defer", ctypes.c_int32), ("solve", ctypes.c_int32)]


class c_tree_view(ctypes.Structure):
    _fields_ = [("n_out", ctypes.c_int64), ("rounds", ctypes.c_int32)] + [
        (name, ctypes.c_void_p) for name in (
            "node_dev", "rank_dev", "s_dev", "status_dev", "r22_rel_dev", "log_scale_dev", "far_count_dev",
            "rows_off_dev", "rows_dev", "skel_off_dev", "skel_dev", "T_off_dev", "T_dev", "ncols_dev", "cols_dev")]


class c_tree_profile(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("calls", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("launches", ctypes.c_int64), ("qr_launches", ctypes.c_int64),
                ("ms", ctypes.c_double * 5), ("qr_flops", ctypes.c_double), ("eval_flops", ctypes.c_double),
                ("qr_bytes", ctypes.c_double), ("qr_ms_round", ctypes.c_double * 8),
                ("items_round", ctypes.c_int64 * 8), ("graph_launches", ctypes.c_int64),
                ("graph_captures", ctypes.c_int64)]


@dataclass(frozen=True)
class Kernel:
    kind: int
    h: float = 1.0
    c: float = 1.0
    p: int = 3

    def c_struct(self) -> c_kernel:
        return c_kernel(int(self.kind), int(self.p), float(self.h), float(self.c))


_lib = None


def lib() -> ctypes.CDLL:
    """Load libffc.so (built by __graft_entry__.build()) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    pi64, pdbl = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    L.ffc_last_error.restype = ctypes.c_char_p
    L.ffc_version.restype = ctypes.c_char_p
    L.ffc_far_field.argtypes = [vp, i32, i64, i32, vp, dbl, dbl, i64, i64, vp, pi64, vp]
    L.ffc_sample_rows.argtypes = [vp, i32, i64, i32, vp, dbl, dbl, i64, i64, i64, u64, u64, vp, pi64, pi64, vp]
    L.ffc_eval_block.argtypes = [c_kernel, vp, i32, vp, i64, vp, i64, i32, vp, i32, vp, i64, pdbl, vp]
    L.ffc_id.argtypes = [vp, i64, i64, i64, i32, i64, dbl, vp, vp, i64, pi64, pdbl, vp]
    L.ffc_id_noalloc.argtypes = [vp, i64, i64, i64, i32, i64, dbl, vp, vp, i64, pi64, pdbl, vp]
    L.ffc_id_error.argtypes = [c_kernel, vp, i32, vp, i64, vp, i64, i32, vp, vp, i64, i64, pdbl, vp]
    L.ffc_tree_depth.argtypes = [i64, i64]
    L.ffc_tree_depth.restype = i32
    L.ffc_build_tree.argtypes = [vp, i32, i64, i32, i64, vp, vp, vp, vp, vp, vp]
    L.ffc_compress_tree.argtypes = [vp, i32, i64, i32, ctypes.POINTER(c_tree), ctypes.POINTER(c_params),
                                    ctypes.POINTER(vp), vp]
    L.ffc_tree_result_view.argtypes = [vp, ctypes.POINTER(c_tree_view)]
    L.ffc_tree_result_free.argtypes = [vp]
    L.ffc_tree_result_free.restype = None
    L.ffc_tree_profile_enable.argtypes = [vp, i32]
    L.ffc_tree_profile_reset.argtypes = [vp]
    L.ffc_tree_profile_get.argtypes = [vp, ctypes.POINTER(c_tree_profile)]
    L.ffc_features.argtypes = [c_kernel, vp, i32, i64, i32, vp, i64, vp, dbl, vp, vp, vp]
    L.ffc_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    L.ffc_sample_weighted.argtypes = [vp, vp, i64, i64, u64, u64, vp, vp]
    L.ffc_propose_rows.argtypes = [c_kernel, vp, i32, i64, i32, vp, dbl, dbl, i64, i64, vp, vp, i64, i64, u64, u64,
                                   vp, pi64, pi64, vp]
    L.ffc_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i32, i64, pdbl, vp, vp]
    L.ffc_adam_step.argtypes = [vp, vp, vp, vp, i64, i64, dbl, dbl, dbl, dbl, vp]
    L.ffc_leverage.argtypes = [vp, i64, i64, i64, dbl, i64, vp, vp, pi64, vp]
    L.ffc_leverage_batched.argtypes = [i32, vp, vp, vp, vp, dbl, i64, vp, vp, vp, vp]
    L.ffc_set_wait_limit.argtypes = [i64]
    L.ffc_set_eval_path.argtypes = [i32]
    L.ffc_skeleton_charges.argtypes = [vp, vp, i64, i64, i64, vp, i64, i64, vp, i64, vp]
    L.ffc_potential.argtypes = [c_kernel, vp, i32, vp, i64, vp, i64, i32, vp, i64, vp, dbl, vp, vp]
    L.ffc_spectrum.argtypes = [vp, i64, i64, i64, dbl, vp, pi64, vp]
    L.ffc_sample_paper.argtypes = [i32, vp, i32, i32, vp, i64, vp, vp, i64, i64, u64, u64, vp, vp]
    L.ffc_sample_leverage.argtypes = [vp, i64, i64, i64, vp, dbl, i64, u64, u64, vp, pi64, pi64, vp]
    L.ffc_tree_apply.argtypes = [vp, i32, i64, i32, ctypes.POINTER(c_tree), vp, vp, i32, i32, dbl, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("ffc_last_error", "ffc_version", "ffc_tree_depth", "ffc_tree_result_free"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int) -> int:
    if status not in SOFT_STATUSES:
        raise FFCError(status, lib().ffc_last_error().decode())
    return status


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"points must be float64 or float32, got {t.dtype}")


def _dev(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def version() -> str:
    return lib().ffc_version().decode()


def ffc_set_wait_limit(polls: int) -> None:
    """Polls of a bounded device wait before it gives up (< 0: the library's default)."""
    _check(lib().ffc_set_wait_limit(int(polls)))


def ffc_set_eval_path(path: int) -> None:
    """The evaluation path EVAL_DEFAULT stands for (one of EVAL_*), process-wide."""
    _check(lib().ffc_set_eval_path(int(path)))


def ffc_far_field(Y, x_c=None, radius=0.0, xi=1.0, ex_begin=0, ex_end=0, stream=None):
    """Ascending far-field indices of Y (int64 CUDA tensor)."""
    _dev(Y, "Y")
    M, d = Y.shape
    idx = torch.empty(M, dtype=torch.int64, device=Y.device)
    cnt = ctypes.c_int64(0)
    _check(lib().ffc_far_field(_ptr(Y), _dtype_code(Y), M, d, _ptr(x_c), float(radius), float(xi),
                               int(ex_begin), int(ex_end), _ptr(idx), ctypes.byref(cnt), _stream(stream)))
    return idx[: cnt.value]


def ffc_sample_rows(Y, s, seed, stream_id, x_c=None, radius=0.0, xi=1.0, ex_begin=0, ex_end=0, stream=None):
    """Uniform far-field sample: returns (rows int64[s_out], far_count, status)."""
    _dev(Y, "Y")
    M, d = Y.shape
    rows = torch.empty(max(int(s), 1), dtype=torch.int64, device=Y.device)
    s_out, fc = ctypes.c_int64(0), ctypes.c_int64(0)
    st = _check(lib().ffc_sample_rows(_ptr(Y), _dtype_code(Y), M, d, _ptr(x_c), float(radius), float(xi),
                                      int(ex_begin), int(ex_end), int(s), ctypes.c_uint64(int(seed)),
                                      ctypes.c_uint64(int(stream_id)), _ptr(rows), ctypes.byref(s_out),
                                      ctypes.byref(fc), _stream(stream)))
    return rows[: s_out.value], fc.value, st


def ffc_eval_block(kernel: Kernel, Y, rows, X, precision=FP64, center=None, K=None, stream=None):
    """K'(rows, X) column-major: returns (K as an (n, s) row-major view's transpose, log_scale).

    The block is stored column-major s x n with ld = s; the returned tensor is
    the s x n matrix view of that storage.
    """
    _dev(Y, "Y"), _dev(X, "X"), _dev(rows, "rows")
    s, (n, d) = rows.numel(), X.shape
    if K is None:
        K = torch.empty((max(n, 1), max(s, 1)), dtype=torch.float64 if precision == FP64 else torch.float32,
                        device=X.device)
    ls = ctypes.c_double(0.0)
    _check(lib().ffc_eval_block(kernel.c_struct(), _ptr(Y), _dtype_code(Y), _ptr(rows), s, _ptr(X), n, d,
                                _ptr(center), int(precision), _ptr(K), max(s, 1), ctypes.byref(ls),
                                _stream(stream)))
    return K[:n, :s].t(), ls.value


def ffc_id(Kcm, r_max, tol=0.0, precision=FP64, stream=None):
    """ID of a column-major block given as its (n, s) storage tensor (overwritten).

    Returns (skel_perm int32[n], T (rank x (n - rank)) float64, rank, r22_rel, status).
    """
    _dev(Kcm, "K")
    n, s = Kcm.shape
    ldt = max(int(r_max), 1)
    skel = torch.empty(max(n, 1), dtype=torch.int32, device=Kcm.device)
    T = torch.empty((max(n, 1), ldt), dtype=torch.float64, device=Kcm.device)
    rank, r22 = ctypes.c_int64(0), ctypes.c_double(0.0)
    st = _check(lib().ffc_id(_ptr(Kcm), s, n, max(s, 1), int(precision), int(r_max), float(tol), _ptr(skel),
                             _ptr(T), ldt, ctypes.byref(rank), ctypes.byref(r22), _stream(stream)))
    r = rank.value
    return skel[:n], T[: n - r, :r].t(), r, r22.value, st


def ffc_id_error(kernel: Kernel, Y, X, skel, T, r, rows=None, ldt=None, stream=None):
    """Full-block relative Frobenius error of an ID; T given as a (ldt, n-r) column-major storage."""
    _dev(Y, "Y"), _dev(X, "X")
    m = rows.numel() if rows is not None else Y.shape[0]
    n, d = X.shape
    err = ctypes.c_double(0.0)
    Tc = T.t().contiguous() if T.numel() else torch.zeros(1, dtype=torch.float64, device=X.device)
    _check(lib().ffc_id_error(kernel.c_struct(), _ptr(Y), _dtype_code(Y), _ptr(rows), m, _ptr(X), n, d,
                              _ptr(skel), _ptr(Tc), max(int(r), 1) if ldt is None else int(ldt), int(r),
                              ctypes.byref(err), _stream(stream)))
    return err.value


def ffc_tree_depth(N, leaf_size) -> int:
    return int(lib().ffc_tree_depth(int(N), int(leaf_size)))


@dataclass
class DeviceTree:
    depth: int
    perm: torch.Tensor
    begin: torch.Tensor
    count: torch.Tensor
    centroid: torch.Tensor
    radius: torch.Tensor

    @property
    def n_nodes(self) -> int:
        return int(self.begin.numel())

    def c_struct(self) -> c_tree:
        return c_tree(self.depth, self.n_nodes, self.begin.data_ptr(), self.count.data_ptr(),
                      self.centroid.data_ptr(), self.radius.data_ptr())


def ffc_build_tree(points, leaf_size, stream=None) -> DeviceTree:
    _dev(points, "points")
    N, d = points.shape
    depth = ffc_tree_depth(N, leaf_size)
    nn = (1 << (depth + 1)) - 1
    dev = points.device
    t = DeviceTree(depth, torch.empty(N, dtype=torch.int64, device=dev), torch.empty(nn, dtype=torch.int64, device=dev),
                   torch.empty(nn, dtype=torch.int64, device=dev), torch.empty((nn, d), dtype=torch.float64, device=dev),
                   torch.empty(nn, dtype=torch.float64, device=dev))
    _check(lib().ffc_build_tree(_ptr(points), _dtype_code(points), N, d, int(leaf_size), _ptr(t.perm), _ptr(t.begin),
                                _ptr(t.count), _ptr(t.centroid), _ptr(t.radius), _stream(stream)))
    return t


class TreeResult:
    """Owns an ffc_tree_result; frees it on close()/deletion."""

    def __init__(self):
        self.handle = ctypes.c_void_p(0)

    def view(self) -> c_tree_view:
        v = c_tree_view()
        _check(lib().ffc_tree_result_view(self.handle, ctypes.byref(v)))
        return v

    def profile_enable(self, enabled: bool = True):
        _check(lib().ffc_tree_profile_enable(self.handle, 1 if enabled else 0))

    def profile_reset(self):
        _check(lib().ffc_tree_profile_reset(self.handle))

    def profile(self) -> dict:
        p = c_tree_profile()
        _check(lib().ffc_tree_profile_get(self.handle, ctypes.byref(p)))
        return {"calls": p.calls, "rounds": p.rounds, "launches": p.launches, "qr_launches": p.qr_launches,
                "ms": dict(zip(PROFILE_PHASES, list(p.ms))), "qr_flops": p.qr_flops, "eval_flops": p.eval_flops,
                "qr_bytes": p.qr_bytes, "qr_ms_round": list(p.qr_ms_round), "items_round": list(p.items_round),
                "graph_launches": p.graph_launches, "graph_captures": p.graph_captures}

    def close(self):
        if self.handle and self.handle.value:
            lib().ffc_tree_result_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ffc_compress_tree(points_perm, tree: DeviceTree, kernel: Kernel, tol=1e-6, precision=FP64, min_level=2, s0=128,
                      s_max=2048, xi=1.0, seed=0, result: TreeResult | None = None, stream=None,
                      proposal: tuple | None = None, pool_rows=0, qr_big_min_s=0,
                      qr_l2_budget_mb=0, sampler: int | None = None, qr_panel=0, nested=False,
                      eval_path=EVAL_DEFAULT, graphs=True, qr_defer=0, solve=SOLVE_DEFAULT) -> TreeResult:
    """Compress every node at level >= min_level; ``proposal`` = (params, proj) selects the learned sampler,
    ``sampler`` one of SAMPLE_* otherwise (default uniform). ``qr_big_min_s``, ``qr_l2_budget_mb``, ``qr_panel``:
    the QR's launch shape and panel width (0 = the library's defaults; 1 = unblocked; see ``autotune``);
    ``eval_path``: one of EVAL_* for the mixed-precision Gaussian / polynomial blocks; ``graphs``: run each round
    as a captured CUDA graph (replayed when the round recurs) instead of direct launches; ``qr_defer``: the QR's
    write-back depth (0 = the library's default, 1 = every step, 2..4 = the lazy form); ``solve``: SOLVE_* of the
    mixed-precision triangular solve."""
    _dev(points_perm, "points_perm")
    N, d = points_perm.shape
    res = result if result is not None else TreeResult()
    proj_p, mlp_p = None, None
    sampler = SAMPLE_UNIFORM if sampler is None else int(sampler)
    if proposal is not None:
        mlp, proj = proposal
        _dev(mlp, "proposal params"), _dev(proj, "proposal proj")
        sampler, proj_p, mlp_p = 1, proj.data_ptr(), mlp.data_ptr()
    p = c_params(kernel.c_struct(), int(precision), int(min_level), int(s0), int(s_max), float(tol), float(xi),
                 ctypes.c_uint64(int(seed)), sampler, int(pool_rows), proj_p, mlp_p, int(qr_big_min_s),
                 int(qr_l2_budget_mb), int(qr_panel), 1 if nested else 0, int(eval_path), 0 if graphs else 1,
                 int(qr_defer), int(solve))
    tr = tree.c_struct()
    _check(lib().ffc_compress_tree(_ptr(points_perm), _dtype_code(points_perm), N, d, ctypes.byref(tr),
                                   ctypes.byref(p), ctypes.byref(res.handle), _stream(stream)))
    return res


APPLY_SKELETON, APPLY_DIRECT = 0, 1
DRAW_DISTANCE, DRAW_INV_DISTANCE, DRAW_NEAREST = 0, 1, 2


def ffc_sample_paper(sampler, Y, cand, s, seed, stream_id, x_c=None, X=None, stream=None):
    """min(s, P) of the candidate rows cand of Y by a paper sampler (DRAW_*), in key order."""
    _dev(Y, "Y"), _dev(cand, "cand")
    M, d = Y.shape
    P = cand.numel()
    keep = min(int(s), P)
    rows = torch.empty(max(keep, 1), dtype=torch.int64, device=Y.device)
    n = X.shape[0] if X is not None else 0
    _check(lib().ffc_sample_paper(int(sampler), _ptr(Y), _dtype_code(Y), d, _ptr(cand), P, _ptr(x_c), _ptr(X), n,
                                  int(s), ctypes.c_uint64(int(seed)), ctypes.c_uint64(int(stream_id)), _ptr(rows),
                                  _stream(stream)))
    return rows[:keep]


def ffc_sample_leverage(Kcm, s, seed, stream_id, eps=1e-6, cand=None, stream=None):
    """Rows of the full block (given as its (n, m) column-major storage) drawn by leverage; returns
    (rows, eps-rank, status)."""
    _dev(Kcm, "K")
    n, m = Kcm.shape
    rows = torch.empty(max(min(int(s), m), 1), dtype=torch.int64, device=Kcm.device)
    s_out, rank = ctypes.c_int64(0), ctypes.c_int64(0)
    st = _check(lib().ffc_sample_leverage(_ptr(Kcm), m, n, m, _ptr(cand), float(eps), int(s),
                                          ctypes.c_uint64(int(seed)), ctypes.c_uint64(int(stream_id)), _ptr(rows),
                                          ctypes.byref(s_out), ctypes.byref(rank), _stream(stream)))
    return rows[:s_out.value], rank.value, st


def ffc_skeleton_charges(skel, T, q, stream=None):
    """q~ = P q for an ID (skel int32[n], T (r x (n - r)) float64 as ffc_id returns it); q: (n,) or (n, nrhs)."""
    _dev(skel, "skel"), _dev(q, "q")
    n = skel.numel()
    r = T.shape[0]
    Tc = T.t().contiguous()                       # column c of T at Tc + c r
    qc = q.reshape(n, -1).t().contiguous()        # column j of q at qc + j n
    nrhs = qc.shape[0]
    qt = torch.empty((nrhs, max(r, 1)), dtype=torch.float64, device=q.device)
    _check(lib().ffc_skeleton_charges(_ptr(skel), _ptr(Tc) if r < n else None, max(r, 1), r, n, _ptr(qc), max(n, 1),
                                      nrhs, _ptr(qt), max(r, 1), _stream(stream)))
    out = qt[:, :r].t()
    return out.reshape(r) if q.dim() == 1 else out


def ffc_potential(kernel: Kernel, Y, X, w, rows=None, cols=None, log_scale=0.0, stream=None):
    """u_i = exp(-log_scale) sum_c K(Y[rows_i], X[cols_c]) w_c (cols None: all of X)."""
    _dev(Y, "Y"), _dev(X, "X"), _dev(w, "w")
    M, d = Y.shape
    n = X.shape[0]
    m = rows.numel() if rows is not None else M
    nc = cols.numel() if cols is not None else n
    u = torch.empty(max(m, 1), dtype=torch.float64, device=Y.device)
    _check(lib().ffc_potential(kernel.c_struct(), _ptr(Y), _dtype_code(Y), _ptr(rows), m, _ptr(X), n, d, _ptr(cols),
                               nc, _ptr(w), float(log_scale), _ptr(u), _stream(stream)))
    return u[:m]


def ffc_tree_apply(points_perm, tree: "DeviceTree", result: "TreeResult", q, mode=APPLY_SKELETON, near_field=True,
                   log_scale=0.0, s_max=2048, stream=None):
    """Potential at every point (tree order) from the compressed tree's representations; returns (u, qt) with
    qt the skeleton charges (n_out x s_max/2, node i's first r_i entries), None in direct mode."""
    _dev(points_perm, "points_perm"), _dev(q, "q")
    N, d = points_perm.shape
    n_out = int(result.view().n_out)
    qt = torch.zeros((n_out, s_max // 2), dtype=torch.float64, device=q.device) if mode == APPLY_SKELETON else None
    u = torch.empty(N, dtype=torch.float64, device=q.device)
    tr = tree.c_struct()
    _check(lib().ffc_tree_apply(_ptr(points_perm), _dtype_code(points_perm), N, d, ctypes.byref(tr), result.handle,
                                _ptr(q), int(mode), 1 if near_field else 0, float(log_scale), _ptr(qt), _ptr(u),
                                _stream(stream)))
    return u, qt


_TORCH_DTYPES = {"int32": torch.int32, "int64": torch.int64, "float64": torch.float64}


def device_view(ptr: int, count: int, dtype: str) -> torch.Tensor:
    """A CUDA tensor viewing `count` elements of library-owned device memory (no copy)."""
    if count == 0 or not ptr:
        return torch.empty(0, dtype=_TORCH_DTYPES[dtype], device="cuda")
    typestr = {"int32": "<i4", "int64": "<i8", "float64": "<f8"}[dtype]

    class _View:
        __cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                    "version": 3, "strides": None}

    return torch.as_tensor(_View(), device="cuda")


def tree_result_views(res: TreeResult) -> dict:
    """Device views of a TreeResult's per-node outputs (valid while `res` lives)."""
    v = res.view()
    n = int(v.n_out)
    out = {"n_out": n, "rounds": int(v.rounds)}
    for name, dt, cnt in (("node", "int32", n), ("rank", "int32", n), ("s", "int32", n), ("status", "int32", n),
                          ("r22_rel", "float64", n), ("log_scale", "float64", n), ("far_count", "int64", n),
                          ("rows_off", "int64", n + 1), ("skel_off", "int64", n + 1), ("T_off", "int64", n + 1)):
        out[name] = device_view(getattr(v, name + "_dev"), cnt, dt)
    out["rows"] = device_view(v.rows_dev, int(out["rows_off"][-1].item()) if n else 0, "int64")
    out["skel"] = device_view(v.skel_dev, int(out["skel_off"][-1].item()) if n else 0, "int32")
    out["T"] = device_view(v.T_dev, int(out["T_off"][-1].item()) if n else 0, "float64")
    out["ncols"] = device_view(v.ncols_dev, n, "int32")
    out["cols"] = device_view(v.cols_dev, int(out["skel_off"][-1].item()) if n else 0, "int32")
    return out


def tree_result_to_host(res: TreeResult) -> dict:
    """numpy copies of a TreeResult's per-node outputs."""
    views = tree_result_views(res)
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in views.items()}


# ---------------------------------------------------------------------------
# learned row proposal and its training


def ffc_features(kernel: Kernel, Y, rows, x_c, radius, proj, stream=None):
    """R x 12 float32 features of the targets Y[rows] for a node (x_c, radius)."""
    _dev(Y, "Y"), _dev(rows, "rows"), _dev(x_c, "x_c"), _dev(proj, "proj")
    M, d = Y.shape
    R = rows.numel()
    F = torch.empty((max(R, 1), N_FEATURES), dtype=torch.float32, device=Y.device)
    _check(lib().ffc_features(kernel.c_struct(), _ptr(Y), _dtype_code(Y), M, d, _ptr(rows), R, _ptr(x_c),
                              float(radius), _ptr(proj), _ptr(F), _stream(stream)))
    return F[:R]


def ffc_mlp_forward(params, feats, stream=None):
    """Logits (float32, one per feature row) of the proposal network."""
    _dev(params, "params"), _dev(feats, "feats")
    R = feats.shape[0]
    out = torch.empty(max(R, 1), dtype=torch.float32, device=feats.device)
    _check(lib().ffc_mlp_forward(_ptr(params), _ptr(feats), R, _ptr(out), _stream(stream)))
    return out[:R]


def ffc_sample_weighted(pool, logits, s, seed, stream_id, stream=None):
    """min(s, P) pool rows drawn without replacement with the mixed network weights."""
    _dev(pool, "pool"), _dev(logits, "logits")
    P = pool.numel()
    n = min(int(s), P)
    rows = torch.empty(max(n, 1), dtype=torch.int64, device=pool.device)
    _check(lib().ffc_sample_weighted(_ptr(pool), _ptr(logits), P, int(s), ctypes.c_uint64(int(seed)),
                                     ctypes.c_uint64(int(stream_id)), _ptr(rows), _stream(stream)))
    return rows[:n]


def ffc_propose_rows(kernel: Kernel, Y, s, seed, stream_id, x_c, radius, proj, params, xi=1.0, ex_begin=0,
                     ex_end=0, pool_rows=0, stream=None):
    """Learned proposal of s far-field rows (pool_rows = 0: the whole far field is the candidate pool).

    Returns (rows int64[s_out], far_count, status)."""
    _dev(Y, "Y"), _dev(x_c, "x_c"), _dev(proj, "proj"), _dev(params, "params")
    M, d = Y.shape
    rows = torch.empty(max(int(s), 1), dtype=torch.int64, device=Y.device)
    s_out, fc = ctypes.c_int64(0), ctypes.c_int64(0)
    st = _check(lib().ffc_propose_rows(kernel.c_struct(), _ptr(Y), _dtype_code(Y), M, d, _ptr(x_c), float(radius),
                                       float(xi), int(ex_begin), int(ex_end), _ptr(proj), _ptr(params),
                                       int(pool_rows), int(s), ctypes.c_uint64(int(seed)),
                                       ctypes.c_uint64(int(stream_id)), _ptr(rows), ctypes.byref(s_out),
                                       ctypes.byref(fc), _stream(stream)))
    return rows[: s_out.value], fc.value, st


def ffc_mlp_loss_grad(params, feats, targets, node_off, grad=None, stream=None):
    """(loss, grad float32[MLP_PARAMS]) of the per-node softmax cross-entropy (targets float64)."""
    for t, nm in ((params, "params"), (feats, "feats"), (targets, "targets"), (node_off, "node_off")):
        _dev(t, nm)
    if grad is None:
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=params.device)
    loss = ctypes.c_double(0.0)
    _check(lib().ffc_mlp_loss_grad(_ptr(params), _ptr(feats), _ptr(targets), _ptr(node_off), node_off.numel() - 1,
                                   feats.shape[0], ctypes.byref(loss), _ptr(grad), _stream(stream)))
    return loss.value, grad


def ffc_adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """In-place Adam update of params (float32) with moments m, v (float32)."""
    for t, nm in ((params, "params"), (grad, "grad"), (m, "m"), (v, "v")):
        _dev(t, nm)
    _check(lib().ffc_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), _stream(stream)))


def ffc_spectrum(Kcm, eps=1e-2, stream=None):
    """(singular values (decreasing), eps-rank, status) of a block given as its (n, m) column-major storage."""
    _dev(Kcm, "K")
    n, m = Kcm.shape
    sigma = torch.empty(n, dtype=torch.float64, device=Kcm.device)
    rank = ctypes.c_int64(0)
    st = _check(lib().ffc_spectrum(_ptr(Kcm), m, n, m, float(eps), _ptr(sigma), ctypes.byref(rank), _stream(stream)))
    return sigma, rank.value, st


def ffc_leverage(Kcm, eps=1e-6, r_fixed=0, stream=None):
    """Leverage scores of the rows of a column-major m x n block given as its (n, m) storage.

    Returns (lev float64[m], sigma float64[n] decreasing, rank, status).
    """
    _dev(Kcm, "K")
    n, m = Kcm.shape
    lev = torch.empty(max(m, 1), dtype=torch.float64, device=Kcm.device)
    sig = torch.empty(max(n, 1), dtype=torch.float64, device=Kcm.device)
    rank = ctypes.c_int64(0)
    st = _check(lib().ffc_leverage(_ptr(Kcm), m, n, m, float(eps), int(r_fixed), _ptr(lev), _ptr(sig),
                                   ctypes.byref(rank), _stream(stream)))
    return lev[:m], sig[:n], rank.value, st


def ffc_leverage_batched(Kcms, eps=1e-6, r_fixed=0, stream=None):
    """ffc_leverage of several column-major blocks (each given as its (n, m) storage) at once.

    Returns a list of (lev float64[m], sigma float64[n], rank) and the status.
    """
    B = len(Kcms)
    for K in Kcms:
        _dev(K, "K")
    P = ctypes.c_void_p * B
    I = ctypes.c_int64 * B
    ns = [int(K.shape[0]) for K in Kcms]
    ms = [int(K.shape[1]) for K in Kcms]
    levs = [torch.empty(max(m, 1), dtype=torch.float64, device=K.device) for m, K in zip(ms, Kcms)]
    sigs = [torch.empty(max(n, 1), dtype=torch.float64, device=K.device) for n, K in zip(ns, Kcms)]
    ranks = I()
    st = _check(lib().ffc_leverage_batched(B, P(*[K.data_ptr() for K in Kcms]), I(*ms), I(*ns), I(*ms),
                                           float(eps), int(r_fixed), P(*[t.data_ptr() for t in levs]),
                                           P(*[t.data_ptr() for t in sigs]), ranks, _stream(stream)))
    return [(levs[b][:ms[b]], sigs[b][:ns[b]], int(ranks[b])) for b in range(B)], st
