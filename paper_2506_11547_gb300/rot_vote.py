"""ctypes binding of librot_vote.so (include/rot_vote.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels. There is no CPU
fallback: if the library is not built, `load()` raises.

Inputs may be numpy float32 arrays (host memory: the library copies them to
the device inside the call), torch CUDA float32 tensors, or any object with a
`data_ptr()` of device memory.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librot_vote.so")

OK, PENDING, EINVAL, ENOMEM, ECUDA, EAGAIN, ETIMEDOUT, EDEGENERATE, ENOTFOUND, ETOOLARGE = 0, 1, -1, -2, -3, -4, -5, -6, -7, -8
STATIC_SCRATCH_BYTES, STATIC_MAX_PAIRS, STATIC_MAX_CELLS = 4 << 20, 32768, 8192
PREC = {"fp32": 0, "fp16": 1, "bf16": 2, "fp16x2": 3, "bf16x2": 4}
RANK = {"excess": 0, "raw": 1}
CHART = {"orthographic": 0, "stereographic": 1}


class rot_vote_config(C.Structure):
    _fields_ = [("grid_n", C.c_int), ("levels", C.c_int), ("top_k", C.c_int), ("precision", C.c_int),
                ("recheck_band", C.c_float), ("rank_mode", C.c_int), ("refit_iters", C.c_int),
                ("device_mem_budget", C.c_size_t), ("max_inflight", C.c_int), ("cuda_stream", C.c_void_p),
                ("use_graphs", C.c_int), ("keep_trace", C.c_int), ("autotune", C.c_int), ("chart", C.c_int)]


class rot_vote_problem(C.Structure):
    _fields_ = [("a", C.c_void_p), ("b", C.c_void_p), ("n", C.c_int64), ("delta", C.c_float),
                ("grid_n", C.c_int), ("levels", C.c_int)]


class rot_vote_result(C.Structure):
    _fields_ = [("q", C.c_double * 4), ("R", C.c_double * 9), ("best_count", C.c_int32), ("inliers", C.c_int32),
                ("best_cell", C.c_int64), ("best_level", C.c_int32), ("refits", C.c_int32), ("tests", C.c_int64),
                ("rechecked", C.c_int64), ("ambiguous", C.c_int64), ("status", C.c_int32), ("ms_gpu", C.c_float),
                ("latency_ms", C.c_float), ("resolved", C.c_int64)]


ALG1_MAX_PEAKS, ALG1_PEAK_CANDIDATES = 64, 16384


class rot_vote_peak(C.Structure):
    _fields_ = [("q", C.c_double * 4), ("cell", C.c_int64), ("count", C.c_int32), ("pad", C.c_int32)]


class rot_vote_alg1_problem(C.Structure):
    _fields_ = [("a", C.c_void_p), ("b", C.c_void_p), ("n", C.c_int64), ("samples", C.c_int),
                ("accum_side", C.c_int), ("accumulator", C.c_void_p), ("peaks", C.c_int), ("min_count", C.c_int),
                ("nms_angle", C.c_float), ("peak_out", C.c_void_p)]


class rot_vote_alg1_result(C.Structure):
    _fields_ = [("q", C.c_double * 4), ("R", C.c_double * 9), ("best_count", C.c_int32), ("status", C.c_int32),
                ("best_cell", C.c_int64), ("samples_cast", C.c_int64), ("rechecked", C.c_int64),
                ("ms_gpu", C.c_float), ("npeaks", C.c_int32), ("peak_threshold", C.c_int32), ("vote_path", C.c_int32),
                ("wrapped_words", C.c_int32)]


class rot_vote_pose_problem(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("n", C.c_int64), ("mu", C.c_float), ("min_length", C.c_float),
                ("delta", C.c_float), ("grid_n", C.c_int), ("levels", C.c_int), ("t_half", C.c_float),
                ("t_cells", C.c_int), ("pairs_a", C.c_void_p), ("pairs_b", C.c_void_p), ("pairs_cap", C.c_int64)]


class rot_vote_pose_result(C.Structure):
    _fields_ = [("rot", rot_vote_result), ("t", C.c_double * 3), ("t_cell", C.c_int64), ("pairs_tested", C.c_int64),
                ("pairs_kept", C.c_int64), ("pairs_rechecked", C.c_int64), ("t_count", C.c_int32),
                ("status", C.c_int32), ("ms_gpu", C.c_float), ("pad", C.c_float)]


class rot_vote_stage(C.Structure):
    _fields_ = [("kind", C.c_int32), ("level", C.c_int32), ("ms", C.c_float), ("kernels", C.c_int32)]


class rot_vote_batch_span(C.Structure):
    _fields_ = [("t_start_ms", C.c_float), ("t_end_ms", C.c_float), ("wave", C.c_int32), ("problems", C.c_int32)]


STAGE_KIND = {0: "pair_prep", 1: "vote", 2: "topk", 3: "children", 4: "fit", 5: "alg1_zero", 6: "alg1_vote",
              7: "alg1_argmax"}

_lib = None

EXPORTS = ("rot_vote_create", "rot_vote_solve", "rot_vote_submit", "rot_vote_poll", "rot_vote_level_trace",
           "rot_vote_stage_times", "rot_vote_destroy", "rot_vote_last_error", "rot_vote_count_cells_static",
           "rot_vote_alg1", "rot_vote_pose", "rot_vote_serve_spans")


def load(path: str = LIB_PATH):
    """Loads the library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(path)
    L.rot_vote_create.argtypes = [C.POINTER(rot_vote_config), C.POINTER(C.c_void_p)]
    L.rot_vote_create.restype = C.c_int
    L.rot_vote_solve.argtypes = [C.c_void_p, C.POINTER(rot_vote_problem), C.c_int, C.POINTER(rot_vote_result)]
    L.rot_vote_solve.restype = C.c_int
    L.rot_vote_submit.argtypes = [C.c_void_p, C.POINTER(rot_vote_problem), C.POINTER(C.c_uint64)]
    L.rot_vote_submit.restype = C.c_int
    L.rot_vote_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(rot_vote_result), C.c_int]
    L.rot_vote_poll.restype = C.c_int
    L.rot_vote_level_trace.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64,
                                       C.POINTER(C.c_int64), C.c_void_p, C.POINTER(C.c_int32)]
    L.rot_vote_level_trace.restype = C.c_int
    L.rot_vote_stage_times.argtypes = [C.c_void_p, C.POINTER(rot_vote_stage), C.c_int, C.POINTER(C.c_int)]
    L.rot_vote_stage_times.restype = C.c_int
    L.rot_vote_serve_spans.argtypes = [C.c_void_p, C.POINTER(rot_vote_batch_span), C.c_int, C.POINTER(C.c_int)]
    L.rot_vote_serve_spans.restype = C.c_int
    L.rot_vote_destroy.argtypes = [C.c_void_p]
    L.rot_vote_destroy.restype = None
    L.rot_vote_last_error.argtypes = [C.c_void_p]
    L.rot_vote_last_error.restype = C.c_char_p
    L.rot_vote_count_cells_static.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int, C.c_void_p,
                                              C.c_int32, C.c_void_p, C.c_void_p]
    L.rot_vote_count_cells_static.restype = C.c_int
    L.rot_vote_alg1.argtypes = [C.c_void_p, C.POINTER(rot_vote_alg1_problem), C.c_int,
                                C.POINTER(rot_vote_alg1_result)]
    L.rot_vote_alg1.restype = C.c_int
    L.rot_vote_pose.argtypes = [C.c_void_p, C.POINTER(rot_vote_pose_problem), C.c_int,
                                C.POINTER(rot_vote_pose_result)]
    L.rot_vote_pose.restype = C.c_int
    _lib = L
    return L


@dataclasses.dataclass
class Result:
    q: np.ndarray
    R: np.ndarray
    best_count: int
    inliers: int
    best_cell: int
    best_level: int
    refits: int
    tests: int
    rechecked: int
    ambiguous: int
    status: int
    ms_gpu: float
    latency_ms: float
    resolved: int = 0

    @staticmethod
    def of(r: rot_vote_result) -> "Result":
        return Result(q=np.array(r.q[:]), R=np.array(r.R[:]).reshape(3, 3), best_count=r.best_count,
                      inliers=r.inliers, best_cell=r.best_cell, best_level=r.best_level, refits=r.refits,
                      tests=r.tests, rechecked=r.rechecked, ambiguous=r.ambiguous, status=r.status,
                      ms_gpu=r.ms_gpu, latency_ms=r.latency_ms, resolved=r.resolved)


@dataclasses.dataclass
class Alg1Result:
    q: np.ndarray
    R: np.ndarray
    best_count: int
    status: int
    best_cell: int
    samples_cast: int
    rechecked: int
    ms_gpu: float
    peak_threshold: int = 0
    peaks: list = dataclasses.field(default_factory=list)  # [(cell, count, q[4])] in peak order
    vote_path: int = 0  # 0 return-less vote; 1 that vote, wrapped, then the recording vote; 2 recording vote only
    wrapped_words: int = 0  # counter words holding a cell with 65536 or more votes

    @staticmethod
    def of(r: rot_vote_alg1_result, peaks=None) -> "Alg1Result":
        pk = [] if peaks is None else [(int(peaks[k].cell), int(peaks[k].count), np.array(peaks[k].q[:]))
                                       for k in range(r.npeaks)]
        return Alg1Result(q=np.array(r.q[:]), R=np.array(r.R[:]).reshape(3, 3), best_count=r.best_count,
                          status=r.status, best_cell=r.best_cell, samples_cast=r.samples_cast,
                          rechecked=r.rechecked, ms_gpu=r.ms_gpu, peak_threshold=r.peak_threshold, peaks=pk,
                          vote_path=r.vote_path, wrapped_words=r.wrapped_words)


@dataclasses.dataclass
class PoseResult:
    rot: Result
    t: np.ndarray
    t_cell: int
    t_count: int
    pairs_tested: int
    pairs_kept: int
    pairs_rechecked: int
    status: int
    ms_gpu: float

    @staticmethod
    def of(r: rot_vote_pose_result) -> "PoseResult":
        return PoseResult(rot=Result.of(r.rot), t=np.array(r.t[:]), t_cell=r.t_cell, t_count=r.t_count,
                          pairs_tested=r.pairs_tested, pairs_kept=r.pairs_kept, pairs_rechecked=r.pairs_rechecked,
                          status=r.status, ms_gpu=r.ms_gpu)


class RotVoteError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rot_vote error {code}: {msg}")
        self.code = code


def _ptr(x):
    """(address, keepalive) of a float32 [n, 3] array or device tensor."""
    if hasattr(x, "data_ptr"):
        if hasattr(x, "dtype") and str(x.dtype) != "torch.float32":
            raise TypeError("inputs must be float32")
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise TypeError("inputs must be contiguous")
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=np.float32)
    return a.ctypes.data, a


def _nrows(x) -> int:
    return int(x.shape[0])


def problem(a, b, delta: float, grid_n: int = 0, levels: int = 0):
    """A rot_vote_problem and the objects that keep its buffers alive."""
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    n = _nrows(a)
    if _nrows(b) != n:
        raise ValueError("a and b differ in length")
    return rot_vote_problem(pa, pb, n, float(delta), int(grid_n), int(levels)), (ka, kb)


class Context:
    """A rot_vote context (rot_vote_create ... rot_vote_destroy)."""

    def __init__(self, grid_n=0, levels=0, top_k=0, precision="fp32", recheck_band=0.0, rank_mode="excess",
                 refit_iters=0, device_mem_budget=0, max_inflight=0, cuda_stream=None, use_graphs=0,
                 keep_trace=0, autotune=0, chart="orthographic"):
        L = load()
        self._L = L
        cfg = rot_vote_config(int(grid_n), int(levels), int(top_k),
                              PREC[precision] if isinstance(precision, str) else int(precision),
                              float(recheck_band), RANK[rank_mode] if isinstance(rank_mode, str) else int(rank_mode),
                              int(refit_iters), int(device_mem_budget), int(max_inflight),
                              C.c_void_p(cuda_stream) if cuda_stream else None, int(use_graphs), int(keep_trace),
                              int(autotune), CHART[chart] if isinstance(chart, str) else int(chart))
        h = C.c_void_p()
        rc = L.rot_vote_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise RotVoteError(rc, "rot_vote_create failed")
        self._h = h
        self._keep = {}

    def last_error(self) -> str:
        return self._L.rot_vote_last_error(self._h).decode()

    def _check(self, rc: int):
        if rc not in (OK, PENDING):
            raise RotVoteError(rc, self.last_error())
        return rc

    def solve(self, problems):
        """problems: list of (a, b, delta[, grid_n[, levels]]). Returns list of Result."""
        n = len(problems)
        arr = (rot_vote_problem * n)()
        keep = []
        for k, pr in enumerate(problems):
            arr[k], kk = problem(*pr)
            keep.append(kk)
        out = (rot_vote_result * n)()
        self._check(self._L.rot_vote_solve(self._h, arr, n, out))
        return [Result.of(out[k]) for k in range(n)]

    def solve_raw(self, arr, n, out):
        """Calls rot_vote_solve on prepared ctypes arrays (for timing loops)."""
        return self._check(self._L.rot_vote_solve(self._h, arr, n, out))

    def submit(self, a, b, delta, grid_n=0, levels=0) -> int:
        pr, kk = problem(a, b, delta, grid_n, levels)
        t = C.c_uint64()
        rc = self._L.rot_vote_submit(self._h, C.byref(pr), C.byref(t))
        if rc == EAGAIN:
            return -1
        self._check(rc)
        self._keep[t.value] = kk
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """Result, or None while pending."""
        out = rot_vote_result()
        rc = self._L.rot_vote_poll(self._h, int(ticket), C.byref(out), int(timeout_us))
        if rc == PENDING:
            return None
        self._check(rc)
        self._keep.pop(ticket, None)
        return Result.of(out)

    def alg1(self, problems, peaks: int = 0, nms_angle: float = 0.0, min_count: int = 0):
        """rot_vote_alg1.  problems: list of (a, b[, samples[, accum_side[, accumulator]]]); accumulator: an
        int32 array or device tensor of accum_side^3 elements that receives the counts.  peaks = M > 0 also
        returns up to M peaks (greedy suppression within nms_angle) in each result's `peaks`.
        Returns Alg1Result list."""
        n = len(problems)
        arr = (rot_vote_alg1_problem * n)()
        keep = []
        pk_bufs = []
        for k, pr in enumerate(problems):
            a, b = pr[0], pr[1]
            J = int(pr[2]) if len(pr) > 2 else 0
            side = int(pr[3]) if len(pr) > 3 else 0
            acc = pr[4] if len(pr) > 4 else None
            pa, ka = _ptr(a)
            pb, kb = _ptr(b)
            if _nrows(b) != _nrows(a):
                raise ValueError("a and b differ in length")
            pacc = 0
            if acc is not None:
                if hasattr(acc, "data_ptr"):
                    if str(acc.dtype) != "torch.int32" or not acc.is_contiguous():
                        raise TypeError("accumulator must be a contiguous int32 tensor")
                    pacc = acc.data_ptr()
                else:
                    if acc.dtype != np.int32 or not acc.flags["C_CONTIGUOUS"]:
                        raise TypeError("accumulator must be a contiguous int32 array")
                    pacc = acc.ctypes.data
                need = (side or 360) ** 3
                if int(np.prod(acc.shape)) != need:
                    raise ValueError(f"accumulator must hold {need} elements")
            pbuf = (rot_vote_peak * max(1, int(peaks)))()
            pk_bufs.append(pbuf)
            arr[k] = rot_vote_alg1_problem(pa, pb, _nrows(a), J, side, pacc or None, int(peaks), int(min_count),
                                           float(nms_angle), C.cast(pbuf, C.c_void_p) if peaks else None)
            keep.append((ka, kb, acc))
        out = (rot_vote_alg1_result * n)()
        self._check(self._L.rot_vote_alg1(self._h, arr, n, out))
        return [Alg1Result.of(out[k], pk_bufs[k] if peaks else None) for k in range(n)]

    def alg1_raw(self, arr, n, out):
        """Calls rot_vote_alg1 on prepared ctypes arrays (for timing loops)."""
        return self._check(self._L.rot_vote_alg1(self._h, arr, n, out))

    def pose(self, x, y, mu: float, delta: float, grid_n: int = 0, levels: int = 0, min_length: float = 0.0,
             t_half: float = 0.0, t_cells: int = 0, pairs_out=None):
        """rot_vote_pose on one problem.  pairs_out: optional (a, b) float32 arrays or device tensors of
        shape [cap, 3] that receive the first cap kept unit pairs.  Returns PoseResult."""
        px, kx = _ptr(x)
        py, ky = _ptr(y)
        if _nrows(x) != _nrows(y):
            raise ValueError("x and y differ in length")
        pa = pb = None
        cap = 0
        if pairs_out is not None:
            oa, ob = pairs_out
            pa = oa.data_ptr() if hasattr(oa, "data_ptr") else oa.ctypes.data
            pb = ob.data_ptr() if hasattr(ob, "data_ptr") else ob.ctypes.data
            cap = int(oa.shape[0])
        pr = rot_vote_pose_problem(px, py, _nrows(x), float(mu), float(min_length), float(delta), int(grid_n),
                                   int(levels), float(t_half), int(t_cells), pa, pb, cap)
        out = rot_vote_pose_result()
        self._check(self._L.rot_vote_pose(self._h, C.byref(pr), 1, C.byref(out)))
        del kx, ky
        return PoseResult.of(out)

    def level_trace(self, problem: int, level: int, cap: int = 0):
        """(idx[n], count[n], kept_idx[k]) of one level of the last solve (keep_trace=1).
        cap = 0: the level's whole table (its size is queried first)."""
        if cap <= 0:
            nc0 = C.c_int64()
            self._check(self._L.rot_vote_level_trace(self._h, int(problem), int(level), None, None, 0,
                                                     C.byref(nc0), None, None))
            cap = max(1, nc0.value)
        idx = np.zeros(cap, np.int64)
        cnt = np.zeros(cap, np.int32)
        kept = np.zeros(64, np.int64)
        nc = C.c_int64()
        nk = C.c_int32()
        self._check(self._L.rot_vote_level_trace(self._h, int(problem), int(level), idx.ctypes.data,
                                                 cnt.ctypes.data, cap, C.byref(nc), kept.ctypes.data, C.byref(nk)))
        m = min(nc.value, cap)
        return idx[:m], cnt[:m], kept[:nk.value]

    def stage_times(self):
        """[(kind, level, ms, kernels)] of the last solve (context created with keep_trace=2):
        each stage's device time and the number of kernels it launched."""
        buf = (rot_vote_stage * 256)()
        n = C.c_int()
        self._check(self._L.rot_vote_stage_times(self._h, buf, 256, C.byref(n)))
        return [(STAGE_KIND[buf[k].kind], buf[k].level, buf[k].ms, buf[k].kernels) for k in range(min(n.value, 256))]

    def serve_spans(self, cap: int = 1 << 16):
        """[(t_start_ms, t_end_ms, wave, problems)] of every completed serving batch: device-time
        spans from the serving start, in completion order."""
        buf = (rot_vote_batch_span * cap)()
        n = C.c_int()
        self._check(self._L.rot_vote_serve_spans(self._h, buf, cap, C.byref(n)))
        return [(buf[k].t_start_ms, buf[k].t_end_ms, buf[k].wave, buf[k].problems) for k in range(min(n.value, cap))]

    def close(self):
        if getattr(self, "_h", None):
            self._L.rot_vote_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_static_args(a, b, cells, counts) -> None:
    """Shapes and devices of count_cells_static's tensors, checked before anything is
    launched: a and b [n, 3] with the same n, cells and counts 1-D of the same length,
    all on one CUDA device, the current one (raises ValueError otherwise)."""
    if a.dim() != 2 or a.shape[1] != 3 or tuple(b.shape) != tuple(a.shape):
        raise ValueError(f"a and b must both be [n, 3]; got {tuple(a.shape)} and {tuple(b.shape)}")
    if cells.dim() != 1 or tuple(counts.shape) != tuple(cells.shape):
        raise ValueError(f"cells and counts must be 1-D of one length; got {tuple(cells.shape)} and "
                         f"{tuple(counts.shape)}")
    devs = {(t.device.type, t.device.index) for t in (a, b, cells, counts)}
    if len(devs) != 1 or next(iter(devs))[0] != "cuda":
        raise ValueError(f"a, b, cells and counts must be on one CUDA device; got {sorted(map(str, devs))}")
    import torch
    if next(iter(devs))[1] != torch.cuda.current_device():
        raise ValueError(f"the tensors are on cuda:{next(iter(devs))[1]}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def count_cells_static(a, b, delta: float, grid_n: int, cells, counts, cuda_stream: int = 0) -> int:
    """rot_vote_count_cells_static: vote counts of the listed cells into `counts`
    with no device allocation.  a, b: device float32 [n, 3]; cells: device int64
    [ncells]; counts: device int32 [ncells].  Returns the rot_vote status."""
    for t, dt in ((a, "torch.float32"), (b, "torch.float32"), (cells, "torch.int64"), (counts, "torch.int32")):
        if str(t.dtype) != dt or not t.is_contiguous():
            raise TypeError(f"expected a contiguous {dt} device tensor")
    check_static_args(a, b, cells, counts)
    return int(load().rot_vote_count_cells_static(a.data_ptr(), b.data_ptr(), int(a.shape[0]), float(delta),
                                                  int(grid_n), cells.data_ptr(), int(cells.shape[0]),
                                                  counts.data_ptr(), int(cuda_stream) or None))
