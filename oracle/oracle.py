"""ctypes wrapper around the C oracle (rv_oracle.c). Test infrastructure only.

Every function here forwards to the C code, which follows the method step by
step in FP64 (App. A pair matrices, the cell grid and covering radius, the
threshold sin^2(delta + r), the vote, the (score desc, idx asc) ranking, the
octant children and the Eq. (stack) eigenvector fit with its refit rule).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "pair_M", "pair_S", "quad", "quat_to_R", "cell_exists", "cell_geom", "tau",
    "level_cells", "vote_cells", "rank", "jacobi4", "canonical", "solve", "OracleResult",
    "AMBIG", "cell_of_point", "fit_cell", "alg1_basis", "alg1_cell", "alg1_table", "alg1", "alg1_centre",
    "alg1_peaks", "pose_pairs", "pose_translation", "pose", "using_library",
]

AMBIG = 1e-6

_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


class _Result(C.Structure):
    _fields_ = [("q", C.c_double * 4), ("R", C.c_double * 9), ("best_count", C.c_int32),
                ("inliers", C.c_int32), ("best_cell", C.c_int64), ("tests", C.c_int64),
                ("ambiguous", C.c_int64), ("status", C.c_int32), ("refits", C.c_int32)]


class _Trace(C.Structure):
    _fields_ = [("cap", C.c_int64), ("ncells", C.c_void_p), ("idx", C.c_void_p), ("count", C.c_void_p),
                ("amb", C.c_void_p), ("tau", C.c_void_p), ("topk_idx", C.c_void_p),
                ("topk_score", C.c_void_p), ("nkept", C.c_void_p)]


def _configure(L):
    """Argument and result types of the C entry points."""
    L.rvo_pair_M.argtypes = [_f32p, _f32p, _f64p]
    L.rvo_pair_S.argtypes = [_f32p, _f32p, _f64p]
    L.rvo_quad.argtypes = [_f64p, _f64p]
    L.rvo_quad.restype = C.c_double
    L.rvo_quat_to_R.argtypes = [_f64p, _f64p]
    L.rvo_cell_exists.argtypes = [C.c_int, C.c_int64, C.c_int64, C.c_int64]
    L.rvo_cell_exists.restype = C.c_int
    L.rvo_cell_geom.argtypes = [C.c_int, C.c_int64, C.c_int64, C.c_int64, _f64p, C.POINTER(C.c_double)]
    L.rvo_cell_geom_chart.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, _f64p,
                                      C.POINTER(C.c_double)]
    L.rvo_tau.argtypes = [C.c_double, C.c_double, C.c_double]
    L.rvo_tau.restype = C.c_double
    L.rvo_level_cells.argtypes = [C.c_int, C.c_void_p]
    L.rvo_level_cells.restype = C.c_int64
    L.rvo_vote_cells.argtypes = [_f32p, _f32p, C.c_int64, C.c_double, C.c_int, C.c_int, _i64p, C.c_int64,
                                 _i32p, _i32p, _f64p, C.c_int]
    L.rvo_vote_cells.restype = C.c_int
    L.rvo_rank.argtypes = [_i32p, _f64p, _i64p, C.c_int64, C.c_int64, C.c_int, C.c_int64, _i64p, _f64p]
    L.rvo_rank.restype = C.c_int64
    L.rvo_jacobi4.argtypes = [_f64p, _f64p, _f64p]
    L.rvo_canonical.argtypes = [_f64p]
    L.rvo_solve.argtypes = [_f32p, _f32p, C.c_int64, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                            C.c_int, C.c_int, C.c_int, C.POINTER(_Result), C.POINTER(_Trace)]
    L.rvo_solve.restype = C.c_int
    L.rvo_fit_cell.argtypes = [_f32p, _f32p, C.c_int64, C.c_double, C.c_int, C.c_int, C.c_int64, C.c_int,
                               C.POINTER(_Result)]
    L.rvo_fit_cell.restype = C.c_int
    L.rvo_alg1_basis.argtypes = [_f32p, _f32p, _f64p, _f64p]
    L.rvo_alg1_basis.restype = C.c_int
    L.rvo_alg1_cell.argtypes = [_f64p, _f64p, C.c_double, C.c_double, C.c_int]
    L.rvo_alg1_cell.restype = C.c_int64
    L.rvo_alg1_table.argtypes = [C.c_int, _f64p]
    L.rvo_alg1_table.restype = None
    L.rvo_alg1.argtypes = [_f32p, _f32p, C.c_int64, _f64p, C.c_int, C.c_int, _i32p, C.POINTER(C.c_int64),
                           C.POINTER(C.c_int32), _f64p]
    L.rvo_alg1.restype = C.c_int64
    L.rvo_alg1_centre.argtypes = [C.c_int, C.c_int64, _f64p]
    L.rvo_alg1_centre.restype = None
    L.rvo_alg1_peaks.argtypes = [_i32p, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_double, _i64p, _i32p, _f64p,
                                 C.POINTER(C.c_int32)]
    L.rvo_alg1_peaks.restype = C.c_int
    L.rvo_pose_pairs.argtypes = [_f32p, _f32p, C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                 C.c_int64]
    L.rvo_pose_pairs.restype = C.c_int64
    L.rvo_pose_translation.argtypes = [_f32p, _f32p, C.c_int64, _f64p, C.c_double, C.c_int, _f64p,
                                       C.POINTER(C.c_int64)]
    L.rvo_pose_translation.restype = C.c_int32
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(_build.build()))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Inside the block every wrapper calls the oracle library at `path` (a
    build of a modified copy of rv_oracle.c), then the regular build again:
    for the tests that plant a mistake in the oracle and check that a pin
    catches it."""
    global _lib
    saved = lib()
    _lib = _configure(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _v3(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(3))


def pair_M(a, b) -> np.ndarray:
    """M = L(a)^T L'(b) of App. A (4x4)."""
    M = np.zeros(16)
    lib().rvo_pair_M(_v3(a), _v3(b), M)
    return M.reshape(4, 4)


def pair_S(a, b) -> np.ndarray:
    """S = (I - M)/2 = I - P (4x4)."""
    S = np.zeros(16)
    lib().rvo_pair_S(_v3(a), _v3(b), S)
    return S.reshape(4, 4)


def quad(S, q) -> float:
    return float(lib().rvo_quad(np.ascontiguousarray(S, dtype=np.float64).reshape(16),
                                np.ascontiguousarray(q, dtype=np.float64)))


def quat_to_R(q) -> np.ndarray:
    R = np.zeros(9)
    lib().rvo_quat_to_R(np.ascontiguousarray(q, dtype=np.float64), R)
    return R.reshape(3, 3)


def cell_exists(n, ix, iy, iz) -> bool:
    return bool(lib().rvo_cell_exists(int(n), int(ix), int(iy), int(iz)))


def cell_geom(n, ix, iy, iz, chart: int = 0):
    """(q_cell[4], chord) of cell (ix, iy, iz) of the n^3 grid; chart 0 orthographic, 1 stereographic."""
    q = np.zeros(4)
    ch = C.c_double()
    lib().rvo_cell_geom_chart(int(chart), int(n), int(ix), int(iy), int(iz), q, C.byref(ch))
    return q, ch.value


def tau(delta: float, chord: float) -> float:
    return float(lib().rvo_tau(np.sin(delta), np.cos(delta), chord))


def level_cells(n: int) -> np.ndarray:
    cnt = lib().rvo_level_cells(int(n), None)
    out = np.zeros(cnt, dtype=np.int64)
    lib().rvo_level_cells(int(n), out.ctypes.data)
    return out


def cell_of_point(n: int, v) -> int:
    """Linear index of the n^3 cell whose box contains the vector part v."""
    h = 2.0 / n
    i = [min(n - 1, max(0, int(np.floor((float(v[k]) + 1.0) / h)))) for k in range(3)]
    return (i[2] * n + i[1]) * n + i[0]


def _f32_pairs(a, b):
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)
    b = np.ascontiguousarray(b, dtype=np.float32).reshape(-1, 3)
    assert a.shape == b.shape
    return a, b


def vote_cells(a, b, delta: float, n_side: int, cells, nthreads: int = 1, chart: int = 0):
    """(count, ambiguous, tau) for each linear cell index in `cells`."""
    a, b = _f32_pairs(a, b)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    cnt = np.zeros(len(cells), dtype=np.int32)
    amb = np.zeros(len(cells), dtype=np.int32)
    tau_ = np.zeros(len(cells), dtype=np.float64)
    rc = lib().rvo_vote_cells(a.reshape(-1), b.reshape(-1), a.shape[0], float(delta), int(n_side), int(chart),
                              cells, len(cells), cnt, amb, tau_, int(nthreads))
    assert rc == 0
    return cnt, amb, tau_


def rank(count, tau_, idx, n_pairs: int, rank_mode: int = 0, k: int = 16):
    """Positions of the top-k cells in (score desc, idx asc) order, and their scores."""
    count = np.ascontiguousarray(count, dtype=np.int32)
    tau_ = np.ascontiguousarray(tau_, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    pos = np.zeros(k, dtype=np.int64)
    sc = np.zeros(k, dtype=np.float64)
    kk = lib().rvo_rank(count, tau_, idx, len(idx), int(n_pairs), int(rank_mode), int(k), pos, sc)
    return pos[:kk], sc[:kk]


def jacobi4(A):
    """(eigenvalues ascending, eigenvector columns) of a symmetric 4x4."""
    ev = np.zeros(4)
    V = np.zeros(16)
    lib().rvo_jacobi4(np.ascontiguousarray(A, dtype=np.float64).reshape(16), ev, V)
    return ev, V.reshape(4, 4)


def canonical(q) -> np.ndarray:
    q = np.array(q, dtype=np.float64)
    lib().rvo_canonical(q)
    return q


@dataclasses.dataclass
class OracleResult:
    q: np.ndarray
    R: np.ndarray
    best_count: int
    inliers: int
    best_cell: int
    tests: int
    ambiguous: int
    status: int
    refits: int
    levels: list  # per level: dict(idx, count, amb, tau, topk_idx, topk_score)


def solve(a, b, delta: float, grid_n: int, levels: int = 0, top_k: int = 16, rank_mode: int = 0,
          refit_iters: int = 8, nthreads: int = 1, trace: bool = True, chart: int = 0) -> OracleResult:
    """The full path: vote on each level, rank, subdivide, fit (chart 0 orthographic, 1 stereographic)."""
    a, b = _f32_pairs(a, b)
    L = lib()
    res = _Result()
    tr_p = None
    keep = []
    if trace:
        cap = int(L.rvo_level_cells(int(grid_n), None))
        cap = max(cap, 8 * top_k)
        nl = levels + 1
        arrs = dict(ncells=np.zeros(nl, np.int64), idx=np.zeros(nl * cap, np.int64),
                    count=np.zeros(nl * cap, np.int32), amb=np.zeros(nl * cap, np.int32),
                    tau=np.zeros(nl * cap, np.float64), topk_idx=np.zeros(nl * top_k, np.int64),
                    topk_score=np.zeros(nl * top_k, np.float64), nkept=np.zeros(nl, np.int64))
        tr = _Trace(cap, *(arrs[k].ctypes.data for k in
                           ("ncells", "idx", "count", "amb", "tau", "topk_idx", "topk_score", "nkept")))
        tr_p = C.byref(tr)
        keep = [tr, arrs]
    L.rvo_solve(a.reshape(-1), b.reshape(-1), a.shape[0], float(delta), int(grid_n), int(levels), int(top_k),
                int(rank_mode), int(refit_iters), int(chart), int(nthreads), C.byref(res), tr_p)
    per_level = []
    if trace:
        arrs = keep[1]
        cap = keep[0].cap
        for lev in range(levels + 1):
            nc = int(arrs["ncells"][lev])
            nk = int(arrs["nkept"][lev])
            sl = slice(lev * cap, lev * cap + nc)
            per_level.append(dict(
                idx=arrs["idx"][sl].copy(), count=arrs["count"][sl].copy(), amb=arrs["amb"][sl].copy(),
                tau=arrs["tau"][sl].copy(),
                topk_idx=arrs["topk_idx"][lev * top_k: lev * top_k + nk].copy(),
                topk_score=arrs["topk_score"][lev * top_k: lev * top_k + nk].copy()))
    return OracleResult(q=np.array(res.q[:]), R=np.array(res.R[:]).reshape(3, 3), best_count=res.best_count,
                        inliers=res.inliers, best_cell=res.best_cell, tests=res.tests,
                        ambiguous=res.ambiguous, status=res.status, refits=res.refits, levels=per_level)


def fit_cell(a, b, delta: float, n_side: int, idx: int, refit_iters: int = 8, chart: int = 0) -> OracleResult:
    """The fit alone (step 8), from winning cell `idx` of the n_side grid."""
    a, b = _f32_pairs(a, b)
    res = _Result()
    lib().rvo_fit_cell(a.reshape(-1), b.reshape(-1), a.shape[0], float(delta), int(n_side), int(chart), int(idx),
                       int(refit_iters), C.byref(res))
    return OracleResult(q=np.array(res.q[:]), R=np.array(res.R[:]).reshape(3, 3), best_count=res.best_count,
                        inliers=res.inliers, best_cell=res.best_cell, tests=res.tests, ambiguous=res.ambiguous,
                        status=res.status, refits=res.refits, levels=[])


def default_threads() -> int:
    return max(1, (os.cpu_count() or 1))


# ---- Alg. 1 (Sec. 4.3.2): sampled circles, stereographic projection, counting grid ----

def alg1_basis(a, b):
    """(ok, q_b1, q_b2) of pair (a, b) (Sec. 4.1)."""
    q1 = np.zeros(4)
    q2 = np.zeros(4)
    ok = lib().rvo_alg1_basis(_v3(a), _v3(b), q1, q2)
    return bool(ok), q1, q2


def alg1_cell(q1, q2, cj: float, sj: float, n: int) -> int:
    return int(lib().rvo_alg1_cell(np.ascontiguousarray(q1, dtype=np.float64), np.ascontiguousarray(q2, dtype=np.float64),
                                   float(cj), float(sj), int(n)))


def alg1_table(J: int) -> np.ndarray:
    """[J, 2] (cos(alpha_j / 2), sin(alpha_j / 2)), alpha_j = -pi + 2 pi j / J."""
    cs = np.zeros(2 * J)
    lib().rvo_alg1_table(int(J), cs)
    return cs.reshape(J, 2)


def alg1(a, b, J: int, n: int):
    """Alg. 1 on one problem: (acc [n^3] int32, best_idx, best_count, q, samples cast)."""
    a, b = _f32_pairs(a, b)
    cs = np.ascontiguousarray(alg1_table(J).reshape(-1))
    acc = np.zeros(int(n) ** 3, dtype=np.int32)
    bi = C.c_int64()
    bc = C.c_int32()
    q = np.zeros(4)
    cast = lib().rvo_alg1(a.reshape(-1), b.reshape(-1), a.shape[0], cs, int(J), int(n), acc, C.byref(bi), C.byref(bc), q)
    return acc, int(bi.value), int(bc.value), q, int(cast)


def alg1_centre(n: int, idx: int) -> np.ndarray:
    """Rotation (canonical quaternion) of the centre of accumulator cell idx."""
    q = np.zeros(4)
    lib().rvo_alg1_centre(int(n), int(idx), q)
    return q


def alg1_peaks(acc, n: int, M: int, theta: float, min_count: int = 1, kmax: int = 16384):
    """Multiple rotations (Sec. 4.4): (idx[k], count[k], q[k, 4], T) of up to M peaks by greedy NMS."""
    acc = np.ascontiguousarray(acc, dtype=np.int32)
    pidx = np.zeros(max(1, M), np.int64)
    pcnt = np.zeros(max(1, M), np.int32)
    pq = np.zeros((max(1, M), 4))
    T = C.c_int32()
    k = lib().rvo_alg1_peaks(acc, int(n), int(M), int(min_count), int(kmax), float(theta), pidx, pcnt,
                             pq.reshape(-1), C.byref(T))
    return pidx[:k], pcnt[:k], pq[:k], int(T.value)


# ---- rigid pose (Sec. 4.5): pairwise length check, rotation vote, translation vote ----

def pose_pairs(x, y, mu: float, lmin: float = 0.0, want_pairs: bool = True):
    """(a[K, 3], b[K, 3]) float32 unit pairs (m/|m|, n/|n|) of the kept i < j pairs, lexicographic order."""
    x, y = _f32_pairs(x, y)
    n = x.shape[0]
    L = lib()
    k = int(L.rvo_pose_pairs(x.reshape(-1), y.reshape(-1), n, float(mu), float(lmin), None, None, 0))
    if not want_pairs:
        return k
    a = np.zeros((max(k, 1), 3), np.float32)
    b = np.zeros((max(k, 1), 3), np.float32)
    L.rvo_pose_pairs(x.reshape(-1), y.reshape(-1), n, float(mu), float(lmin), a.ctypes.data, b.ctypes.data, k)
    return a[:k], b[:k]


def pose_translation(x, y, R, L_half: float = 5.0, G: int = 400):
    """(t[3] cell centre, cell index, count) of the translation vote with rotation R."""
    x, y = _f32_pairs(x, y)
    t = np.zeros(3)
    cell = C.c_int64()
    cnt = lib().rvo_pose_translation(x.reshape(-1), y.reshape(-1), x.shape[0],
                                     np.ascontiguousarray(R, dtype=np.float64).reshape(9), float(L_half), int(G), t,
                                     C.byref(cell))
    return t, int(cell.value), int(cnt)


def pose(x, y, mu: float, delta: float, grid_n: int, levels: int, lmin: float = 0.0, L_half: float = 5.0,
         G: int = 400, chart: int = 0, nthreads: int = 1):
    """The whole pose pipeline: kept pairs, the rotation solve over them, the translation vote.
    Returns (OracleResult of the rotation, t, cell, count, kept pairs)."""
    a, b = pose_pairs(x, y, mu, lmin)
    r = solve(a, b, delta, grid_n=grid_n, levels=levels, chart=chart, nthreads=nthreads, trace=False)
    t, cell, cnt = pose_translation(x, y, r.R, L_half, G)
    return r, t, cell, cnt, len(a)
