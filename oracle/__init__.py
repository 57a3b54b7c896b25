"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package; the product path (``paper_1512_01641_gb300``) never
does, and shares no code with it.

``oracle.c`` holds the definitions (overlap counts, features, sigmoid
similarity, Needleman-Wunsch fill and traceback with the UP > LEFT > DIAG tie
rule, soft log-sum-exp alignment with its adjoint).  This module builds it
with gcc on first use and marshals NumPy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MOVE_DIAG, MOVE_UP, MOVE_LEFT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (plain gcc, portable flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            i8p = np.ctypeslib.ndpointer(np.int8, flags="C")
            L.oracle_counts.argtypes = [i32p, C.c_int64, i32p, C.c_int64, i32p, i32p,
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
            L.oracle_nw_fill.argtypes = [C.c_int64, C.c_int64, f64p, C.c_double, f64p]
            L.oracle_nw_traceback.argtypes = [C.c_int64, C.c_int64, C.c_double, f64p, i8p]
            L.oracle_nw_traceback.restype = C.c_int64
            L.oracle_soft_nw.argtypes = [C.c_int64, C.c_int64, f64p, C.c_double, C.c_double,
                                         f64p, f64p, f64p, C.POINTER(C.c_double)]
            L.oracle_features.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int64, f64p]
            L.oracle_similarity.argtypes = [f64p, f64p, C.c_double]
            L.oracle_similarity.restype = C.c_double
            L.oracle_mine.argtypes = [C.c_int64, i64p, i64p, i64p, i32p, i64p, i64p, i32p,
                                      i32p, i32p, f64p, C.c_double, C.c_double,
                                      i64p, f64p, i64p, i32p, i32p, f64p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            L.oracle_mine.restype = C.c_int
            _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# single sentence pair
# ---------------------------------------------------------------------------
def counts(src, tgt, dic) -> tuple[int, int]:
    """(ms, mt) of one source/target sentence pair."""
    ms, mt = C.c_int32(), C.c_int32()
    s, t = _c(src, np.int32), _c(tgt, np.int32)
    lib().oracle_counts(s, len(s), t, len(t), _c(dic.off, np.int32), _c(dic.tgt, np.int32),
                        C.byref(ms), C.byref(mt))
    return ms.value, mt.value


def features(ms, mt, ls, lt) -> np.ndarray:
    f = np.zeros(4, np.float64)
    lib().oracle_features(int(ms), int(mt), int(ls), int(lt), f)
    return f


def similarity(f, w, b) -> float:
    return lib().oracle_similarity(_c(f, np.float64), _c(w, np.float64), float(b))


# ---------------------------------------------------------------------------
# alignment on an explicit similarity matrix
# ---------------------------------------------------------------------------
def nw(s, p):
    """Hard NW on an N x M similarity matrix.  Returns (H, moves, diag) where H is
    (N+1)x(M+1), moves are in walk order from (N,M), and diag is the ascending
    list of 0-based (i, j) cells taken diagonally."""
    s = _c(np.atleast_2d(s), np.float64) if np.size(s) else np.zeros(np.shape(s), np.float64)
    N, M = s.shape
    H = np.zeros((N + 1) * (M + 1), np.float64)
    L = lib()
    L.oracle_nw_fill(N, M, s.reshape(-1) if s.size else np.zeros(1), float(p), H)
    mv = np.zeros(N + M + 1, np.int8)
    n = L.oracle_nw_traceback(N, M, float(p), H, mv)
    mv = mv[:n]
    diag = []
    i = j = 0
    for m in mv[::-1]:
        if m == MOVE_DIAG:
            diag.append((i, j))
            i += 1
            j += 1
        elif m == MOVE_UP:
            i += 1
        else:
            j += 1
    return H.reshape(N + 1, M + 1), mv, diag


def soft_nw(s, p, gamma):
    """Soft NW: returns (V, E, dV/dp); V is (N+1)x(M+1), E = dV(N,M)/ds (N x M)."""
    s = _c(s, np.float64)
    N, M = s.shape
    V = np.zeros((N + 1) * (M + 1), np.float64)
    Q = np.zeros_like(V)
    E = np.zeros(max(N * M, 1), np.float64)
    dp = C.c_double()
    lib().oracle_soft_nw(N, M, s.reshape(-1) if s.size else np.zeros(1), float(p), float(gamma),
                         V, E, Q, C.byref(dp))
    return V.reshape(N + 1, M + 1), E[:N * M].reshape(N, M), dp.value


def path_score(s, p, diag) -> float:
    """Score of the monotone alignment whose diagonal cells are ``diag``:
    sum of their similarities minus p per unmatched sentence.  Raises if the
    cells are not strictly increasing in both coordinates."""
    s = np.asarray(s, np.float64)
    N, M = s.shape
    tot = 0.0
    pi = pj = -1
    for (i, j) in diag:
        if not (i > pi and j > pj and 0 <= i < N and 0 <= j < M):
            raise ValueError(f"not a monotone alignment at ({i},{j})")
        tot += s[i, j]
        pi, pj = i, j
    return tot - p * (N + M - 2 * len(diag))


# ---------------------------------------------------------------------------
# whole batches
# ---------------------------------------------------------------------------
def mine(batch, w, b, gap, thr, pairs=None, n_threads=None, want_counts=False, want_sim=False):
    """Mine the listed pairs of a synth.Batch.

    Returns a dict with, per listed pair: ``score`` (H(N,M)), ``diag`` (list of
    (i, j, s) on the optimal path, ascending), ``links`` (the diag cells with
    s >= thr) and optionally ``counts`` (N x M x 2 int32: ms, mt) and ``sim``
    (N x M float64 similarities)."""
    src, tgt, dic = batch.src, batch.tgt, batch.dic
    if pairs is None:
        pairs = np.arange(batch.n_pairs)
    pairs = _c(pairs, np.int64)
    N = src.doc_sizes()[pairs]
    M = tgt.doc_sizes()[pairs]
    cap = np.minimum(N, M)
    out_off = np.zeros(len(pairs) + 1, np.int64)
    np.cumsum(cap, out=out_off[1:])
    tot = int(out_off[-1])
    score = np.zeros(len(pairs), np.float64)
    nd = np.zeros(len(pairs), np.int64)
    di = np.zeros(max(tot, 1), np.int32)
    dj = np.zeros(max(tot, 1), np.int32)
    ds = np.zeros(max(tot, 1), np.float64)
    cnt = None
    sim = None
    cell_off = np.zeros(len(pairs) + 1, np.int64)
    np.cumsum(N * M, out=cell_off[1:])
    if want_counts:
        cnt = np.zeros(max(int(cell_off[-1]) * 2, 1), np.int32)
    if want_sim:
        sim = np.zeros(max(int(cell_off[-1]), 1), np.float64)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    used = lib().oracle_mine(len(pairs), pairs,
                             _c(src.doc_sent_off, np.int64), _c(src.sent_tok_off, np.int64), _c(src.tok, np.int32),
                             _c(tgt.doc_sent_off, np.int64), _c(tgt.sent_tok_off, np.int64), _c(tgt.tok, np.int32),
                             _c(dic.off, np.int32), _c(dic.tgt, np.int32),
                             _c(w, np.float64), float(b), float(gap),
                             out_off, score, nd, di, dj, ds,
                             cnt.ctypes.data if cnt is not None else None,
                             sim.ctypes.data if sim is not None else None,
                             cell_off.ctypes.data,
                             int(n_threads))
    res = {"score": score, "diag": [], "links": [], "threads": used}
    for k in range(len(pairs)):
        a = out_off[k]
        n = nd[k]
        d = [(int(di[a + t]), int(dj[a + t]), float(ds[a + t])) for t in range(n)]
        res["diag"].append(d)
        res["links"].append([x for x in d if x[2] >= thr])
    if want_counts:
        res["counts"] = [cnt[2 * cell_off[k]:2 * cell_off[k + 1]].reshape(N[k], M[k], 2)
                         for k in range(len(pairs))]
    if want_sim:
        res["sim"] = [sim[cell_off[k]:cell_off[k + 1]].reshape(N[k], M[k]) for k in range(len(pairs))]
    return res
