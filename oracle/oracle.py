"""ctypes wrapper of the C++ oracle.  Numpy in, numpy out; all arrays on the host."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        P = C.c_void_p
        i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
        _lib.orc_priors.argtypes = [i32, P, i32, P]
        _lib.orc_bp.argtypes = [i32, i32, i64, P, P, P, i64, P, i32, f64, i32, i32, i32, i32,
                                P, P, P, P]
        _lib.orc_gf2_rank.argtypes = [i32, i32, P]
        _lib.orc_gf2_rank.restype = i32
        _lib.orc_gf2_solve.argtypes = [i32, i32, P, P, P, P]
        _lib.orc_gf2_solve.restype = i32
        _lib.orc_osd0.argtypes = [i32, i32, i64, P, P, P, P, P]
        _lib.orc_osd0.restype = i32
        _lib.orc_lsd.argtypes = [i32, i32, i64, P, P, i64, P, P, P, i32, i32, i32, i32, P, P, P,
                                 P, P]
        _lib.orc_decode.argtypes = [i32, i32, i64, P, P, P, i64, P, i32, f64, i32, i32, i32, i32,
                                    P, P, P, P, P]
        _lib.orc_logical_failures.argtypes = [i32, i32, P, i64, P, i32, P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _coo(h):
    h = np.asarray(h, dtype=np.uint8)
    r, c = np.nonzero(h)
    return h.shape[0], h.shape[1], np.ascontiguousarray(r, np.int32), np.ascontiguousarray(c, np.int32)


def _probs(probs, n):
    p = np.asarray(probs, dtype=np.float64)
    if p.ndim == 0:
        p = np.full(n, float(p))
    return np.ascontiguousarray(p)


def priors(probs, precision: int = 0):
    p = np.ascontiguousarray(np.asarray(probs, dtype=np.float64))
    out = np.empty_like(p)
    lib().orc_priors(p.shape[0], _p(p), precision, _p(out))
    return out


def bp(h, probs, syndromes, iters, alpha=0.625, method=0, early_exit=1, precision=0, nthreads=0):
    """Returns (llr [shots][n] float64, hard [shots][n] u8, iters_used [shots], converged [shots])."""
    m, n, r, c = _coo(h)
    s = np.ascontiguousarray(np.atleast_2d(syndromes), dtype=np.uint8)
    shots = s.shape[0]
    p = _probs(probs, n)
    llr = np.empty((shots, n), np.float64)
    hard = np.empty((shots, n), np.uint8)
    used = np.empty(shots, np.int32)
    conv = np.empty(shots, np.uint8)
    rc = lib().orc_bp(m, n, r.size, _p(r), _p(c), _p(p), shots, _p(s), iters, alpha, method,
                      early_exit, precision, nthreads, _p(llr), _p(hard), _p(used), _p(conv))
    if rc:
        raise ValueError("orc_bp: invalid matrix")
    return llr, hard, used, conv


def gf2_rank(a) -> int:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8) & 1)
    return int(lib().orc_gf2_rank(a.shape[0], a.shape[1], _p(a)))


def gf2_solve(a, b):
    """Returns (solvable, x, pivots): x supported on the greedy column basis (index order)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8) & 1)
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint8) & 1)
    x = np.zeros(a.shape[1], np.uint8)
    piv = np.zeros(a.shape[1], np.uint8)
    ok = lib().orc_gf2_solve(a.shape[0], a.shape[1], _p(a), _p(b), _p(x), _p(piv))
    return bool(ok), x, piv


def osd0(h, syndrome, llr):
    m, n, r, c = _coo(h)
    s = np.ascontiguousarray(syndrome, dtype=np.uint8)
    l = np.ascontiguousarray(llr, dtype=np.float64)
    out = np.zeros(n, np.uint8)
    ok = lib().orc_osd0(m, n, r.size, _p(r), _p(c), _p(s), _p(l), _p(out))
    return bool(ok), out


def lsd(h, syndromes, llrs, order=0, probs=None, single_cluster=False, nthreads=0, labels=False,
        osd_cs=-1):
    """LSD on given soft information.  order = mu (LSD-mu, App. D); osd_cs = -1 reprocesses
    each cluster with OSD-E of order mu, osd_cs = w >= 0 with the combination sweep of
    order w (needs mu >= 1).

    Returns dict(corrections, status, nu, kappa, steps[, det_lab, fault_lab]).
    """
    m, n, r, c = _coo(h)
    s = np.ascontiguousarray(np.atleast_2d(syndromes), dtype=np.uint8)
    shots = s.shape[0]
    l = np.ascontiguousarray(np.atleast_2d(llrs), dtype=np.float64)
    assert l.shape == (shots, n)
    p = None if probs is None else _probs(probs, n)
    corr = np.zeros((shots, n), np.uint8)
    st = np.zeros(shots, np.uint8)
    info = np.zeros((shots, 3), np.int32)
    dl = np.zeros((shots, m), np.int32) if labels else None
    fl = np.zeros((shots, n), np.int32) if labels else None
    rc = lib().orc_lsd(m, n, r.size, _p(r), _p(c), shots, _p(s), _p(l), _p(p), order, osd_cs,
                       int(single_cluster), nthreads, _p(corr), _p(st), _p(info), _p(dl), _p(fl))
    if rc:
        raise ValueError("orc_lsd: invalid arguments")
    out = dict(corrections=corr, status=st, nu=info[:, 0], kappa=info[:, 1], steps=info[:, 2])
    if labels:
        out["det_lab"] = dl
        out["fault_lab"] = fl
    return out


def decode(h, probs, syndromes, bp_iters, alpha=0.625, lsd_order=0, precision=1, nthreads=0,
           want_llr=False, osd_cs=-1):
    """BP then LSD.  Returns dict(corrections, status, bp_iters, nu, kappa, steps[, llr])."""
    m, n, r, c = _coo(h)
    s = np.ascontiguousarray(np.atleast_2d(syndromes), dtype=np.uint8)
    shots = s.shape[0]
    p = _probs(probs, n)
    corr = np.zeros((shots, n), np.uint8)
    st = np.zeros(shots, np.uint8)
    used = np.zeros(shots, np.int32)
    info = np.zeros((shots, 3), np.int32)
    llr = np.zeros((shots, n), np.float64) if want_llr else None
    rc = lib().orc_decode(m, n, r.size, _p(r), _p(c), _p(p), shots, _p(s), bp_iters, alpha,
                          lsd_order, osd_cs, precision, nthreads, _p(corr), _p(st), _p(used),
                          _p(info), _p(llr))
    if rc:
        raise ValueError("orc_decode: invalid arguments")
    out = dict(corrections=corr, status=st, bp_iters=used, nu=info[:, 0], kappa=info[:, 1],
               steps=info[:, 2])
    if want_llr:
        out["llr"] = llr
    return out


def logical_failures(hz, residuals, nthreads=0):
    hz = np.ascontiguousarray(np.asarray(hz, dtype=np.uint8))
    res = np.ascontiguousarray(np.atleast_2d(residuals), dtype=np.uint8)
    fail = np.zeros(res.shape[0], np.uint8)
    lib().orc_logical_failures(hz.shape[0], hz.shape[1], _p(hz), res.shape[0], _p(res), nthreads,
                               _p(fail))
    return fail
