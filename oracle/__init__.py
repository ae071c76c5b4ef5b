"""FP64 CPU oracle for the HMM recognition hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package. The product path (the
CUDA library and its Python binding in ``paper_1310_3322_gb300``) never does,
and the two share no code: inputs reach both only through the seeded
generators in ``paper_1310_3322_gb300.synth``, which hold none of the method's
arithmetic.

The paper (Sec. 2.7) names three HMM kernels -- Forward, Viterbi and
Baum-Welch -- without printing their equations, so the oracle follows the
textbook definitions (Rabiner 1989): forward log-likelihood (eqs. 19-21),
Viterbi score and path (eqs. 32-35), expected counts from the backward variable
(eqs. 24-25, 37-38) and re-estimation (eq. 40), all in FP64 log space in
``hmm_oracle.c``. ``softmax_rows`` (FP64 numpy) turns row logits into
probabilities for the gradient configurations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_LIB = None

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_SYMBOL = -5


def build(force: bool = False) -> str:
    """Compile hmm_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_LIBDIR, exist_ok=True)
    up_to_date = (
        os.path.exists(_LIBPATH)
        and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC)
        and os.path.getmtime(_LIBPATH) >= os.path.getmtime(os.path.join(_HERE, "hmm_oracle.h"))
    )
    if force or not up_to_date:
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _lib():
    global _LIB
    if _LIB is None:
        build()
        lib = ctypes.CDLL(_LIBPATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        ci = ctypes.c_int
        lib.orc_forward.argtypes = [ci, ci, ci, dp, dp, dp, ip, lp, ip, ci, ip, dp, ip, ci]
        lib.orc_forward.restype = ci
        lib.orc_viterbi.argtypes = [ci, ci, ci, dp, dp, dp, ip, lp, ip, ci, ip, dp, ip, ip, dp, ci]
        lib.orc_viterbi.restype = ci
        lib.orc_forward_backward.argtypes = [ci, ci, ci, dp, dp, dp, ip, lp, ip, ci, ip, dp, dp,
                                             dp, dp, dp, ci]
        lib.orc_forward_backward.restype = ci
        lib.orc_softmax_grad.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_softmax_grad.restype = None
        lib.orc_mstep.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_mstep.restype = None
        _LIB = lib
    return _LIB


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Params:
    """pi [K,N], A [K,N,N] (row = from-state), B [K,N,M], FP64 probabilities."""

    pi: np.ndarray
    A: np.ndarray
    B: np.ndarray

    @property
    def dims(self):
        K, N = self.pi.shape
        return K, N, self.B.shape[2]


def params(pi, A, B) -> Params:
    pi, A, B = _d(pi), _d(A), _d(B)
    if pi.ndim == 1:
        pi, A, B = pi[None], A[None], B[None]
    return Params(pi, A, B)


def softmax_rows(logits: np.ndarray) -> np.ndarray:
    """Row-wise softmax over the last axis in FP64: p = exp(x - max) / sum."""
    x = np.asarray(logits, dtype=np.float64)
    e = np.exp(x - x.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def _seqs(symbols, offsets, lengths, model_of_seq):
    sym = _i32(symbols)
    if sym.size == 0:
        sym = np.zeros(1, np.int32)
    off, ln = _i64(offsets), _i32(lengths)
    mos = None if model_of_seq is None else _i32(model_of_seq)
    return sym, off, ln, mos


def forward(p: Params, symbols, offsets, lengths, model_of_seq=None, nthreads=1):
    """log P(O_s | lambda_k): [S,K] (and argmax [S]) or [S] when labelled."""
    K, N, M = p.dims
    sym, off, ln, mos = _seqs(symbols, offsets, lengths, model_of_seq)
    S = ln.shape[0]
    out = np.empty((S,) if mos is not None else (S, K), np.float64)
    am = np.empty(S, np.int32)
    rc = _lib().orc_forward(K, N, M, _p(p.pi, ctypes.c_double), _p(p.A, ctypes.c_double),
                            _p(p.B, ctypes.c_double), _p(sym, ctypes.c_int32),
                            _p(off, ctypes.c_int64), _p(ln, ctypes.c_int32), S,
                            _p(mos, ctypes.c_int32), _p(out, ctypes.c_double),
                            _p(am, ctypes.c_int32), int(nthreads))
    if rc not in (ORC_OK, ORC_ERR_SYMBOL):
        raise ValueError(f"orc_forward rc={rc}")
    return (out, am, rc) if mos is None else (out, None, rc)


def viterbi(p: Params, symbols, offsets, lengths, model_of_seq=None, want_path=True,
            nthreads=1):
    """Returns (score [S,K] or [S], best_model [S], path [total] or None,
    margin [S], rc)."""
    K, N, M = p.dims
    sym, off, ln, mos = _seqs(symbols, offsets, lengths, model_of_seq)
    S = ln.shape[0]
    score = np.empty((S,) if mos is not None else (S, K), np.float64)
    best = np.empty(S, np.int32)
    path = np.full(max(int(np.asarray(symbols).size), 1), -1, np.int32) if want_path else None
    margin = np.empty(S, np.float64)
    rc = _lib().orc_viterbi(K, N, M, _p(p.pi, ctypes.c_double), _p(p.A, ctypes.c_double),
                            _p(p.B, ctypes.c_double), _p(sym, ctypes.c_int32),
                            _p(off, ctypes.c_int64), _p(ln, ctypes.c_int32), S,
                            _p(mos, ctypes.c_int32), _p(score, ctypes.c_double),
                            _p(best, ctypes.c_int32), _p(path, ctypes.c_int32),
                            _p(margin, ctypes.c_double), int(nthreads))
    if rc not in (ORC_OK, ORC_ERR_SYMBOL):
        raise ValueError(f"orc_viterbi rc={rc}")
    if path is not None:
        path = path[: int(np.asarray(symbols).size)]
    return score, best, path, margin, rc


def forward_backward(p: Params, symbols, offsets, lengths, model_of_seq=None, weight=None,
                     nthreads=1):
    """Returns (loglik, cnt_pi [K,N], cnt_A [K,N,N], cnt_B [K,N,M], rc)."""
    K, N, M = p.dims
    sym, off, ln, mos = _seqs(symbols, offsets, lengths, model_of_seq)
    S = ln.shape[0]
    w = None if weight is None else _d(weight)
    ll = np.empty((S,) if mos is not None else (S, K), np.float64)
    cpi = np.zeros((K, N))
    cA = np.zeros((K, N, N))
    cB = np.zeros((K, N, M))
    rc = _lib().orc_forward_backward(
        K, N, M, _p(p.pi, ctypes.c_double), _p(p.A, ctypes.c_double), _p(p.B, ctypes.c_double),
        _p(sym, ctypes.c_int32), _p(off, ctypes.c_int64), _p(ln, ctypes.c_int32), S,
        _p(mos, ctypes.c_int32), _p(w, ctypes.c_double), _p(ll, ctypes.c_double),
        _p(cpi, ctypes.c_double), _p(cA, ctypes.c_double), _p(cB, ctypes.c_double),
        int(nthreads))
    if rc not in (ORC_OK, ORC_ERR_SYMBOL):
        raise ValueError(f"orc_forward_backward rc={rc}")
    return ll, cpi, cA, cB, rc


def softmax_grad(p: Params, cpi, cA, cB):
    """Gradient of sum_s w_s log P w.r.t. the row logits: g = C - p * rowsum(C)."""
    K, N, M = p.dims
    cpi, cA, cB = _d(cpi), _d(cA), _d(cB)
    gpi, gA, gB = np.empty_like(cpi), np.empty_like(cA), np.empty_like(cB)
    dp = ctypes.c_double
    _lib().orc_softmax_grad(K, N, M, _p(p.pi, dp), _p(p.A, dp), _p(p.B, dp), _p(cpi, dp),
                            _p(cA, dp), _p(cB, dp), _p(gpi, dp), _p(gA, dp), _p(gB, dp))
    return gpi, gA, gB


def mstep(p: Params, cpi, cA, cB) -> Params:
    """Baum-Welch re-estimation (Rabiner eq. 40) from expected counts."""
    K, N, M = p.dims
    cpi, cA, cB = _d(cpi), _d(cA), _d(cB)
    out = Params(np.empty_like(p.pi), np.empty_like(p.A), np.empty_like(p.B))
    dp = ctypes.c_double
    _lib().orc_mstep(K, N, M, _p(p.pi, dp), _p(p.A, dp), _p(p.B, dp), _p(cpi, dp), _p(cA, dp),
                     _p(cB, dp), _p(out.pi, dp), _p(out.A, dp), _p(out.B, dp))
    return out
