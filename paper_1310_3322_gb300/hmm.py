"""Thin Python binding of the C-ABI in ``include/hmm.h`` (argument marshalling
only: every step of the hot path runs in ``libhmmgb.so``'s CUDA kernels).

The functions carry the C names. They take CUDA ``torch.Tensor`` arguments
(PyTorch is used for device memory and streams), allocate the outputs and the
caller-side workspace with torch, pass raw device pointers to the library on
the current torch stream, and raise ``HmmError`` on a negative return code.
There is no CPU fallback: if the library is missing or fails to load, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass, replace
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhmmgb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "hmm.h")

HMM_OK = 0
HMM_ERR_ARG = -1
HMM_ERR_CUDA = -2
HMM_ERR_WORKSPACE = -3
HMM_ERR_UNSUPPORTED = -4
HMM_ERR_DEVICE = -5
HMM_STATUS_SYMBOL = 0x1
HMM_STATUS_PARAM = 0x2
HMM_STATUS_SEQ = 0x4
HMM_STATUS_TIMEOUT = 0x8

HMM_FP32, HMM_BF16_MMA, HMM_TF32_MMA, HMM_AUTO = 0, 1, 2, 3
HMM_OP_FORWARD, HMM_OP_VITERBI, HMM_OP_FORWARD_BACKWARD, HMM_OP_FORWARD_SCAN = 0, 1, 2, 3
HMM_TUNE_VITERBI_PATHS = 3
HMM_TUNE_FB_RANGES = 4


class HmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class hmm_dims_t(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("N", ctypes.c_int32), ("M", ctypes.c_int32)]


class hmm_seqs_t(ctypes.Structure):
    _fields_ = [("symbols", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("lengths", ctypes.c_void_p), ("model_of_seq", ctypes.c_void_p),
                ("S", ctypes.c_int32), ("max_len", ctypes.c_int32),
                ("total_obs", ctypes.c_int64), ("model_base", ctypes.c_void_p),
                ("model_span", ctypes.c_int32)]


_lib = None
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIG = {
    "hmm_workspace_size": (_I32, [hmm_dims_t, ctypes.POINTER(hmm_seqs_t), _I32,
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "hmm_max_states": (_I32, [_I32, _I32]),
    "hmm_forward_backward_workspace_size": (_I32, [hmm_dims_t, ctypes.POINTER(hmm_seqs_t), _I32,
                                                   ctypes.POINTER(ctypes.c_size_t)]),
    "hmm_forward": (_I32, [hmm_dims_t, _VP, _VP, _VP, ctypes.POINTER(hmm_seqs_t), _I32, _VP,
                           _VP, _VP, ctypes.c_size_t, _VP]),
    "hmm_forward_static": (_I32, [hmm_dims_t, _VP, _VP, _VP, ctypes.POINTER(hmm_seqs_t), _I32,
                                  _VP, _VP, _VP]),
    "hmm_forward_scan": (_I32, [hmm_dims_t, _VP, _VP, _VP, ctypes.POINTER(hmm_seqs_t), _I32, _VP,
                                _VP, _VP, ctypes.c_size_t, _VP]),
    "hmm_forward_scan_workspace_size": (_I32, [hmm_dims_t, ctypes.POINTER(hmm_seqs_t), _I32,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "hmm_viterbi": (_I32, [hmm_dims_t, _VP, _VP, _VP, ctypes.POINTER(hmm_seqs_t), _VP, _VP, _VP,
                           _VP, ctypes.c_size_t, _VP]),
    "hmm_forward_backward": (_I32, [hmm_dims_t, _VP, _VP, _VP, ctypes.POINTER(hmm_seqs_t), _VP,
                                    _I32, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "hmm_softmax_rows": (_I32, [hmm_dims_t, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "hmm_softmax_grad": (_I32, [hmm_dims_t, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "hmm_mstep": (_I32, [hmm_dims_t, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "hmm_adam_step": (_I32, [ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP, _VP]),
    "hmm_get_device_status": (_I32, [_VP, _VP, ctypes.POINTER(_I32)]),
    "hmm_set_tuning": (_I32, [_I32, _I32, _I32]),
    "hmm_get_tuning": (_I32, [_I32, _I32, ctypes.POINTER(_I32)]),
    "hmm_tuning_candidates": (_I32, [_I32, _I32, ctypes.POINTER(_I32), _I32]),
    "hmm_last_error": (ctypes.c_char_p, []),
    "hmm_fma_probe": (_I32, [_I32, _I32, ctypes.c_int64, _I32, _VP, _VP]),
    "hmm_set_wait_limit": (_I32, [ctypes.c_int64]),
    "hmm_get_wait_limit": (ctypes.c_uint32, []),
    "hmm_timing_enable": (_I32, [_I32]),
    "hmm_timing_reset": (_I32, []),
    "hmm_timing_read": (_I32, [_I32, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_double)]),
}

TIMING_KINDS = ("setup", "forward", "viterbi_scores", "viterbi_paths", "adjoint",
                "count_reduce", "softmax_rows", "softmax_grad", "adam", "mstep", "scan_chunks",
                "scan_combine", "adjoint_pass")


def lib():
    """The loaded ``libhmmgb.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def header_symbols() -> list:
    """Every function the public header declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:const\s+)?\w+\*?\s+\*?(hmm_\w+)\s*\(", text, re.M)))


def hmm_last_error() -> str:
    return (lib().hmm_last_error() or b"").decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise HmmError(rc, hmm_last_error())
    return rc


def _torch():
    import torch
    return torch


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous (dense, row-major)")
    return t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


@dataclass
class Sequences:
    """Ragged batch on the device: ``symbols`` int32 [total_obs], ``offsets``
    int64 [S], ``lengths`` int32 [S], optional ``model_of_seq`` int32 [S];
    ``max_len`` bounds every length (host value). ``model_base`` int32 [S] with
    ``model_span`` scores sequence s against models [base[s], base[s] + span)
    only (one HMM set per role)."""

    symbols: object
    offsets: object
    lengths: object
    max_len: int
    model_of_seq: object = None
    model_base: object = None
    model_span: int = 0

    @property
    def S(self) -> int:
        return int(self.lengths.shape[0])

    @property
    def total_obs(self) -> int:
        return int(self.symbols.shape[0])

    def labelled(self, model_of_seq) -> "Sequences":
        return replace(self, model_of_seq=model_of_seq)

    def all_models(self) -> "Sequences":
        return replace(self, model_of_seq=None, model_base=None, model_span=0)

    def model_sets(self, model_base, span: int) -> "Sequences":
        """Every sequence against its own set of ``span`` consecutive models."""
        return replace(self, model_of_seq=None, model_base=model_base, model_span=int(span))

    @property
    def span(self) -> Optional[int]:
        """Models each sequence is scored against in all-models mode (None:
        all K)."""
        return self.model_span if self.model_base is not None else None

    def c(self) -> hmm_seqs_t:
        return hmm_seqs_t(_ptr(self.symbols), _ptr(self.offsets), _ptr(self.lengths),
                          _ptr(self.model_of_seq), self.S, int(self.max_len), self.total_obs,
                          _ptr(self.model_base), int(self.model_span))

    @staticmethod
    def from_numpy(symbols, offsets, lengths, model_of_seq=None, device="cuda",
                   max_len: Optional[int] = None) -> "Sequences":
        torch = _torch()
        lengths = np.asarray(lengths, np.int32)
        ml = int(lengths.max()) if (max_len is None and lengths.size) else (max_len or 0)
        sym = np.asarray(symbols, np.int32)
        return Sequences(
            symbols=torch.from_numpy(sym.copy() if sym.size else np.zeros(0, np.int32)).to(device),
            offsets=torch.from_numpy(np.asarray(offsets, np.int64).copy()).to(device),
            lengths=torch.from_numpy(lengths.copy()).to(device),
            max_len=ml,
            model_of_seq=None if model_of_seq is None else
            torch.from_numpy(np.asarray(model_of_seq, np.int32).copy()).to(device))


class Workspace:
    """Caller-owned device scratch buffer for the library (grown on demand by
    torch; the library itself never allocates)."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes: int):
        torch = _torch()
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


_default_ws = {}


def _ws(workspace, device):
    if workspace is not None:
        return workspace
    torch = _torch()
    device = torch.device(device)
    if device.type == "cuda" and device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    key = str(device)
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def _dims(pi, B) -> hmm_dims_t:
    K, N = int(pi.shape[0]), int(pi.shape[1])
    return hmm_dims_t(K, N, int(B.shape[2]))


def hmm_workspace_size(dims: hmm_dims_t, seqs: Sequences, op: int) -> int:
    out = ctypes.c_size_t(0)
    c = seqs.c()
    _check(lib().hmm_workspace_size(dims, ctypes.byref(c), op, ctypes.byref(out)))
    return int(out.value)


def hmm_forward_backward_workspace_size(dims: hmm_dims_t, seqs: Sequences, precision: int) -> int:
    out = ctypes.c_size_t(0)
    c = seqs.c()
    _check(lib().hmm_forward_backward_workspace_size(dims, ctypes.byref(c), precision,
                                                     ctypes.byref(out)))
    return int(out.value)


def hmm_max_states(op: int, precision: int = HMM_FP32) -> int:
    return _check(lib().hmm_max_states(op, precision))


def hmm_forward(pi, A, B, seqs: Sequences, precision: int = HMM_FP32, want_argmax=True,
                loglik=None, argmax=None, workspace: Optional[Workspace] = None, stream=None):
    """log P(O_s | lambda_k): [S,K] (+ argmax [S]) or [S] when labelled."""
    torch = _torch()
    dims = _dims(pi, B)
    S, K = seqs.S, (seqs.span or dims.K)
    all_models = seqs.model_of_seq is None
    if loglik is None:
        loglik = torch.empty((S, K) if all_models else (S,), dtype=torch.float32, device=pi.device)
    if all_models and want_argmax and argmax is None:
        argmax = torch.empty(S, dtype=torch.int32, device=pi.device)
    ws = _ws(workspace, pi.device)
    nbytes = hmm_workspace_size(dims, seqs, HMM_OP_FORWARD)
    buf = ws.get(nbytes)
    c = seqs.c()
    _check(lib().hmm_forward(dims, _ptr(pi), _ptr(A), _ptr(B), ctypes.byref(c), precision,
                             _ptr(loglik), _ptr(argmax if all_models else None), _ptr(buf),
                             buf.numel(), _stream(stream)))
    return loglik, (argmax if all_models else None)


def hmm_forward_scan_workspace_size(dims: hmm_dims_t, seqs: Sequences, chunk: int = 0) -> int:
    out = ctypes.c_size_t(0)
    c = seqs.c()
    _check(lib().hmm_forward_scan_workspace_size(dims, ctypes.byref(c), int(chunk),
                                                 ctypes.byref(out)))
    return int(out.value)


def hmm_forward_scan(pi, A, B, seqs: Sequences, chunk: int = 0, want_argmax=True, loglik=None,
                     argmax=None, workspace: Optional[Workspace] = None, stream=None):
    """Parallel-in-time forward (chunk products + ordered combine): the
    outputs of hmm_forward with HMM_FP32, for batches of few long sequences.
    ``chunk`` = steps per chunk (0: automatic)."""
    torch = _torch()
    dims = _dims(pi, B)
    S, K = seqs.S, (seqs.span or dims.K)
    all_models = seqs.model_of_seq is None
    if loglik is None:
        loglik = torch.empty((S, K) if all_models else (S,), dtype=torch.float32, device=pi.device)
    if all_models and want_argmax and argmax is None:
        argmax = torch.empty(S, dtype=torch.int32, device=pi.device)
    ws = _ws(workspace, pi.device)
    buf = ws.get(hmm_forward_scan_workspace_size(dims, seqs, chunk))
    c = seqs.c()
    _check(lib().hmm_forward_scan(dims, _ptr(pi), _ptr(A), _ptr(B), ctypes.byref(c), int(chunk),
                                  _ptr(loglik), _ptr(argmax if all_models else None), _ptr(buf),
                                  buf.numel(), _stream(stream)))
    return loglik, (argmax if all_models else None)


def hmm_forward_static(pi, A, B, seqs: Sequences, precision: int = HMM_FP32, want_argmax=True,
                       loglik=None, argmax=None, stream=None):
    """hmm_forward without a workspace: the library's fixed scratch array is
    used instead (see include/hmm.h). Outputs as in hmm_forward."""
    torch = _torch()
    dims = _dims(pi, B)
    S, K = seqs.S, (seqs.span or dims.K)
    all_models = seqs.model_of_seq is None
    if loglik is None:
        loglik = torch.empty((S, K) if all_models else (S,), dtype=torch.float32, device=pi.device)
    if all_models and want_argmax and argmax is None:
        argmax = torch.empty(S, dtype=torch.int32, device=pi.device)
    c = seqs.c()
    _check(lib().hmm_forward_static(dims, _ptr(pi), _ptr(A), _ptr(B), ctypes.byref(c), precision,
                                    _ptr(loglik), _ptr(argmax if all_models else None),
                                    _stream(stream)))
    return loglik, (argmax if all_models else None)


def hmm_viterbi(pi, A, B, seqs: Sequences, want_path=True, want_best=True, score=None,
                best_model=None, path=None, workspace: Optional[Workspace] = None, stream=None):
    """(score [S,K] or [S], best_model [S], path [total_obs])."""
    torch = _torch()
    dims = _dims(pi, B)
    S, K = seqs.S, (seqs.span or dims.K)
    all_models = seqs.model_of_seq is None
    if score is None:
        score = torch.empty((S, K) if all_models else (S,), dtype=torch.float32, device=pi.device)
    if want_best and best_model is None:
        best_model = torch.empty(S, dtype=torch.int32, device=pi.device)
    if want_path and path is None:
        path = torch.empty(max(seqs.total_obs, 1), dtype=torch.int32, device=pi.device)
    ws = _ws(workspace, pi.device)
    buf = ws.get(hmm_workspace_size(dims, seqs, HMM_OP_VITERBI))
    c = seqs.c()
    _check(lib().hmm_viterbi(dims, _ptr(pi), _ptr(A), _ptr(B), ctypes.byref(c), _ptr(score),
                             _ptr(best_model), _ptr(path), _ptr(buf), buf.numel(),
                             _stream(stream)))
    if path is not None:
        path = path[: seqs.total_obs]
    return score, best_model, path


def hmm_forward_backward(pi, A, B, seqs: Sequences, weight=None, precision: int = HMM_FP32,
                         loglik=None, counts=None, workspace: Optional[Workspace] = None,
                         stream=None):
    """(loglik, cnt_pi [K,N], cnt_A [K,N,N], cnt_B [K,N,M])."""
    torch = _torch()
    dims = _dims(pi, B)
    S, K, N, M = seqs.S, dims.K, dims.N, dims.M
    all_models = seqs.model_of_seq is None
    if loglik is None:
        loglik = torch.empty((S, K) if all_models else (S,), dtype=torch.float32, device=pi.device)
    if counts is None:
        counts = (torch.empty((K, N), dtype=torch.float32, device=pi.device),
                  torch.empty((K, N, N), dtype=torch.float32, device=pi.device),
                  torch.empty((K, N, M), dtype=torch.float32, device=pi.device))
    ws = _ws(workspace, pi.device)
    buf = ws.get(hmm_forward_backward_workspace_size(dims, seqs, precision))
    c = seqs.c()
    _check(lib().hmm_forward_backward(dims, _ptr(pi), _ptr(A), _ptr(B), ctypes.byref(c),
                                      _ptr(weight), precision, _ptr(loglik), _ptr(counts[0]),
                                      _ptr(counts[1]), _ptr(counts[2]), _ptr(buf), buf.numel(),
                                      _stream(stream)))
    return (loglik,) + tuple(counts)


def hmm_softmax_rows(lpi, lA, lB, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = (torch.empty_like(lpi), torch.empty_like(lA), torch.empty_like(lB))
    _check(lib().hmm_softmax_rows(_dims(lpi, lB), _ptr(lpi), _ptr(lA), _ptr(lB), _ptr(out[0]),
                                  _ptr(out[1]), _ptr(out[2]), _stream(stream)))
    return out


def hmm_softmax_grad(pi, A, B, cpi, cA, cB, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = (torch.empty_like(cpi), torch.empty_like(cA), torch.empty_like(cB))
    _check(lib().hmm_softmax_grad(_dims(pi, B), _ptr(pi), _ptr(A), _ptr(B), _ptr(cpi), _ptr(cA),
                                  _ptr(cB), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                  _stream(stream)))
    return out


def hmm_mstep(pi, A, B, cpi, cA, cB, out=None, stream=None):
    """Baum-Welch re-estimation from expected counts; ``out=(pi, A, B)`` updates
    the parameters in place."""
    torch = _torch()
    if out is None:
        out = (torch.empty_like(pi), torch.empty_like(A), torch.empty_like(B))
    _check(lib().hmm_mstep(_dims(pi, B), _ptr(pi), _ptr(A), _ptr(B), _ptr(cpi), _ptr(cA),
                           _ptr(cB), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream)))
    return out


def hmm_adam_step(param, grad, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0,
                  step_counter=None, stream=None):
    """Adam on ``param`` in place; ``step_counter`` is a device int32 tensor
    of one element (steps taken so far), advanced by the call."""
    if step_counter is None:
        raise ValueError("step_counter (a device int32 tensor) is required")
    _check(lib().hmm_adam_step(param.numel(), _ptr(param), _ptr(grad), _ptr(m), _ptr(v),
                               float(lr), float(beta1), float(beta2), float(eps),
                               float(grad_scale), _ptr(step_counter), _stream(stream)))


def hmm_get_device_status(workspace, stream=None) -> int:
    """Device status word of the last call that used ``workspace`` (a
    ``Workspace`` or its buffer); synchronises the stream."""
    buf = workspace.buf if isinstance(workspace, Workspace) else workspace
    st = ctypes.c_int32(0)
    rc = lib().hmm_get_device_status(_ptr(buf), _stream(stream), ctypes.byref(st))
    if rc not in (HMM_OK, HMM_ERR_DEVICE):
        _check(rc)
    return int(st.value)


def default_workspace(device="cuda") -> Workspace:
    return _ws(None, device)


def hmm_set_tuning(op: int, n_pad: int, lanes: int):
    _check(lib().hmm_set_tuning(op, n_pad, lanes))


def hmm_get_tuning(op: int, n_pad: int) -> int:
    v = ctypes.c_int32(0)
    _check(lib().hmm_get_tuning(op, n_pad, ctypes.byref(v)))
    return int(v.value)


def hmm_tuning_candidates(op: int, n_pad: int) -> list:
    buf = (ctypes.c_int32 * 16)()
    n = _check(lib().hmm_tuning_candidates(op, n_pad, buf, 16))
    return [int(buf[i]) for i in range(min(n, 16))]


def hmm_fma_probe(blocks: int, threads: int, iters: int, mode: int, out, stream=None):
    """FP32 FMA throughput probe; returns the flop count of the launch."""
    _check(lib().hmm_fma_probe(int(blocks), int(threads), int(iters), int(mode), _ptr(out),
                               _stream(stream)))
    return blocks * threads * iters * 32 * (2 if mode == 1 else 1)


def hmm_set_wait_limit(polls: int = -1):
    """Polls before a tensor-core kernel's step wait gives up (< 0: the
    default; 0: every such wait gives up at once)."""
    _check(lib().hmm_set_wait_limit(int(polls)))


def hmm_get_wait_limit() -> int:
    return int(lib().hmm_get_wait_limit())


def hmm_timing_enable(on: bool = True):
    _check(lib().hmm_timing_enable(1 if on else 0))


def hmm_timing_reset():
    _check(lib().hmm_timing_reset())


def hmm_timing_read() -> dict:
    """{kind: (launches, total_ms)} since the last reset (synchronises)."""
    out = {}
    for i, name in enumerate(TIMING_KINDS):
        n, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
        _check(lib().hmm_timing_read(i, ctypes.byref(n), ctypes.byref(ms)))
        out[name] = (int(n.value), float(ms.value))
    return out
