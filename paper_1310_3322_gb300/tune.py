"""Autotuner for the lanes-per-pair choice of each kernel and the number of
segment ranges per pair of the SIMT adjoint.

For a given batch and model shape it times every instantiated candidate of
the forward, Viterbi-score, Viterbi-path and adjoint kernels (and, for the
adjoint, every number of segment ranges, timed together with the count
reduction, whose input grows with it) with the library's CUDA-event timing,
keeps the fastest, installs it with hmm_set_tuning, and caches the choice in a
JSON file keyed by the GPU name, kernel, padded state count, number of models
and coarse buckets of the batch size and maximum length. Every candidate
computes the same recursion, so the choice affects only speed.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

from . import hmm

KERNEL_OF = {hmm.HMM_OP_FORWARD: "forward", hmm.HMM_OP_VITERBI: "viterbi_scores",
             hmm.HMM_TUNE_VITERBI_PATHS: "viterbi_paths",
             hmm.HMM_OP_FORWARD_BACKWARD: "adjoint",
             hmm.HMM_TUNE_FB_RANGES: "adjoint_ranges"}
# timing kinds summed for each tuned op
TIMED = {hmm.HMM_OP_FORWARD_BACKWARD: ("adjoint", "adjoint_pass"),
         hmm.HMM_TUNE_FB_RANGES: ("adjoint", "adjoint_pass", "count_reduce")}
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hmmgb_tuning.json")


def n_pad(N: int) -> int:
    for p in (4, 8, 16, 32, 64):
        if N <= p:
            return p
    raise ValueError(N)


def _bucket(x: int) -> int:
    return 0 if x <= 0 else int(math.log2(x))


def key(gpu: str, op: int, N: int, K: int, S: int, max_len: int) -> str:
    return f"{gpu}|{KERNEL_OF[op]}|np{n_pad(N)}|K{K}|S{_bucket(S)}|T{_bucket(max_len)}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _run(op, pi, A, B, seqs, labelled, ws):
    if op == hmm.HMM_OP_FORWARD:
        hmm.hmm_forward(pi, A, B, seqs, workspace=ws)
    elif op in (hmm.HMM_OP_VITERBI, hmm.HMM_TUNE_VITERBI_PATHS):
        hmm.hmm_viterbi(pi, A, B, seqs, workspace=ws)
    else:  # the adjoint: lanes per pair or segment ranges
        hmm.hmm_forward_backward(pi, A, B, labelled, workspace=ws)


def autotune(pi, A, B, seqs, labelled=None, ops=None, repeats: int = 3,
             cache: Optional[str] = DEFAULT_CACHE, force: bool = False) -> dict:
    """Times every candidate for each op on this batch; installs and returns
    {kernel: {"lanes": best, "ms": {lanes: ms}}}."""
    import torch
    K, N = int(pi.shape[0]), int(pi.shape[1])
    gpu = torch.cuda.get_device_name(pi.device)
    ops = ops or [hmm.HMM_OP_FORWARD, hmm.HMM_OP_VITERBI, hmm.HMM_TUNE_VITERBI_PATHS,
                  hmm.HMM_OP_FORWARD_BACKWARD, hmm.HMM_TUNE_FB_RANGES]
    table = _load(cache) if cache else {}
    ws = hmm.Workspace(pi.device)
    out = {}
    for op in ops:
        if op in (hmm.HMM_OP_FORWARD_BACKWARD, hmm.HMM_TUNE_FB_RANGES) and (
                labelled is None or N > hmm.hmm_max_states(hmm.HMM_OP_FORWARD_BACKWARD)):
            continue
        np_ = n_pad(N)
        cands = hmm.hmm_tuning_candidates(op, np_)
        if not cands:
            continue
        k = key(gpu, op, N, K, seqs.S, seqs.max_len)
        if not force and k in table and table[k]["lanes"] in cands:
            hmm.hmm_set_tuning(op, np_, table[k]["lanes"])
            out[KERNEL_OF[op]] = dict(table[k], cached=True)
            continue
        times = {}
        for g in cands:
            hmm.hmm_set_tuning(op, np_, g)
            _run(op, pi, A, B, seqs, labelled, ws)        # warm
            torch.cuda.synchronize()
            hmm.hmm_timing_reset()
            hmm.hmm_timing_enable(True)
            for _ in range(repeats):
                _run(op, pi, A, B, seqs, labelled, ws)
            torch.cuda.synchronize()
            tr = hmm.hmm_timing_read()
            hmm.hmm_timing_enable(False)
            times[g] = sum(tr[kd][1] / max(tr[kd][0], 1) for kd in TIMED.get(op, (KERNEL_OF[op],)))
        best = min(times, key=times.get)
        hmm.hmm_set_tuning(op, np_, best)
        table[k] = {"lanes": best, "ms": {str(g): v for g, v in times.items()}}
        out[KERNEL_OF[op]] = dict(table[k], cached=False)
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return out
