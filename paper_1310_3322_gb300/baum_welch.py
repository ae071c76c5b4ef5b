"""Baum-Welch re-estimation loop on the GPU (Sec. 2.7 "Baum-Welch"; Rabiner
1989 eqs. 37-40): alternate the library's forward-backward E-step
(``hmm_forward_backward``: expected counts and log-likelihoods) and its
M-step (``hmm_mstep``: row-normalised counts, in place), iterating until the
total log-likelihood stops rising.

Every arithmetic step runs in the library's kernels; this module only holds
the buffers, captures ``chunk`` iterations in one CUDA graph and checks
convergence on the host between replays.
"""
from __future__ import annotations

from typing import List, Optional

from . import hmm


def baum_welch(pi, A, B, seqs: hmm.Sequences, max_iters: int = 50, tol: float = 1e-7,
               chunk: int = 5, precision: int = hmm.HMM_AUTO, graph: bool = True,
               workspace: Optional[hmm.Workspace] = None) -> List[float]:
    """Re-estimates ``pi`` [K,N], ``A`` [K,N,N] and ``B`` [K,N,M] (device FP32
    probability tensors) in place on the sequences (usually labelled:
    ``seqs.model_of_seq`` gives each sequence's model). Returns the total
    log-likelihood sum_s log P(O_s | lambda) before each iteration that ran.
    Runs at most ``max_iters`` iterations in groups of ``chunk`` (one
    CUDA-graph replay each when ``graph``; the first group runs eagerly) and
    stops after a group whose last iteration raised the total by no more than
    ``tol`` times its magnitude."""
    import torch
    K, N, M = int(pi.shape[0]), int(pi.shape[1]), int(B.shape[2])
    dev = pi.device
    rows = seqs.S if seqs.model_of_seq is not None else seqs.S * K
    hist = torch.empty((chunk, rows), dtype=torch.float32, device=dev)
    counts = (torch.empty((K, N), device=dev), torch.empty((K, N, N), device=dev),
              torch.empty((K, N, M), device=dev))
    ws = workspace if workspace is not None else hmm.default_workspace(dev)
    ws.get(hmm.hmm_workspace_size(hmm.hmm_dims_t(K, N, M), seqs,
                                  hmm.HMM_OP_FORWARD_BACKWARD))

    def one(i):
        hmm.hmm_forward_backward(pi, A, B, seqs, precision=precision, loglik=hist[i],
                                 counts=counts, workspace=ws)
        hmm.hmm_mstep(pi, A, B, *counts, out=(pi, A, B))

    g = None
    history: List[float] = []
    while len(history) < max_iters:
        n = min(chunk, max_iters - len(history))
        if graph and n == chunk and history:
            if g is None:
                side = torch.cuda.Stream(device=dev)
                side.wait_stream(torch.cuda.current_stream(dev))
                g = torch.cuda.CUDAGraph()
                with torch.cuda.stream(side):
                    with torch.cuda.graph(g, stream=side):
                        for i in range(chunk):
                            one(i)
                torch.cuda.current_stream(dev).wait_stream(side)
            g.replay()  # (capture recorded the chunk without running it)
        else:
            for i in range(n):
                one(i)
        history += hist[:n].double().sum(dim=1).cpu().tolist()
        if len(history) >= 2 and history[-1] - history[-2] <= tol * abs(history[-1]):
            break
    return history
