"""GB300-native discrete-HMM recognition hot path (arXiv 1310.3322, Sec. 2.7).

Scaled-forward log-likelihoods, Viterbi decoding and the forward-backward
adjoint of ragged symbol sequences against K per-activity HMMs, as
hand-written sm_103a CUDA behind the C-ABI in ``include/hmm.h``.
``paper_1310_3322_gb300.hmm`` is the thin Python binding (argument marshalling
only); ``paper_1310_3322_gb300.synth`` draws the seeded synthetic workloads.
"""
__all__ = ["hmm", "synth"]
