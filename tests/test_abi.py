"""The C-ABI library loads, exports every symbol include/hmm.h declares, and
rejects bad arguments on the host before touching a device (CPU only: no call
here reaches a kernel launch)."""
import ctypes
import subprocess

import pytest

from paper_1310_3322_gb300 import hmm


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return hmm.lib()


def test_every_declared_symbol_is_exported(lib):
    names = hmm.header_symbols()
    assert len(names) >= 13
    out = subprocess.run(["nm", "-D", "--defined-only", hmm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_library_has_no_torch_dependency(lib):
    out = subprocess.run(["ldd", hmm.LIB_PATH], capture_output=True, text=True).stdout
    assert "torch" not in out and "c10" not in out


def test_sm103a_code_only():
    from paper_1310_3322_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def _fake(i):
    # 256-byte aligned dummy addresses; host-side checks fail before any use
    return 0x7f0000000000 + 0x100000 * i


def _seqs(S=4, max_len=10, total=40, mos=False):
    return hmm.hmm_seqs_t(_fake(1), _fake(2), _fake(3), _fake(4) if mos else None, S, max_len,
                          total)


def test_workspace_size_is_host_only_and_monotone(lib):
    d = hmm.hmm_dims_t(10, 16, 32)
    sizes = []
    for S in (0, 1, 100, 4096):
        q = _seqs(S=S, total=S * 300)
        out = ctypes.c_size_t()
        assert lib.hmm_workspace_size(d, ctypes.byref(q), hmm.HMM_OP_VITERBI, ctypes.byref(out)) == 0
        sizes.append(out.value)
    assert sizes == sorted(sizes) and sizes[0] >= 256 and sizes[0] % 256 == 0
    q = _seqs(S=100)
    out = ctypes.c_size_t()
    assert lib.hmm_workspace_size(d, ctypes.byref(q), 7, ctypes.byref(out)) == hmm.HMM_ERR_ARG
    # N up to 128 for the forward, the adjoint (tensor cores above 64) and
    # Viterbi; the tensor-core adjoint takes M <= 256
    big = hmm.hmm_dims_t(4, 128, 256)
    assert lib.hmm_workspace_size(big, ctypes.byref(q), hmm.HMM_OP_FORWARD, ctypes.byref(out)) == 0
    assert out.value >= 4 * 128 * 128 * 4
    # Viterbi to 128 states (one warp per pair above 64), uint8 backpointers
    assert lib.hmm_workspace_size(big, ctypes.byref(q), hmm.HMM_OP_VITERBI,
                                  ctypes.byref(out)) == 0
    assert out.value >= q.total_obs * 128
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(4, 129, 8), ctypes.byref(q), hmm.HMM_OP_VITERBI,
                                  ctypes.byref(out)) == hmm.HMM_ERR_UNSUPPORTED
    assert lib.hmm_max_states(hmm.HMM_OP_VITERBI, hmm.HMM_FP32) == 128
    assert lib.hmm_workspace_size(big, ctypes.byref(q), hmm.HMM_OP_FORWARD_BACKWARD,
                                  ctypes.byref(out)) == 0
    # per-tile count slots and per-CTA checkpoint buffers
    assert out.value >= (100 // 128 + 1 + 4) * 128 * (1 + 128 + 256) * 4
    # above 128 states: per-step rows of both passes (4 buffers of K * total_obs * N_pad)
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(4, 129, 8), ctypes.byref(q),
                                  hmm.HMM_OP_FORWARD_BACKWARD, ctypes.byref(out)) == 0
    assert out.value >= 4 * 4 * q.total_obs * 256 * 4
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(1, 300, 200), ctypes.byref(q),
                                  hmm.HMM_OP_FORWARD_BACKWARD, ctypes.byref(out)) \
        == hmm.HMM_ERR_UNSUPPORTED
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(1, 513, 8), ctypes.byref(q),
                                  hmm.HMM_OP_FORWARD_BACKWARD, ctypes.byref(out)) \
        == hmm.HMM_ERR_UNSUPPORTED
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(4, 65, 300), ctypes.byref(q),
                                  hmm.HMM_OP_FORWARD_BACKWARD, ctypes.byref(out)) \
        == hmm.HMM_ERR_UNSUPPORTED
    # the forward goes to 512 states (BF16 A^T images of every model included)
    wide = hmm.hmm_dims_t(3, 512, 64)
    assert lib.hmm_workspace_size(wide, ctypes.byref(q), hmm.HMM_OP_FORWARD, ctypes.byref(out)) == 0
    assert out.value >= 3 * 512 * 512 * (4 + 2)
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(3, 513, 64), ctypes.byref(q), hmm.HMM_OP_FORWARD,
                                  ctypes.byref(out)) == hmm.HMM_ERR_UNSUPPORTED


def _forward(lib, dims, seqs, pi=_fake(5), loglik=_fake(8), ws=_fake(9), ws_bytes=1 << 30,
             precision=hmm.HMM_FP32):
    return lib.hmm_forward(dims, pi, _fake(6), _fake(7), ctypes.byref(seqs), precision, loglik,
                           None, ws, ws_bytes, None)


def test_forward_argument_errors(lib):
    d = hmm.hmm_dims_t(2, 4, 8)
    q = _seqs()
    assert _forward(lib, d, q, pi=None) == hmm.HMM_ERR_ARG
    assert "pi/A/B" in hmm.hmm_last_error()
    assert _forward(lib, d, q, loglik=None) == hmm.HMM_ERR_ARG
    assert _forward(lib, hmm.hmm_dims_t(0, 4, 8), q) == hmm.HMM_ERR_ARG
    assert _forward(lib, hmm.hmm_dims_t(2, 65, 8), q) == hmm.HMM_ERR_UNSUPPORTED
    assert _forward(lib, d, q, precision=9) == hmm.HMM_ERR_ARG
    assert _forward(lib, d, q, precision=hmm.HMM_BF16_MMA) == hmm.HMM_ERR_UNSUPPORTED
    assert _forward(lib, d, q, ws=None) == hmm.HMM_ERR_WORKSPACE
    assert _forward(lib, d, q, ws=_fake(9) + 4) == hmm.HMM_ERR_WORKSPACE
    assert _forward(lib, d, q, ws_bytes=16) == hmm.HMM_ERR_WORKSPACE
    assert "need" in hmm.hmm_last_error()
    neg = hmm.hmm_seqs_t(_fake(1), _fake(2), _fake(3), None, -1, 10, 40)
    assert _forward(lib, d, neg) == hmm.HMM_ERR_ARG
    mis = hmm.hmm_seqs_t(_fake(1), _fake(2) + 4, _fake(3), None, 4, 10, 40)
    assert _forward(lib, d, mis) == hmm.HMM_ERR_ARG
    # S == 0 is a no-op that returns before any CUDA call
    assert _forward(lib, d, _seqs(S=0)) == hmm.HMM_OK


def test_viterbi_and_adjoint_argument_errors(lib):
    d = hmm.hmm_dims_t(2, 4, 8)
    q = _seqs()
    assert lib.hmm_viterbi(d, _fake(5), _fake(6), _fake(7), ctypes.byref(q), None, None, None,
                           _fake(9), 1 << 30, None) == hmm.HMM_ERR_ARG
    assert lib.hmm_forward_backward(d, _fake(5), _fake(6), _fake(7), ctypes.byref(q), None,
                                    hmm.HMM_FP32, _fake(8), None, _fake(11), _fake(12),
                                    _fake(9), 1 << 30, None) == hmm.HMM_ERR_ARG
    big = hmm.hmm_dims_t(2, 65, 8)
    assert lib.hmm_forward_backward(big, _fake(5), _fake(6), _fake(7), ctypes.byref(q), None,
                                    hmm.HMM_FP32, _fake(8), _fake(10), _fake(11), _fake(12),
                                    _fake(9), 1 << 30, None) == hmm.HMM_ERR_UNSUPPORTED
    # adjoint shared-memory limit: very long sequences with many symbols
    huge = hmm.hmm_seqs_t(_fake(1), _fake(2), _fake(3), None, 4, 2_000_000, 8_000_000)
    assert lib.hmm_forward_backward(hmm.hmm_dims_t(2, 32, 2048), _fake(5), _fake(6), _fake(7),
                                    ctypes.byref(huge), None, hmm.HMM_FP32, _fake(8), _fake(10),
                                    _fake(11), _fake(12), _fake(9), 1 << 40, None) \
        == hmm.HMM_ERR_UNSUPPORTED
    assert lib.hmm_adam_step(10, _fake(1), _fake(2), _fake(3), _fake(4), 0.1, 0.9, 0.999, 1e-8,
                             1.0, None, None) == hmm.HMM_ERR_ARG
    assert lib.hmm_adam_step(0, None, None, None, None, 0.1, 0.9, 0.999, 1e-8, 1.0, _fake(5),
                             None) == hmm.HMM_OK
    st = ctypes.c_int32()
    assert lib.hmm_get_device_status(None, None, ctypes.byref(st)) == hmm.HMM_ERR_ARG
    # Baum-Welch M-step: host-side checks only (nothing is launched)
    f = [_fake(i) for i in range(1, 10)]
    assert lib.hmm_mstep(d, None, *f[1:], None) == hmm.HMM_ERR_ARG
    assert lib.hmm_mstep(d, *f[:5], None, *f[6:], None) == hmm.HMM_ERR_ARG
    assert lib.hmm_mstep(hmm.hmm_dims_t(2, 0, 8), *f, None) == hmm.HMM_ERR_ARG
    # the tensor-core forward goes to 512 states, TF32 to 128
    assert _forward(lib, hmm.hmm_dims_t(2, 513, 8), q, precision=hmm.HMM_BF16_MMA) \
        == hmm.HMM_ERR_UNSUPPORTED
    assert _forward(lib, hmm.hmm_dims_t(2, 200, 8), q, precision=hmm.HMM_TF32_MMA) \
        == hmm.HMM_ERR_UNSUPPORTED


def test_tuning_table(lib):
    for op in (hmm.HMM_OP_FORWARD, hmm.HMM_OP_VITERBI, hmm.HMM_OP_FORWARD_BACKWARD,
               hmm.HMM_TUNE_VITERBI_PATHS):
        for n_pad in (4, 8, 16, 32):
            cands = hmm.hmm_tuning_candidates(op, n_pad)
            assert cands and all(32 % g == 0 and n_pad % g == 0 for g in cands)
            assert hmm.hmm_get_tuning(op, n_pad) == cands[0]
    with pytest.raises(hmm.HmmError):
        hmm.hmm_set_tuning(hmm.HMM_OP_FORWARD, 16, 3)
    hmm.hmm_set_tuning(hmm.HMM_OP_FORWARD, 16, 4)
    assert hmm.hmm_get_tuning(hmm.HMM_OP_FORWARD, 16) == 4
    hmm.hmm_set_tuning(hmm.HMM_OP_FORWARD, 16, 0)
    assert hmm.hmm_get_tuning(hmm.HMM_OP_FORWARD, 16) == 2
    assert hmm.hmm_max_states(hmm.HMM_OP_FORWARD) == 64
    assert hmm.hmm_max_states(hmm.HMM_OP_FORWARD_BACKWARD) == 64
    assert hmm.hmm_max_states(hmm.HMM_OP_FORWARD_BACKWARD, hmm.HMM_BF16_MMA) == 512
    assert hmm.hmm_max_states(hmm.HMM_OP_FORWARD, hmm.HMM_BF16_MMA) == 512
    assert hmm.hmm_max_states(hmm.HMM_OP_FORWARD, hmm.HMM_TF32_MMA) == 128
    assert hmm.hmm_max_states(hmm.HMM_OP_VITERBI, hmm.HMM_BF16_MMA) == 0


def test_last_error_is_thread_local(lib):
    import threading
    d = hmm.hmm_dims_t(2, 4, 8)
    _forward(lib, d, _seqs(), pi=None)
    seen = {}

    def other():
        seen["msg"] = hmm.hmm_last_error()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["msg"] == "" and "pi/A/B" in hmm.hmm_last_error()


def test_model_set_argument_errors(lib):
    d = hmm.hmm_dims_t(6, 4, 8)

    def sets(base=_fake(4), span=3, mos=None):
        return hmm.hmm_seqs_t(_fake(1), _fake(2), _fake(3), mos, 4, 10, 40, base, span)

    assert _forward(lib, d, sets(span=0)) == hmm.HMM_ERR_ARG
    assert "model_span" in hmm.hmm_last_error()
    assert _forward(lib, d, sets(span=7)) == hmm.HMM_ERR_ARG
    assert _forward(lib, d, sets(base=_fake(4) + 2)) == hmm.HMM_ERR_ARG
    assert _forward(lib, d, sets(mos=_fake(10))) == hmm.HMM_ERR_ARG
    assert "both" in hmm.hmm_last_error()
    # sets are for recognition: the tensor-core forward and the adjoint refuse them
    wide = hmm.hmm_dims_t(6, 128, 8)
    assert _forward(lib, wide, sets(), precision=hmm.HMM_BF16_MMA) == hmm.HMM_ERR_UNSUPPORTED
    assert lib.hmm_forward_backward(d, _fake(5), _fake(6), _fake(7), ctypes.byref(sets()), None,
                                    hmm.HMM_FP32, _fake(8), _fake(10), _fake(11), _fake(12),
                                    _fake(9), 1 << 30, None) == hmm.HMM_ERR_UNSUPPORTED
    # S == 0 with a valid set returns before any CUDA call
    q0 = sets()
    q0.S = 0
    assert _forward(lib, d, q0) == hmm.HMM_OK


def test_scan_host_checks(lib):
    d = hmm.hmm_dims_t(2, 16, 8)
    q = _seqs(S=4, max_len=10000, total=40000)
    out = ctypes.c_size_t()
    sizes = []
    for chunk in (0, 16, 64, 1024):
        assert lib.hmm_forward_scan_workspace_size(d, ctypes.byref(q), chunk,
                                                   ctypes.byref(out)) == 0
        sizes.append(out.value)
    # smaller chunks need more chunk-product storage (N_pad^2 + N_pad floats each)
    assert sizes[1] > sizes[2] > sizes[3]
    assert sizes[1] >= 2 * (40000 // 16) * (16 * 16 + 16) * 4
    # the op code takes the automatic chunk
    assert lib.hmm_workspace_size(d, ctypes.byref(q), hmm.HMM_OP_FORWARD_SCAN,
                                  ctypes.byref(out)) == 0
    assert out.value == sizes[0]
    assert lib.hmm_max_states(hmm.HMM_OP_FORWARD_SCAN, hmm.HMM_FP32) == 32
    assert lib.hmm_forward_scan_workspace_size(d, ctypes.byref(q), -1,
                                               ctypes.byref(out)) == hmm.HMM_ERR_ARG
    assert lib.hmm_forward_scan_workspace_size(d, ctypes.byref(q), 65537,
                                               ctypes.byref(out)) == hmm.HMM_ERR_ARG
    assert lib.hmm_forward_scan_workspace_size(hmm.hmm_dims_t(2, 33, 8), ctypes.byref(q), 0,
                                               ctypes.byref(out)) == hmm.HMM_ERR_UNSUPPORTED

    def scan(dims, seqs, chunk=0, loglik=_fake(8), ws=_fake(9), ws_bytes=1 << 40):
        return lib.hmm_forward_scan(dims, _fake(5), _fake(6), _fake(7), ctypes.byref(seqs),
                                    chunk, loglik, None, ws, ws_bytes, None)

    assert scan(d, q, chunk=-3) == hmm.HMM_ERR_ARG
    assert scan(d, q, loglik=None) == hmm.HMM_ERR_ARG
    assert scan(hmm.hmm_dims_t(2, 33, 8), q) == hmm.HMM_ERR_UNSUPPORTED
    assert scan(d, q, ws_bytes=1024) == hmm.HMM_ERR_WORKSPACE
    assert "need" in hmm.hmm_last_error()
    assert scan(d, _seqs(S=0)) == hmm.HMM_OK


def test_python_binding_marshals_model_sets_and_scan_sizes(lib):
    """Host side of the binding (CPU tensors stand in for device buffers; no
    kernel is launched): model sets reach the C struct, output widths follow
    the set size, and the scan workspace query goes through the binding."""
    import torch
    S = 6
    seqs = hmm.Sequences(symbols=torch.zeros(60, dtype=torch.int32),
                         offsets=torch.arange(S, dtype=torch.int64) * 10,
                         lengths=torch.full((S,), 10, dtype=torch.int32), max_len=10)
    assert seqs.span is None and seqs.c().model_base is None
    base = torch.tensor([0, 3, 0, 3, 0, 3], dtype=torch.int32)
    sets = seqs.model_sets(base, 3)
    c = sets.c()
    assert c.model_base == base.data_ptr() and c.model_span == 3 and c.model_of_seq is None
    assert sets.span == 3 and sets.all_models().span is None
    dims = hmm.hmm_dims_t(6, 16, 8)
    auto = hmm.hmm_forward_scan_workspace_size(dims, seqs, 0)
    assert auto == hmm.hmm_workspace_size(dims, seqs, hmm.HMM_OP_FORWARD_SCAN)
    assert hmm.hmm_forward_scan_workspace_size(dims, seqs, 1) > auto
    # model sets shrink the chunk-product storage to the set size
    assert hmm.hmm_forward_scan_workspace_size(dims, sets, 1) < \
        hmm.hmm_forward_scan_workspace_size(dims, seqs, 1)
    with pytest.raises(ValueError):  # non-contiguous tensors are refused
        hmm.Sequences(symbols=torch.zeros(60, dtype=torch.int32)[::2], offsets=seqs.offsets,
                      lengths=seqs.lengths, max_len=10).c()


def test_forward_backward_workspace_size_by_precision(lib):
    """The adjoint's workspace at each precision (host only): the TF32 path
    keeps every step's rows (X, Bh, V, G of 128 floats: one block of
    total_obs rows when labelled, K blocks when every sequence is scored
    against every model); other precisions as hmm_workspace_size. Limits: the
    TF32 path takes 64 < N <= 128 and M <= 256; above 128 states the bound on
    M is the cluster forward's emission slice (M <= 173 at 512 padded states;
    the emission counts no longer hold a state-by-symbol table)."""
    f = lib.hmm_forward_backward_workspace_size
    out, ref = ctypes.c_size_t(), ctypes.c_size_t()
    total = 100 * 300
    d = hmm.hmm_dims_t(4, 128, 256)
    lab = _seqs(S=100, max_len=300, total=total, mos=True)
    every = _seqs(S=100, max_len=300, total=total)
    assert f(d, ctypes.byref(lab), hmm.HMM_TF32_MMA, ctypes.byref(out)) == 0
    t_lab = out.value
    assert t_lab >= 4 * total * 128 * 4 and t_lab % 256 == 0
    assert f(d, ctypes.byref(every), hmm.HMM_TF32_MMA, ctypes.byref(out)) == 0
    assert out.value >= 4 * 4 * total * 128 * 4 and out.value > t_lab
    for prec in (hmm.HMM_BF16_MMA, hmm.HMM_AUTO):
        assert f(d, ctypes.byref(lab), prec, ctypes.byref(out)) == 0
        assert lib.hmm_workspace_size(d, ctypes.byref(lab), hmm.HMM_OP_FORWARD_BACKWARD,
                                      ctypes.byref(ref)) == 0
        assert out.value == ref.value
    for dims in (hmm.hmm_dims_t(4, 64, 32), hmm.hmm_dims_t(4, 129, 32),
                 hmm.hmm_dims_t(4, 128, 257)):
        assert f(dims, ctypes.byref(lab), hmm.HMM_TF32_MMA, ctypes.byref(out)) \
            == hmm.HMM_ERR_UNSUPPORTED
    one = _seqs(S=100, max_len=300, total=total)
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(1, 300, 173), ctypes.byref(one),
                                  hmm.HMM_OP_FORWARD_BACKWARD, ctypes.byref(out)) == 0
    assert out.value >= 4 * total * 512 * 4
    assert lib.hmm_workspace_size(hmm.hmm_dims_t(1, 300, 174), ctypes.byref(one),
                                  hmm.HMM_OP_FORWARD_BACKWARD, ctypes.byref(out)) \
        == hmm.HMM_ERR_UNSUPPORTED
