"""The multi-rank path on CPU: two gloo ranks shard a batch with the
length-balanced partition, each computes its shard's expected counts and
log-likelihoods (with the FP64 oracle standing in for a rank's GPU), and the
count all-reduce reproduces the single-process result; recognition needs no
exchange."""
import os

import numpy as np
import pytest

from paper_1310_3322_gb300 import dist as hdist
from paper_1310_3322_gb300 import synth


def test_partition_covers_every_sequence_once_and_balances():
    w = synth.make_workload("batched", n_seqs=1000)
    for world in (1, 2, 3, 8):
        parts = [hdist.shard_sequences(w.lengths, world, r) for r in range(world)]
        allidx = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allidx, np.arange(w.S))
        loads = [int(w.lengths[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(w.lengths.max())
        # deterministic
        again = [hdist.shard_sequences(w.lengths, world, r) for r in range(world)]
        for a, b in zip(parts, again):
            np.testing.assert_array_equal(a, b)
    with pytest.raises(ValueError):
        hdist.shard_sequences(w.lengths, 2, 2)


def test_subset_packs_sequences():
    w = synth.make_workload("plain", n_seqs=10, lengths=("uniform", 0, 9))
    idx = np.array([7, 2, 5])
    sym, off, ln = hdist.subset(w.symbols, w.offsets, w.lengths, idx)
    for j, s in enumerate(idx):
        np.testing.assert_array_equal(sym[off[j]: off[j] + ln[j]],
                                      w.symbols[w.offsets[s]: w.offsets[s] + w.lengths[s]])


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.make_workload("gradient", n_seqs=64, lengths=("uniform", 5, 60))
    idx = hdist.shard_sequences(w.lengths, world, rank)
    sym, off, ln = hdist.subset(w.symbols, w.offsets, w.lengths, idx)
    P = oracle.params(w.pi, w.A, w.B)
    ll, cpi, cA, cB, _ = oracle.forward_backward(P, sym, off, ln, w.labels[idx])
    rec, am, _ = oracle.forward(P, sym, off, ln)
    t = [torch.from_numpy(x.copy()) for x in (cpi, cA, cB)]
    hdist.allreduce_counts(t)
    # gather recognition results (outputs only, not a data-path exchange)
    full_am = torch.full((w.S,), -9, dtype=torch.int64)
    full_am[torch.from_numpy(idx)] = torch.from_numpy(am.astype(np.int64))
    dist.all_reduce(full_am, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.savez(os.path.join(out_dir, "dist.npz"), cpi=t[0].numpy(), cA=t[1].numpy(),
                 cB=t[2].numpy(), am=full_am.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_process_counts(tmp_path):
    import socket
    import torch.multiprocessing as mp
    import oracle
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = np.load(tmp_path / "dist.npz")
    w = synth.make_workload("gradient", n_seqs=64, lengths=("uniform", 5, 60))
    P = oracle.params(w.pi, w.A, w.B)
    _, cpi, cA, cB, _ = oracle.forward_backward(P, w.symbols, w.offsets, w.lengths, w.labels)
    _, am, _ = oracle.forward(P, w.symbols, w.offsets, w.lengths)
    np.testing.assert_allclose(got["cpi"], cpi, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["cA"], cA, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["cB"], cB, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(got["am"], am)
