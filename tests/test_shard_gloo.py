"""Member sharding over processes (CPU, gloo, world size 2): the gathered
statistics and their mixture are bit-identical to a single-process run."""
import os
import socket

import numpy as np
import pytest

import ens_inputs as I
from paper_2506_23712_gb300.shard import gather_stats, partition_members

NQ, NT = 8, 16


def member_stats(i, lam):
    counts = I.synthetic_member_counts([lam], NQ, NT, 50000, seed=1000 + i)[0]
    rng = np.random.Generator(np.random.Philox(key=2000 + i))
    return counts, rng.standard_normal(48)


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, lams, Ns, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = partition_members(Ns, world)
    mine = parts[rank]
    c = np.array([member_stats(i, lams[i])[0] for i in mine]).reshape(len(mine), -1)
    m = np.array([member_stats(i, lams[i])[1] for i in mine]).reshape(len(mine), 48)
    all_c, all_m = gather_stats(mine, c, m, len(lams))
    if rank == 0:
        np.savez(out_path, counts=all_c, moments=all_m)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_balances_work():
    Ns = [128] * 24 + [256] * 12 + [384] * 4
    parts = partition_members(Ns, 4)
    assert sorted(sum(parts, [])) == list(range(len(Ns)))
    loads = [sum(Ns[i] ** 3 for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.2
    assert partition_members(Ns, 4) == parts          # deterministic
    # equal members: round-robin, 8 per rank
    assert partition_members([256] * 64, 8) == [list(range(r, 64, 8)) for r in range(8)]


def test_gather_and_mix_match_single_process(tmp_path):
    import torch.multiprocessing as mp
    import oracle as O
    import oracle.mixture as OM
    lams = list(np.linspace(-2.5, 2.5, 7))
    Ns = [32, 64, 32, 16, 64, 32, 16]
    out = str(tmp_path / "gathered.npz")
    mp.start_processes(_worker, args=(2, free_port(), lams, Ns, out), nprocs=2, start_method="spawn")
    got = np.load(out)
    ref_c = np.array([member_stats(i, l)[0] for i, l in enumerate(lams)])
    ref_m = np.array([member_stats(i, l)[1] for i, l in enumerate(lams)])
    assert np.array_equal(got["counts"], ref_c) and np.array_equal(got["moments"], ref_m)
    h = O.HistSpec(qr_bins=NQ, tail_bins=NT)
    w, _ = OM.member_weights(lams, "gauss_paper", c=0.023, Z=1.5)
    a = OM.mix_counts(got["counts"], w, h)
    b = OM.mix_counts(ref_c, w, h)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
