"""Row sharding over ranks, run as two gloo processes on the CPU.

Each rank answers its shard_range of a batch with the FP64 oracle (the GPU
path computes the same rows on the box), reduces its whole groups, and the
ranks gather; the assembled rows and groups must equal the oracle run on the
whole batch in one process, exactly (each row's value does not depend on the
other rows), and the ranges must tile the batch with groups kept whole.
"""
import os
import socket

import numpy as np
import pytest

from paper_2609_35619_b300.shard import shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("Q,G,world", [(0, 0, 2), (1, 0, 2), (257, 0, 2), (640, 64, 2), (650, 64, 3),
                                       (1000, 7, 4), (5, 16, 4)])
def test_ranges_tile_the_batch_and_keep_groups(Q, G, world):
    rs = [shard_range(Q, G, r, world) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == Q
    for (a0, b0), (a1, b1) in zip(rs, rs[1:]):
        assert b0 == a1
    Gs = max(G, 1)
    for a, b in rs:
        assert (a % Gs == 0 or a == Q) and (b % Gs == 0 or b == Q)
    groups = [(b - a + Gs - 1) // Gs for a, b in rs]
    assert max(groups) - min(groups) <= 1


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import cs_synth as S
    import oracle
    from paper_2609_35619_b300.shard import gather_rows, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = S.tiny_scene()
    q = S.tiny_queries(q=640)
    G = 64
    a, b = shard_range(q.shape[0], G, rank, world)
    res = oracle.query(sc, q[a:b], 0, 1.0)
    rows = torch.as_tensor(np.stack([res["mean_cost"], res["count_nbr"].astype(np.float64),
                                     res["collide"].astype(np.float64)], 1))
    grp = oracle.group_reduce(res["mean_cost"], res["collide"], G)
    full = gather_rows(rows, q.shape[0], G, world)
    gm = gather_rows(torch.as_tensor(np.stack([grp[0], grp[1].astype(np.float64)], 1)),
                     (q.shape[0] + G - 1) // G, 1, world)
    if rank == 0:
        np.savez(out_path, rows=full.numpy(), groups=gm.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gather_equals_one_process(tmp_path):
    import torch.multiprocessing as mp

    import cs_synth as S
    import oracle
    out = str(tmp_path / "gathered.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    sc = S.tiny_scene()
    q = S.tiny_queries(q=640)
    ref = oracle.query(sc, q, 0, 1.0)
    np.testing.assert_array_equal(got["rows"][:, 0], ref["mean_cost"])
    np.testing.assert_array_equal(got["rows"][:, 1], ref["count_nbr"])
    np.testing.assert_array_equal(got["rows"][:, 2], ref["collide"])
    gm, gc = oracle.group_reduce(ref["mean_cost"], ref["collide"], 64)
    np.testing.assert_array_equal(got["groups"][:, 0], gm)
    np.testing.assert_array_equal(got["groups"][:, 1], gc)
