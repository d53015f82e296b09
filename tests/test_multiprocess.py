"""The N > 1 benchmark path on CPU: two gloo ranks run the benchmark's barrier
and max-over-ranks timing, and the whole-job rate counts every rank's blocks
over the slowest rank's time; the shards are disjoint q sets over the same k
states (weak scaling, no data-path collective)."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo")
    try:
        ws, r, _ = bench._dist()
        assert (ws, r) == (2, rank)
        bench._barrier(ws)
        ms = 100.0 + 50.0 * rank                    # rank 1 is the slower one
        mx = bench._barrier_max(ws, ms)
        value = bench._weak_value(50, 200, 3, ws, mx)
        with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
            f.write(f"{mx} {value}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_max_time():
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(_free_port(), d), nprocs=2, join=True, start_method="spawn")
        res = [tuple(map(float, open(os.path.join(d, f"r{r}.txt")).read().split())) for r in range(2)]
    for mx, value in res:
        assert mx == 150.0
        assert value == pytest.approx(2 * 50 * 200 * 3 / 0.150)


def test_shards_are_disjoint_q_sets_over_the_same_k_states():
    a, b = synth.make_mid_shard(0), synth.make_mid_shard(1)
    assert a.qpts.shape == b.qpts.shape == (50, 3)
    assert set(a.q_index.tolist()).isdisjoint(b.q_index.tolist())
    assert not np.allclose(a.qpts, b.qpts)
    assert np.array_equal(a.kpts, b.kpts) and np.array_equal(a.Ek, b.Ek) and np.array_equal(a.G_int, b.G_int)
    assert np.array_equal(a.Zk[:2], b.Zk[:2])
