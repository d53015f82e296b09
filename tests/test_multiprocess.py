"""The N > 1 path on CPU (two gloo ranks): the benchmark's barrier and
max-over-ranks timing, the whole-job rate over the slowest rank's time, the
disjoint q shards over the same k states (weak scaling), and the one data
exchange: each rank bins the loss tables of its own q, the bin sums and
counts are combined by an all-reduce, and the rate of the combined table
equals the rate of the union binned on one rank."""
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


def _bins_rank(rank, port, outdir, tables, qmag, edges, w):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from oracle import rate as orate
    from paper_2603_12326_gb300 import shards
    dist.init_process_group("gloo")
    try:
        mine = [i for i in range(len(tables)) if i % 2 == rank]       # rank r holds q number r, r + 2, ...
        L = np.concatenate([tables[i] for i in mine], axis=0)
        q = np.concatenate([qmag[i] for i in mine])
        m, _, c = orate.bin_loss(q, L, edges)
        gm, gc = shards.combine_bins(m, c)
        nz = gc > 0
        centres = 0.5 * (edges[1:] + edges[:-1])
        dR = orate.dR_dw(centres[nz], w, gm[nz], orate.HaloParams()) if rank == 0 else np.zeros(len(w))
        np.savez(os.path.join(outdir, f"b{rank}.npz"), mean=gm, count=gc, dR=dR)
    finally:
        dist.destroy_process_group()


def test_loss_bins_combined_over_two_ranks_equal_one_rank():
    from oracle import rate as orate
    from oracle import rpa
    p = synth.make_small(nq=4, nw=30)
    tables, qmag = [], []
    for iq in range(4):
        o = rpa.solve_q(p, iq)
        tables.append(o["L_lfe"].T)                   # [(G)][w]
        qmag.append(np.linalg.norm(p.qpts[iq][None, :] + p.G_int @ p.cell.recip, axis=1))
    edges = np.linspace(0.0, 2.5, 13)
    m1, centres, c1 = orate.bin_loss(np.concatenate(qmag), np.concatenate(tables, axis=0), edges)
    nz = c1 > 0
    dR1 = orate.dR_dw(centres[nz], p.w, m1[nz], orate.HaloParams())
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_bins_rank, args=(_free_port(), d, tables, qmag, edges, p.w), nprocs=2, join=True,
                           start_method="spawn")
        got = [np.load(os.path.join(d, f"b{r}.npz")) for r in range(2)]
    for g in got:
        assert np.array_equal(g["count"], c1)
        assert np.allclose(g["mean"], m1, rtol=1e-12, atol=1e-14 * np.max(m1))     # summation order only
    assert np.allclose(got[0]["dR"], dR1, rtol=1e-12, atol=0) and np.max(dR1) > 0


def test_shards_are_disjoint_q_sets_over_the_same_k_states():
    a, b = synth.make_mid_shard(0), synth.make_mid_shard(1)
    assert a.qpts.shape == b.qpts.shape == (50, 3)
    assert set(a.q_index.tolist()).isdisjoint(b.q_index.tolist())
    assert not np.allclose(a.qpts, b.qpts)
    assert np.array_equal(a.kpts, b.kpts) and np.array_equal(a.Ek, b.Ek) and np.array_equal(a.G_int, b.G_int)
    assert np.array_equal(a.Zk[:2], b.Zk[:2])
