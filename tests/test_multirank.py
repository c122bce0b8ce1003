"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards into independent products, one per rank (weak scaling, no
collective on the data path); the only collectives are the timing barrier and
the maximum over ranks of the measured time, which the whole-job value uses.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        ms_max = bench.reduce_max(ms, dist, "cpu")
        value = bench.job_gflops(1000, world, 4, ms_max)
        dist.barrier()
        out[rank] = (ms_max, value, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 2.0 * 1000 * 4 / 15e-3 / 1e9)
    assert res[0][2] != res[1][2]                     # independent products per rank


def test_single_process_needs_no_group():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.job_gflops(10, 1, 1, 1.0) == pytest.approx(2e-5)


def _offset_worker(rank, world, port, out):
    from paper_2206_06611_gb300 import brm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nnz = [7, 0, 123456789012][rank]              # int64 counts, one rank empty
        out[rank] = brm.global_row_offset(nnz, None, "cpu")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_shards_find_their_global_offsets(world):
    """Row-sharded products (the static split of Section III-D over GPUs):
    every rank learns where its rows' entries start in the global C, and the
    global nnz, from one all-gather of the ranks' nnz."""
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_offset_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    counts = [7, 0, 123456789012][:world]
    for r in range(world):
        assert res[r] == (sum(counts[:r]), sum(counts))


def _dB_worker(rank, world, port, out):
    import torch
    from paper_2206_06611_gb300 import brm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the library's backward on the rank's rows is replaced by a stand-in
        # (there is no GPU here): its dB partial is rank-specific
        def fake(A, B, C, dC):
            return A.val * 0 + rank, torch.arange(B.nnz, dtype=torch.float64) * (rank + 1)
        brm.brm_spgemm_backward = fake
        rp = torch.tensor([0, 2, 3, 5], dtype=torch.int32)
        A = brm.DeviceCSR(3, 4, rp, torch.zeros(5, dtype=torch.int32), torch.ones(5, dtype=torch.float64))
        B = brm.DeviceCSR(4, 2, torch.tensor([0, 1, 2, 3, 4], dtype=torch.int32),
                          torch.zeros(4, dtype=torch.int32), torch.ones(4, dtype=torch.float64))
        r0, r1 = [(0, 1), (1, 3), (3, 3)][rank] if world == 3 else [(0, 2), (2, 3)][rank]
        dA, dB = brm.spgemm_sharded_backward(A, B, None, None, r0, r1)
        out[rank] = (dA.tolist(), dB.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_shards_sum_their_dB(world):
    """The backward of a row-sharded product: every rank keeps the dA of its
    rows' entries of A and gets the sum of all ranks' dB from one all-reduce."""
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_dB_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    want = [float(k * sum(r + 1 for r in range(world))) for k in range(4)]
    rows = [(0, 1), (1, 3), (3, 3)] if world == 3 else [(0, 2), (2, 3)]
    rp = [0, 2, 3, 5]
    for r in range(world):
        dA, dB = res[r]
        assert dB == want
        assert dA == [float(r)] * (rp[rows[r][1]] - rp[rows[r][0]])
