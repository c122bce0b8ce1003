"""One product over several GPUs by the static row split (Section III-D):
brm_row_split against the oracle's nprod-balanced groups, and the shards --
computed one after another on one GPU, each a BRMerge-Precise call on its
slice of A's rows with B whole -- put together into exactly the C of a
single call and of the oracle, and their backward (dA per shard, dB summed
over the shards).  (The all-gather of the shards' nnz and the all-reduce of
their dB are covered by gloo ranks in test_multirank.py.)"""
import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import assert_rows_exact, bins_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402


@pytest.mark.parametrize("case", ["rmat", "bins"])
@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_row_shards_rebuild_the_product(case, parts):
    A, B = (I.rmat(13, 16, seed=90),) * 2 if case == "rmat" else bins_matrix(seed=14)
    dA, dB = brm.to_device(A), brm.to_device(B)
    bounds = brm.brm_row_split(dA, dB, parts)
    want = oracle.balanced_row_groups(oracle.row_nprod(A, B), parts)
    assert bounds == [int(x) for x in want]
    full = brm.brm_spgemm_precise(dA, dB)
    rps, cols, vals, off = [np.zeros(1, np.int64)], [], [], 0
    for p in range(parts):
        r0, r1 = bounds[p], bounds[p + 1]
        C = brm.brm_spgemm_precise(brm.row_slice(dA, r0, r1), dB)
        torch.cuda.synchronize()
        assert C.rows == r1 - r0
        rps.append(C.rp.cpu().numpy()[1:] + off)
        cols.append(C.col.cpu().numpy())
        vals.append(C.val.cpu().numpy())
        off += C.nnz
    rp = np.concatenate(rps)
    joined = brm.DeviceCSR(A.rows, B.cols, torch.from_numpy(rp), torch.from_numpy(np.concatenate(cols)),
                           torch.from_numpy(np.concatenate(vals)))
    assert np.array_equal(rp, full.rp.cpu().numpy())
    assert np.array_equal(joined.col.numpy(), full.col.cpu().numpy())
    assert np.array_equal(joined.val.numpy(), full.val.cpu().numpy())
    assert_rows_exact(joined, oracle.alg1(A, B))


def test_row_split_edge_cases():
    A = I.erdos_renyi(10, 3, seed=91)
    dA = brm.to_device(A)
    # more parts than rows: some parts are empty, the bounds stay ordered
    b = brm.brm_row_split(dA, dA, 16)
    assert b[0] == 0 and b[-1] == 10 and all(x <= y for x, y in zip(b, b[1:]))
    with pytest.raises(brm.BrmError):
        brm.brm_row_split(dA, dA, 0)


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("parts", [2, 3])
def test_row_shards_backward(parts):
    """The backward of a row-sharded product: every shard's dA (its rows'
    entries of A) is the single call's dA bit for bit, and the shards' dB
    added up is the single call's dB up to the order of the sum (FP64 sums
    of ~1e2 terms of unit size: 1e-12 relative); through
    spgemm_sharded_backward on a one-rank group as well."""
    import os
    import torch.distributed as dist
    A = I.normal_values(I.rmat(12, 16, seed=92), 93, dtype=np.float64)
    B = I.normal_values(I.erdos_renyi(A.cols, 6, seed=94), 95, dtype=np.float64)
    dA, dB = brm.to_device(A), brm.to_device(B)
    full = brm.brm_spgemm_precise(dA, dB)
    G = torch.from_numpy(I.rand_normal(96, I.S_GRAD, np.arange(full.nnz))).cuda()
    ga, gb = brm.brm_spgemm_backward(dA, dB, full, G)
    bounds = brm.brm_row_split(dA, dB, parts)
    rp = full.rp.cpu().numpy()
    ga_parts, gb_sum = [], torch.zeros_like(gb)
    for p in range(parts):
        r0, r1 = bounds[p], bounds[p + 1]
        Cp = brm.brm_spgemm_precise(brm.row_slice(dA, r0, r1), dB)
        Gp = G[int(rp[r0]):int(rp[r1])].contiguous()
        a, b = brm.brm_spgemm_backward(brm.row_slice(dA, r0, r1), dB, Cp, Gp)
        ga_parts.append(a)
        gb_sum += b
    assert torch.equal(torch.cat(ga_parts), ga)
    scale = torch.linalg.vector_norm(gb).item()
    assert torch.linalg.vector_norm(gb_sum - gb).item() <= 1e-12 * scale
    ra, rb = oracle.backward(A, B, rp, full.col.cpu().numpy(), G.cpu().numpy())
    assert np.array_equal(ga.cpu().numpy(), ra)
    assert np.abs(gb_sum.cpu().numpy() - rb).max() <= 1e-12 * max(np.abs(rb).max(), 1.0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        C1, r0, r1, off, total = brm.spgemm_sharded(dA, dB)
        assert (r0, r1, off, total) == (0, A.rows, 0, full.nnz)
        a1, b1 = brm.spgemm_sharded_backward(dA, dB, C1, G, r0, r1)
        assert torch.equal(a1, ga) and torch.equal(b1, gb)
    finally:
        dist.destroy_process_group()
