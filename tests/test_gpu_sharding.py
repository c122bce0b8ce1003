"""One product over several GPUs by the static row split (Section III-D):
brm_row_split against the oracle's nprod-balanced groups, and the shards --
computed one after another on one GPU, each a BRMerge-Precise call on its
slice of A's rows with B whole -- put together into exactly the C of a
single call and of the oracle.  (The all-gather of the shards' nnz is covered
by two gloo ranks in test_multirank.py.)"""
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
