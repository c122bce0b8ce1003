"""Batched products (brm_spgemm_batched, brm_batch_*, brm_autotune).

Every product of a batch must come out exactly as the same product alone:
bit-exact against brm_spgemm_precise and against the oracle's Algorithm 1 in
the same precision.  Prepared batches must recompute C from new values of
the same inputs (directly and through a CUDA graph), and the autotuner must
return options that give the same result.
"""
import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import assert_rows_exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402


def _mix(count, dtype, seed=I.DEFAULT_SEED):
    # the batched workload's recipe at small sizes: n_i log-uniform in
    # [100, 3000], half 3-D Laplacians, half ER with 4..32 per row
    return I.batched_mix(count, seed=seed, nmin=100, nmax=3000, dtype=dtype)


def _check_products(C, off, mats, prec, dtype):
    parts = brm.split(C, off, [M.cols for M in mats])
    for M, Cp in zip(mats, parts):
        assert_rows_exact(Cp, oracle.alg1(M, M, prec=prec))
        Cs = brm.brm_spgemm_precise(brm.to_device(M, dtype=dtype), brm.to_device(M, dtype=dtype))
        assert torch.equal(Cp.rp, Cs.rp) and torch.equal(Cp.col, Cs.col) and torch.equal(Cp.val, Cs.val)


@pytest.mark.parametrize("prec,dtype,comp", [("f64", np.float64, False), ("f32", np.float32, False),
                                             ("f32c", np.float32, True)])
def test_batched_mix_matches_single_products(prec, dtype, comp):
    mats = _mix(24, dtype)
    dev = [brm.to_device(M, dtype=dtype) for M in mats]
    C, off = brm.brm_spgemm_batched(dev, dev, compensated=comp)
    assert off[0] == 0 and off[-1] == sum(M.rows for M in mats) == C.rows
    parts = brm.split(C, off, [M.cols for M in mats])
    for M, Cp in zip(mats, parts):
        assert_rows_exact(Cp, oracle.alg1(M, M, prec=prec))
    if not comp:
        _check_products(C, off, mats, prec, dtype)


def test_batched_all_bins_and_empty_products():
    """Products with rows in every bin (R-MAT has long rows), an empty product
    (no rows) and one whose C is empty, mixed with A != B products."""
    R = I.rmat(12, 16, seed=61)
    E = I.erdos_renyi(700, 9, seed=62)
    Z = I.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    N = I.CSR(6, 5, np.zeros(7, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B5 = I.erdos_renyi(5, 2, seed=63)
    As = [R, Z, E, N]
    Bs = [R, B5, I.erdos_renyi(700, 30, seed=64), B5]
    C, off = brm.brm_spgemm_batched([brm.to_device(M) for M in As], [brm.to_device(M) for M in Bs])
    parts = brm.split(C, off, [M.cols for M in Bs])
    for A, B, Cp in zip(As, Bs, parts):
        assert_rows_exact(Cp, oracle.alg1(A, B))


def test_prepared_batch_reuse_and_graph():
    """New values in the same arrays: numeric() and graph_launch() give the
    product of the new values (structure reuse)."""
    mats = _mix(12, np.float64, seed=65)
    dev = [brm.to_device(M) for M in mats]
    b = brm.Batch(dev, dev)
    b.numeric()
    b.check()
    C, off = b.result()
    _check_products(C, off, mats, "f64", np.float64)
    for round_ in range(2):
        new = []
        for i, (M, D) in enumerate(zip(mats, dev)):
            v = I.rand_sym(70 + round_, i, np.arange(M.nnz))
            D.val.copy_(torch.from_numpy(v))
            new.append(I.CSR(M.rows, M.cols, M.rp, M.col, v))
        if round_ == 0:
            b.numeric()
        else:
            b.graph_launch()
            b.graph_launch()        # a replay gives the same result
        b.check()
        C, off = b.result()
        parts = brm.split(C, off, [M.cols for M in new])
        for M, Cp in zip(new, parts):
            assert_rows_exact(Cp, oracle.alg1(M, M))
    b.close()


def test_autotune_options_give_the_same_result():
    mats = _mix(8, np.float64, seed=66)
    dev = [brm.to_device(M) for M in mats]
    opts, ms = brm.brm_autotune(dev, dev)
    assert ms > 0 and opts["reg_keys"] in (8, 16, 32) and 1 <= opts["reg_warps"] <= 8
    # the thresholds come from the second stage's candidates
    full = 32 * opts["reg_keys"]
    assert opts["reg_max_nprod"] in (full, full // 2, full // 4)
    assert opts["warp_max_nprod"] in (256, 128, 64) and opts["block_max_nprod"] in (4096, 2048, 1024)
    C, off = brm.brm_spgemm_batched(dev, dev, **opts)
    _check_products(C, off, mats, "f64", np.float64)


def test_batched_rejects_mixed_dtypes():
    A = I.erdos_renyi(50, 4, seed=67)
    d64, d32 = brm.to_device(A), brm.to_device(A, dtype=np.float32)
    with pytest.raises(brm.BrmError) as e:
        brm.brm_spgemm_batched([d64, d32], [d64, d32])
    assert e.value.code == -3
