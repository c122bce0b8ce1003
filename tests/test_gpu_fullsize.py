"""Parity at the full sizes of the workloads, with the default options (the
launch configuration the benchmark times).

* R-MAT scale 20, C = A*A, FP64 and FP32 with the default options, and FP64
  with every long row in column tiles: nnz(C) is about 9.7e9, beyond 2^32,
  so the int64 output offsets of every numeric kernel are exercised.
  Every row length is compared with the oracle's symbolic pass; the values
  of sampled rows -- the 100 rows with the most products (up to ~9.7 M
  products and ~40 k lists), 400 seeded random rows, and the rows whose slice
  of C holds offset 2^31 - 1, 2^31, 2^32 - 1, 2^32 or 2^33 -- are compared bit
  for bit with the oracle's Algorithm 1 in the same precision (FP64 also
  within 1e-12 of Gustavson's Eq. 2 per row).
* The batched workload: all 512 products of the mix in one batched call,
  FP64 and FP32; for 13 seeded products (the largest among them) every row
  length against the oracle's symbolic pass and 300 sampled rows bit for bit
  against Algorithm 1.
* The differentiable workload (A R-MAT scale 18, B Erdos-Renyi 2^18 with 8
  per row, N(0,1) values): the FP32 forward and hand-written backward through
  torch autograd against the FP64 oracle's gradients over the whole
  matrices; on its 512-row slice in FP64, h = 1 finite differences of the GPU
  forward pass (the loss is linear in every entry, so the difference is the
  gradient up to rounding) and the oracle's gradients.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import RTOL_F64, assert_sample_exact, device_rows, rowwise_rel_err, straddling_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402

THREADS = os.cpu_count() or 1


def _release():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def rmat20():
    A = I.rmat(20, 16)
    return A, oracle.row_nprod(A, A), {}


def _rmat20_rows(A, nprod, rp):
    top = np.argsort(-nprod, kind="stable")[:100]
    rnd = I.rand_below(2020, 1, np.arange(400), A.rows)
    marks = [2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1, 2 ** 32, 2 ** 33]
    return np.unique(np.concatenate([top, rnd, straddling_rows(rp, marks)]))


def _rmat20_check(rmat20, prec, dtype, **opts):
    A, nprod, cache = rmat20
    dA = brm.to_device(A, dtype=dtype)
    C = brm.brm_spgemm_precise(dA, dA, **opts)
    torch.cuda.synchronize()
    rp = C.rp.cpu().numpy()
    assert rp[-1] > 2 ** 32, "the workload no longer exercises 64-bit output offsets"
    if prec == "f64":
        if "nnz" not in cache:
            cache["nnz"] = oracle.symbolic_parallel(A, A, threads=THREADS)
        assert np.array_equal(np.diff(rp), cache["nnz"])
    rows = _rmat20_rows(A, nprod, rp)
    crp, col, val = device_rows(C, rows)
    del C, dA
    _release()
    key = (prec, rows.tobytes())
    if key not in cache:
        cache[key] = oracle.alg1_parallel(A, A, rows, prec, THREADS)
    assert_sample_exact(crp, col, val, cache[key])
    return rows, crp, val


@pytest.mark.parametrize("prec,dtype", [("f64", np.float64), ("f32", np.float32)])
def test_rmat_scale20_full_size(rmat20, prec, dtype):
    A = rmat20[0]
    rows, crp, val = _rmat20_check(rmat20, prec, dtype)
    if prec == "f64":
        g = oracle.gustavson_parallel(A, A, THREADS, rows, with_abs=True)
        assert rowwise_rel_err(crp, val, g.val, g.abs).max(initial=0.0) <= RTOL_F64


def test_rmat_scale20_every_long_row_tiled(rmat20):
    """The same checks with every long row of at most 65535 lists in column
    tiles (long_window 2): the hub rows, up to ~40k lists, search their lists
    block by block with their cursors in device memory."""
    _rmat20_check(rmat20, "f64", np.float64, long_window=2)


@pytest.fixture(scope="module")
def mix512():
    return I.batched_mix(512)


@pytest.mark.parametrize("prec,dtype", [("f64", np.float64), ("f32", np.float32)])
def test_batched_512_full_size(mix512, prec, dtype):
    mats = [M.astype(dtype) for M in mix512]
    dev = [brm.to_device(M) for M in mats]
    C, off = brm.brm_spgemm_batched(dev, dev)
    torch.cuda.synchronize()
    assert off[-1] == C.rows == sum(M.rows for M in mats)
    rp = C.rp.cpu().numpy()
    sizes = np.array([int(oracle.row_nprod(M, M).sum()) for M in mats])
    pick = np.unique(np.concatenate([[int(np.argmax(sizes))], I.rand_below(512, 3, np.arange(12), 512)]))
    samples = []
    for p in pick:
        M, r0 = mats[int(p)], int(off[int(p)])
        assert np.array_equal(np.diff(rp[r0:r0 + M.rows + 1]), oracle.symbolic_parallel(M, M, threads=THREADS))
        npr = oracle.row_nprod(M, M)
        rows = np.unique(np.concatenate([np.argsort(-npr, kind="stable")[:50],
                                         I.rand_below(513, int(p), np.arange(250), M.rows)]))
        samples.append((M, rows, device_rows(C, rows + r0)))
    del C, dev
    _release()
    for M, rows, (crp, col, val) in samples:
        assert_sample_exact(crp, col, val, oracle.alg1_parallel(M, M, rows, prec, THREADS))


def _rel(x, ref):
    x = np.asarray(x, dtype=np.float64)
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


def test_differentiable_full_size():
    A = I.normal_values(I.rmat(18, 16), 101)
    B = I.normal_values(I.erdos_renyi(1 << 18, 8), 102)
    dA, dB = brm.to_device(A), brm.to_device(B)
    a_val = dA.val.clone().requires_grad_(True)
    b_val = dB.val.clone().requires_grad_(True)
    C = brm.spgemm(brm.DeviceCSR(A.rows, A.cols, dA.rp, dA.col, a_val),
                   brm.DeviceCSR(B.rows, B.cols, dB.rp, dB.col, b_val))
    G = torch.from_numpy(I.rand_normal(103, I.S_GRAD, np.arange(C.nnz)).astype(np.float32)).cuda()
    (C.val * G).sum().backward()
    crp, ccol, g64 = C.rp.cpu().numpy(), C.col.cpu().numpy(), G.cpu().numpy().astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ra, rb = oracle.backward(A64, B64, crp, ccol, g64)
    # FP32 sums of <= ~130 (dA) and a few hundred (dB) terms of N(0,1) size
    assert _rel(a_val.grad.cpu().numpy(), ra) < 1e-5
    assert _rel(b_val.grad.cpu().numpy(), rb) < 1e-5

    # the 512-row slice in FP64: rows 0 .. 511 of A (R-MAT's densest rows)
    ns = 512
    e = int(A.rp[ns])
    S = I.CSR(ns, A.cols, A.rp[:ns + 1].copy(), A.col[:e].copy(), A64.val[:e].copy())
    dS, dB64 = brm.to_device(S), brm.to_device(B64)
    CS = brm.brm_spgemm_precise(dS, dB64)
    assert np.array_equal(CS.rp.cpu().numpy(), crp[:ns + 1]) and np.array_equal(CS.col.cpu().numpy(),
                                                                                 ccol[:crp[ns]])
    GS = torch.from_numpy(g64[:crp[ns]]).cuda()
    ga, gb = brm.brm_spgemm_backward(dS, dB64, CS, GS)
    sa, sb = oracle.backward(S, B64, crp[:ns + 1], ccol[:crp[ns]], g64[:crp[ns]])
    assert np.array_equal(ga.cpu().numpy(), sa)
    assert np.array_equal(gb.cpu().numpy(), sb)

    def fd(Sm, Bm):
        # loss(perturbed) - loss(S, B), summed over the entries of C that moved
        Cm = brm.brm_spgemm_precise(brm.to_device(Sm), brm.to_device(Bm))
        assert torch.equal(Cm.col, CS.col)
        return float(((Cm.val - CS.val) * GS).sum().item())

    pick_a = I.rand_below(104, 1, np.arange(16), e)
    touched = np.unique(S.col)
    brows = touched[I.rand_below(105, 1, np.arange(16), len(touched))]
    blen = np.diff(B.rp.astype(np.int64))
    brows = brows[blen[brows] > 0]
    pick_b = B.rp[brows].astype(np.int64) + I.rand_below(106, 1, np.arange(len(brows)), 1 << 30) % blen[brows]
    for q in pick_a:
        v = S.val.copy()
        v[q] += 1.0
        d = fd(I.CSR(S.rows, S.cols, S.rp, S.col, v), B64)
        assert abs(d - float(ga[q])) <= 1e-9 * (1.0 + abs(d))
    for q in pick_b:
        v = B64.val.copy()
        v[q] += 1.0
        d = fd(S, I.CSR(B64.rows, B64.cols, B64.rp, B64.col, v))
        assert abs(d - float(gb[q])) <= 1e-9 * (1.0 + abs(d))
