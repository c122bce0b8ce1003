"""The differentiable form: brm_spgemm_backward and the autograd binding.

For loss = sum(C * G) with G on C's pattern,
  dA = (G B^T) on A's pattern, dB = (A^T G) on B's pattern.
Checks:
* dA and dB bit-exact against the oracle's backward in FP64 (both sum dA_ik
  sequentially over B_k* in column order and dB_kj over the rows i in
  increasing order, products rounded, no fused multiply-add), and the same
  bits from call to call;
* FP32 against the FP64 oracle within a stated relative tolerance;
* finite differences of the GPU forward pass (the loss is linear in each
  operand, so L(A + h E_ik) - L(A) = h dA_ik up to rounding for any h);
* torch autograd through brm.spgemm gives the same gradients.
"""
import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402


def _grad_pattern(C, seed, dtype):
    return torch.from_numpy(I.rand_normal(seed, I.S_GRAD, np.arange(C.nnz)).astype(dtype)).cuda()


def _rel(x, ref):
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


@pytest.mark.parametrize("case", ["int", "er", "rmat"])
def test_backward_f64_against_oracle(case):
    if case == "int":
        A, B = I.random_int(60, 80, 0.2, 41, 0), I.random_int(80, 70, 0.15, 41, 1)
    elif case == "er":
        A, B = I.erdos_renyi(3000, 12, seed=42), I.erdos_renyi(3000, 9, seed=43)
    else:
        A, B = I.rmat(11, 8, seed=44), I.erdos_renyi(2048, 8, seed=45)
    dA, dB = brm.to_device(A), brm.to_device(B)
    C = brm.brm_spgemm_precise(dA, dB)
    G = _grad_pattern(C, 46, np.float64)
    if case == "int":
        G = torch.round(G * 3)
    ga, gb = brm.brm_spgemm_backward(dA, dB, C, G)
    ra, rb = oracle.backward(A, B, C.rp.cpu().numpy(), C.col.cpu().numpy(), G.cpu().numpy())
    assert np.array_equal(ga.cpu().numpy(), ra)
    assert np.array_equal(gb.cpu().numpy(), rb)


def test_backward_f32_against_f64_oracle():
    """FP32 values (N(0,1), the differentiable workload's distribution): error
    against the FP64 oracle below 1e-5 normwise (a few FP32 roundings per
    entry over sums of <= ~100 terms)."""
    A = I.normal_values(I.rmat(11, 16, seed=47), 48)
    B = I.normal_values(I.erdos_renyi(2048, 8, seed=49), 50)
    dA, dB = brm.to_device(A), brm.to_device(B)
    C = brm.brm_spgemm_precise(dA, dB)
    G = _grad_pattern(C, 51, np.float32)
    ga, gb = brm.brm_spgemm_backward(dA, dB, C, G)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ra, rb = oracle.backward(A64, B64, C.rp.cpu().numpy(), C.col.cpu().numpy(), G.cpu().numpy().astype(np.float64))
    assert _rel(ga.cpu().numpy().astype(np.float64), ra) < 1e-5
    assert _rel(gb.cpu().numpy().astype(np.float64), rb) < 1e-5


def test_finite_differences_and_autograd():
    """512-row slice: h = 1 steps on sampled entries of A and B through the
    GPU forward pass, and the same gradients from torch autograd."""
    A = I.rmat(10, 8, seed=52)
    A = I.CSR(A.rows, A.cols, A.rp, A.col, A.val)
    B = I.erdos_renyi(1024, 8, seed=53)
    dA, dB = brm.to_device(A), brm.to_device(B)
    C = brm.brm_spgemm_precise(dA, dB)
    G = _grad_pattern(C, 54, np.float64)
    ga, gb = brm.brm_spgemm_backward(dA, dB, C, G)

    def loss(Am, Bm):
        Cm = brm.brm_spgemm_precise(brm.to_device(Am), brm.to_device(Bm))
        assert torch.equal(Cm.col, C.col)
        return float((Cm.val * G).sum().item())

    L0 = loss(A, B)
    rows512 = np.arange(min(512, A.rows))
    ents_a = np.arange(A.rp[rows512[0]], A.rp[rows512[-1] + 1])
    pick_a = ents_a[I.rand_below(55, 1, np.arange(12), len(ents_a))]
    pick_b = I.rand_below(56, 1, np.arange(12), B.nnz)
    for e in pick_a:
        v = A.val.copy()
        v[e] += 1.0
        fd = loss(I.CSR(A.rows, A.cols, A.rp, A.col, v), B) - L0
        assert abs(fd - float(ga[e])) <= 1e-9 * (1 + abs(fd))
    for e in pick_b:
        v = B.val.copy()
        v[e] += 1.0
        fd = loss(A, I.CSR(B.rows, B.cols, B.rp, B.col, v)) - L0
        assert abs(fd - float(gb[e])) <= 1e-9 * (1 + abs(fd))

    a_val = dA.val.clone().requires_grad_(True)
    b_val = dB.val.clone().requires_grad_(True)
    Ct = brm.spgemm(brm.DeviceCSR(A.rows, A.cols, dA.rp, dA.col, a_val),
                    brm.DeviceCSR(B.rows, B.cols, dB.rp, dB.col, b_val))
    (Ct.val * G).sum().backward()
    assert torch.equal(a_val.grad, ga)
    assert torch.equal(b_val.grad, gb)


def test_backward_rejects_wrong_pattern():
    A, B = I.erdos_renyi(200, 5, seed=57), I.erdos_renyi(200, 5, seed=58)
    dA, dB = brm.to_device(A), brm.to_device(B)
    C = brm.brm_spgemm_precise(dA, dB)
    col = C.col.clone()
    col[3] = (int(col[3]) + 1) % B.cols
    bad = brm.DeviceCSR(C.rows, C.cols, C.rp, col, C.val)
    with pytest.raises(brm.BrmError):
        brm.brm_spgemm_backward(dA, dB, bad, C.val.clone())


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_backward_deterministic_and_crowded_columns(dtype):
    """Columns of A held by thousands of rows (their buckets are sorted by a
    thread block in device memory, the rest by one warp): dB bit-exact against
    the oracle in FP64, and identical bits over repeated calls in both
    precisions."""
    k, n, m = 600, 900, 5000
    B = I.erdos_renyi(k, 7, seed=60, ncols=n)
    hot = np.array([3, 17, 400])
    rows = []
    for i in range(m):
        u = I.rand_u64(61, i, np.arange(12)) % np.uint64(k)
        c = np.unique(u.astype(np.int64))[:6]
        take = hot[I.rand_unit(62, i, np.arange(3)) < np.array([0.9, 0.5, 0.25])]
        rows.append(np.unique(np.concatenate([c, take])))
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    A = I.CSR(m, k, rp.astype(np.int32), col, I.rand_sym(63, 1, np.arange(len(col))))
    A, B = A.astype(dtype), B.astype(dtype)
    dA, dB = brm.to_device(A), brm.to_device(B)
    C = brm.brm_spgemm_precise(dA, dB)
    G = _grad_pattern(C, 64, dtype)
    ga, gb = brm.brm_spgemm_backward(dA, dB, C, G)
    for _ in range(3):
        ga2, gb2 = brm.brm_spgemm_backward(dA, dB, C, G)
        assert torch.equal(ga, ga2) and torch.equal(gb, gb2)
    _, gb_only = brm.brm_spgemm_backward(dA, dB, C, G, want_da=False)
    assert torch.equal(gb, gb_only)
    if dtype == np.float64:
        ra, rb = oracle.backward(A, B, C.rp.cpu().numpy(), C.col.cpu().numpy(), G.cpu().numpy())
        assert np.array_equal(ga.cpu().numpy(), ra)
        assert np.array_equal(gb.cpu().numpy(), rb)
