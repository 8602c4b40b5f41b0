"""Tensor-core BF16 GEMM (tcgen05) of the proposal network against its definition.

D[m][n] = sum_k A[m][k] B[n][k] in exact arithmetic on the bf16 inputs; the
kernel accumulates in FP32, so the bound is 1e-5 * sum_k |A[m][k] B[n][k]|
(summation error of K FP32 additions, with margin).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rand(shape, gen, scale=1.0):
    return (torch.randn(shape, generator=gen) * scale).to(torch.bfloat16)


def _ref(A, B):
    a = A.double().numpy()
    b = B.double().numpy()
    return a @ b.T, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 64), (200, 256, 256), (2000, 512, 256),
                                   (300, 100, 80), (64, 256, 2000), (1000, 64, 128)])
def test_gemm_matches_definition(gpu, M, N, K):
    import paper_2502_08673_b300 as P
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A, B = _rand((M, K), g), _rand((N, K), g)
    ref, mag = _ref(A, B)
    out = torch.full((M, N), float("nan"), device=gpu)
    st = torch.zeros(1, dtype=torch.int32, device=gpu)
    P.sat_gemm_bf16(A.to(gpu), B.to(gpu), out_f32=out, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    d = np.abs(out.cpu().double().numpy() - ref)
    assert (d <= 1e-5 * mag + 1e-6).all(), float(d.max())


def test_gemm_epilogues(gpu):
    """bias + GELU with the pre-activation stored, transposed bf16 store, GELU' product."""
    import paper_2502_08673_b300 as P
    g = torch.Generator().manual_seed(5)
    M, N, K = 384, 192, 128
    A, B = _rand((M, K), g, 0.3), _rand((N, K), g, 0.3)
    bias = torch.randn(N, generator=g)
    ref, mag = _ref(A, B)
    z = ref + bias.double().numpy()[None, :]
    erf = np.vectorize(math.erf)
    gelu = 0.5 * z * (1 + erf(z / math.sqrt(2)))
    dA = A.to(gpu)
    pre = torch.zeros(M, N, device=gpu)
    out = torch.zeros(M, N, device=gpu)
    out_t = torch.zeros(N, M, dtype=torch.bfloat16, device=gpu)
    st = torch.zeros(1, dtype=torch.int32, device=gpu)
    P.sat_gemm_bf16(dA, B.to(gpu), bias=bias.to(gpu), epilogue=1, pre=pre, alpha=2.0, out_f32=out, out_t_bf16=out_t,
                    status=st)
    torch.cuda.synchronize()
    tol = 1e-5 * mag + 1e-6
    assert (np.abs(pre.cpu().double().numpy() - z) <= tol).all()
    assert (np.abs(out.cpu().double().numpy() - 2 * gelu) <= 2.5 * tol + 1e-6).all()
    assert (np.abs(out_t.cpu().double().numpy().T - 2 * gelu) <= 2 ** -7 * np.abs(2 * gelu) + 1e-5).all()
    # GELU'(pre) * (A B^T)
    out2 = torch.zeros(M, N, device=gpu)
    P.sat_gemm_bf16(dA, B.to(gpu), epilogue=2, pre=pre, out_f32=out2, status=st)
    torch.cuda.synchronize()
    p = pre.cpu().double().numpy()
    gp = 0.5 * (1 + erf(p / math.sqrt(2))) + p * np.exp(-0.5 * p * p) / math.sqrt(2 * math.pi)
    assert (np.abs(out2.cpu().double().numpy() - ref * gp) <= 1.5 * tol + 1e-6).all()
    assert int(st.item()) == 0
