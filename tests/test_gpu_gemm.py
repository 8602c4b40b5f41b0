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


@pytest.mark.parametrize("M,N,K,out", [(70001, 300, 136, "f32"), (20000, 2000, 256, "t_f32"),
                                       (65536, 256, 64, "bf16"), (9000, 520, 36, "f32")])
def test_gemm_persistent_many_tiles(gpu, M, N, K, out):
    """Far more tiles than SMs (accumulator and stage rings wrap many times), ragged M/N/K
    (K = 36 leaves part of an 8-column TMA box and a whole box out of range); rows sampled."""
    import paper_2502_08673_b300 as P
    g = torch.Generator().manual_seed(M + N + K)
    A, B = _rand((M, K), g), _rand((N, K), g)
    bias = torch.randn(N, generator=g)
    st = torch.zeros(1, dtype=torch.int32, device=gpu)
    kw = {}
    if out == "f32":
        o = torch.full((M, N), float("nan"), device=gpu)
        kw["out_f32"] = o
    elif out == "bf16":
        o = torch.zeros((M, N), dtype=torch.bfloat16, device=gpu)
        kw["out_bf16"] = o
    else:
        o = torch.full((N, M), float("nan"), device=gpu)
        kw["out_t_f32"] = o
    ld = (K + 7) // 8 * 8  # leading dimensions must be multiples of 8; K itself need not be
    dA = torch.zeros((M, ld), dtype=torch.bfloat16, device=gpu)
    dB = torch.zeros((N, ld), dtype=torch.bfloat16, device=gpu)
    dA[:, :K] = A.to(gpu)
    dB[:, :K] = B.to(gpu)
    if ld > K:  # the padding holds garbage that must not be read
        dA[:, K:] = 1e4
        dB[:, K:] = 1e4
    P.sat_gemm_bf16(dA[:, :K], dB[:, :K], bias=bias.to(gpu), status=st, **kw)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rows = torch.cat([torch.arange(0, 130), torch.randint(0, M, (400,), generator=g), torch.arange(M - 130, M)])
    got = (o.t() if out == "t_f32" else o)[rows.to(gpu)].cpu().double().numpy()
    a = A[rows].double().numpy()
    ref = a @ B.double().numpy().T + bias.double().numpy()[None, :]
    mag = np.abs(a) @ np.abs(B.double().numpy()).T + np.abs(bias.double().numpy())[None, :]
    tol = 1e-5 * mag + 1e-6
    if out == "bf16":
        tol = 2 ** -8 * np.abs(ref) + tol
    d = np.abs(got - ref)
    assert (d <= tol).all(), float(d.max())


def test_gemm_unaligned_outputs(gpu):
    """Outputs whose row stride is not a multiple of 16 bytes take the direct-store path;
    aligned ones in the same call take the staged tensor stores."""
    import paper_2502_08673_b300 as P
    g = torch.Generator().manual_seed(11)
    M, N, K = 301, 99, 64
    A, B = _rand((M, K), g), _rand((N, K), g)
    bias = torch.randn(N, generator=g)
    ref, mag = _ref(A, B)
    ref = ref + bias.double().numpy()[None, :]
    tol = 1e-5 * (mag + np.abs(bias.double().numpy())[None, :]) + 1e-6
    st = torch.zeros(1, dtype=torch.int32, device=gpu)
    out = torch.full((M, N), float("nan"), device=gpu)            # ldo = 99: direct
    out_t = torch.zeros((N, M), dtype=torch.bfloat16, device=gpu)  # ldt = 301: direct
    out_tf = torch.full((N, 304), float("nan"), device=gpu)[:, :M]  # ldt = 304: staged
    P.sat_gemm_bf16(A.to(gpu), B.to(gpu), bias=bias.to(gpu), out_f32=out, out_t_bf16=out_t, status=st)
    P.sat_gemm_bf16(A.to(gpu), B.to(gpu), bias=bias.to(gpu), out_t_f32=out_tf, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert (np.abs(out.cpu().double().numpy() - ref) <= tol).all()
    assert (np.abs(out_tf.cpu().double().numpy().T - ref) <= tol).all()
    assert (np.abs(out_t.cpu().double().numpy().T - ref) <= 2 ** -8 * np.abs(ref) + tol).all()
