"""The surrogate's tcgen05 GEMM (TMA + tensor memory) against float64 on the same BF16
inputs.  FP32 accumulation of K products: each element is within K * 2^-23 of the sum of
|a_k b_k| (a loose bound on the accumulation error); the BF16 epilogue adds half a BF16
ulp (2^-8 relative)."""
import numpy as np
import pytest

from paper_1903_10741_gb300 import ffs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(M, N, K, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    A = (torch.randn(M, K, generator=g) * scale).to(torch.bfloat16)
    B = (torch.randn(N, K, generator=g) * scale).to(torch.bfloat16)
    bias = torch.randn(N, generator=g).float()
    a, b = A.double().numpy(), B.double().numpy()
    return A.cuda(), B.cuda(), bias.cuda(), a @ b.T, np.abs(a) @ np.abs(b).T, bias.double().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 256, 64), (256, 256, 128), (384, 1664, 256),
                                   (4096, 256, 1664), (256, 1664, 4096)])
def test_gemm_f32_matches_float64(M, N, K):
    A, B, _, ref, mag, _ = _case(M, N, K, seed=M + N + K)
    C = ffs.tensor_gemm(A, B).cpu().double().numpy()
    tol = K * 2.0 ** -23 * mag + 1e-30
    bad = np.abs(C - ref) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], C[bad][:5], ref[bad][:5])


@pytest.mark.parametrize("M,N,K", [(128, 256, 192), (512, 128, 256), (1024, 256, 1664)])
def test_gemm_bias_relu_bf16(M, N, K):
    A, B, bias, ref, mag, b = _case(M, N, K, seed=7 * M + K)
    C = ffs.tensor_gemm(A, B, bias=bias, relu_bf16=True).float().cpu().double().numpy()
    want = np.maximum(ref + b[None, :], 0.0)
    tol = K * 2.0 ** -23 * mag + 2.0 ** -8 * np.abs(want) + 1e-30
    bad = np.abs(C - want) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], C[bad][:5], want[bad][:5])


def test_gemm_structured_operands_exact():
    """Small integers are exact in BF16 and their products sum exactly in FP32: the result
    must equal the integer matrix product, which catches any misplaced row, column or K
    slice (a swizzle or descriptor error)."""
    M, N, K = 256, 256, 320
    rng = np.random.default_rng(5)
    a = rng.integers(-4, 5, size=(M, K)).astype(np.float32)
    b = rng.integers(-4, 5, size=(N, K)).astype(np.float32)
    A = torch.from_numpy(a).to(torch.bfloat16).cuda()
    B = torch.from_numpy(b).to(torch.bfloat16).cuda()
    C = ffs.tensor_gemm(A, B).cpu().numpy()
    assert np.array_equal(C, a.astype(np.int64) @ b.astype(np.int64).T)


def test_gemm_rejects_bad_shapes():
    A = torch.zeros((100, 64), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ffs.FFSError):
        ffs.tensor_gemm(A, B)
    A = torch.zeros((128, 48), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((128, 48), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ffs.FFSError):
        ffs.tensor_gemm(A, B)
