"""The tensor-core contraction (sph_mm_bf16: tcgen05, BF16 operands, FP32
accumulation in tensor memory) against a plain PyTorch FP32 product of the
same BF16 values on the CPU.  The sums differ only in FP32 rounding order, so
the bound is relative to the sum of |a_ik b_jk| (a few FP32 ulps of K terms)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1702_07760_gb300 import build as B
    from paper_1702_07760_gb300 import sph
    B.build()
    sph.load()
    torch.cuda.set_device(0)
    return torch, sph


def _run(torch, sph, M, N, K, lda=None, ldb=None, k_split=0, accumulate=False, seed=0):
    g = torch.Generator().manual_seed(seed)
    lda = lda or K
    ldb = ldb or K
    A = (torch.randn(M, lda, generator=g) * 0.5).to(torch.bfloat16)
    B = (torch.randn(N, ldb, generator=g) * 0.5).to(torch.bfloat16)
    ref = A[:, :K].float() @ B[:, :K].float().T
    bound = (A[:, :K].float().abs() @ B[:, :K].float().abs().T) * (K * 2.0 ** -22) + 1e-30
    dA, dB = A.cuda(), B.cuda()
    C0 = torch.randn(M, N, generator=g) if accumulate else torch.zeros(M, N)
    dC = C0.cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    sph.mm_bf16(dA.data_ptr(), lda, dB.data_ptr(), ldb, dC.data_ptr(), N, M, N, K, k_split, accumulate, s,
                err.data_ptr())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = dC.cpu() - (C0 if accumulate else 0)
    return got, ref, bound


@pytest.mark.parametrize("M,N,K", [(300, 128, 128), (128, 256, 256), (77, 16, 16), (1000, 64, 48),
                                   (513, 32, 80), (256, 128, 192)])
def test_gemm_matches_fp32_reference(env, M, N, K):
    torch, sph = env
    got, ref, bound = _run(torch, sph, M, N, K, seed=M + N + K)
    err = (got - ref).abs()
    print(f"\n[gemm {M}x{N}x{K}] max |err| {err.max():.3e}, max err/bound {(err / bound).max():.3f}")
    assert torch.all(err <= bound)


def test_gemm_leading_dimensions_and_split_k(env):
    torch, sph = env
    got, ref, bound = _run(torch, sph, 200, 128, 96, lda=104, ldb=128, seed=3)
    assert torch.all((got - ref).abs() <= bound)
    got, ref, bound = _run(torch, sph, 128, 128, 4096, k_split=512, accumulate=True, seed=4)
    err = (got - ref).abs()
    assert torch.all(err <= 2 * bound + 1e-5), err.max()
