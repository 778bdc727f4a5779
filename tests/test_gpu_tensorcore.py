"""The tcgen05 tensor-core mainloop (BF16 x BF16 -> FP32 in TMEM) through
its C-ABI test hook, against a plain matmul of the same BF16 values, for
K-major and MN-major operand layouts."""
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def capi():
    from paper_2509_25044_gb300 import build, capi
    build.build()
    capi.load()
    return capi


@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 1), (0, 1), (1, 0)])
@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (256, 32, 192), (128, 64, 128), (384, 48, 64), (128, 128, 256)])
def test_gemm_matches_matmul(capi, a_mn, b_mn, M, N, K):
    g = torch.Generator(device=DEV).manual_seed(M * 7 + N * 3 + K + 11 * a_mn + 5 * b_mn)
    A = torch.randn((M, K), generator=g, device=DEV).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g, device=DEV).to(torch.bfloat16)
    Ain = A.t().contiguous() if a_mn else A.contiguous()
    Bin = B.t().contiguous() if b_mn else B.contiguous()
    C = capi.reg_debug_gemm_bf16(Ain, Bin, M, N, K, a_mn, b_mn)
    torch.cuda.synchronize()
    ref = A.double() @ B.double().t()
    err = (C.double() - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4, err
    assert capi.reg_get_device_error() == 0
