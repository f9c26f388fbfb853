"""The tcgen05/TMA BF16 GEMM against the CPU reference (oracle/mlp.py), with
the same tolerances as the mma.sync kernel: FP32-accumulated outputs within
K 2^-24 sum|a b| of the FP64 product of the same BF16 inputs, BF16 outputs
within one BF16 rounding."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def S():
    return torch.cuda.current_stream().cuda_stream


def rand(shape, seed):
    return ref.bf16(np.random.default_rng(seed).standard_normal(shape))


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 128, 1024), (300, 200, 96), (7, 33, 64), (16, 1024, 288),
                                   (4096, 1024, 1024), (1024, 288, 4096)])
def test_tc_gemm_modes(M, N, K):
    from paper_2204_00602_gb300 import _abi as abi
    A, B = rand((M, K), 1), rand((N, K), 2)
    bias = np.random.default_rng(3).standard_normal(N).astype(np.float32)
    Ad = torch.from_numpy(A.astype(np.float32)).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B.astype(np.float32)).cuda().to(torch.bfloat16)
    bd = torch.from_numpy(bias).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = ref.gemm(A, B)
    bound = ref.gemm_error_bound(A, B, K)
    out = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    abi.pcv_gemm_bf16_tc(Ad, K, Bd, K, M, N, K, 0, None, out, N, None, 0, None, 0, err, S())
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.all(np.abs(out.cpu().numpy() - C) <= bound)
    pre = torch.empty(M, N, dtype=torch.float32, device="cuda")
    act = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.pcv_gemm_bf16_tc(Ad, K, Bd, K, M, N, K, 1, bd, pre, N, act, N, None, 0, err, S())
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.all(np.abs(pre.cpu().numpy() - (C + bias)) <= bound + 1e-6 * np.abs(bias))
    g = ref.gelu(pre.cpu().numpy().astype(np.float64))
    assert np.all(np.abs(act.float().cpu().numpy() - g) <= 2 ** -8 * np.abs(g) + 1e-6)
    P = np.random.default_rng(4).standard_normal((M, N)).astype(np.float32)
    outb = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.pcv_gemm_bf16_tc(Ad, K, Bd, K, M, N, K, 3, None, None, 0, outb, N, torch.from_numpy(P).cuda(), N, err, S())
    torch.cuda.synchronize()
    want = C * ref.gelu_grad(P.astype(np.float64))
    assert np.all(np.abs(outb.float().cpu().numpy() - want) <=
                  2 ** -8 * np.abs(want) + 2 * bound * np.abs(ref.gelu_grad(P)) + 1e-6)
