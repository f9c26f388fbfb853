"""The time-out path of the tensor-core kernels, exercised without a fault.

Every mbarrier wait of the distribution's product kernel and of the BF16
GEMM gives up after a bounded number of polls.  pcv_set_wait_limit(1) makes
those waits run out almost at once (a load or an MMA takes far longer than
one poll), so the kernels take their failure path: record the role that gave
up, wait (with a separate bound) for their own loads and MMAs in flight,
release tensor memory and return.  The tests check that the status comes back
as PCV_ETIMEOUT (the error flag for the GEMM), and that the next call with the
default bound, on the same workspace, is correct again: the context is intact.
"""
import math

import numpy as np
import pytest

import oracle
import pcv_inputs as pin
from oracle import mlp as ref

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


def stream():
    return torch.cuda.current_stream().cuda_stream


def test_distribution_timeout_is_reported_and_the_next_call_is_correct(pcv):
    abi = pcv.abi
    m, n = 12, 6
    U = torch.from_numpy(pin.haar_unitary(m, 8101)).cuda()
    t = pin.single_photon_input(m, n)
    ws = pcv.workspace(abi.pcv_distribution_tc_workspace(m, n), U.device)
    abi.pcv_set_wait_limit(1)
    try:
        pcv.distribution(U, t, algo=pcv.PCV_ALGO_FACTOR_TC, ws=ws)
        with pytest.raises(abi.PcvError) as e:
            abi.pcv_distribution_status(ws, stream())
        assert e.value.code == abi.PCV_ETIMEOUT
    finally:
        abi.pcv_set_wait_limit(0)
    prob, amp = pcv.distribution(U, t, algo=pcv.PCV_ALGO_FACTOR_TC, ws=ws)
    assert abi.pcv_distribution_status(ws, stream()) == abi.PCV_OK
    p_ref, a_ref = oracle.distribution(U.cpu().numpy(), t)
    floor = 1.0 / math.sqrt(len(p_ref))
    assert np.max(np.abs(amp.cpu().numpy() - a_ref) / np.maximum(np.abs(a_ref), floor)) <= 1e-10
    assert oracle.tvd(prob.cpu().numpy(), p_ref) <= 1e-12


def test_gemm_timeout_sets_the_error_flag_and_the_next_call_is_correct():
    from paper_2204_00602_gb300 import _abi as abi
    M, N, K = 512, 256, 1024
    A = ref.bf16(np.random.default_rng(1).standard_normal((M, K)))
    B = ref.bf16(np.random.default_rng(2).standard_normal((N, K)))
    Ad = torch.from_numpy(A.astype(np.float32)).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B.astype(np.float32)).cuda().to(torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    abi.pcv_set_wait_limit(1)
    try:
        abi.pcv_gemm_bf16_tc(Ad, K, Bd, K, M, N, K, 0, None, out, N, None, 0, None, 0, err, stream())
        torch.cuda.synchronize()
    finally:
        abi.pcv_set_wait_limit(0)
    assert err.item() != 0
    err.zero_()
    abi.pcv_gemm_bf16_tc(Ad, K, Bd, K, M, N, K, 0, None, out, N, None, 0, None, 0, err, stream())
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.all(np.abs(out.cpu().numpy() - ref.gemm(A, B)) <= ref.gemm_error_bound(A, B, K))
