"""pcv_distribution_static, the entry point for callers that cannot allocate
device memory (an application that owns all device memory through its own
pool, or a service that allows no allocation after start-up).  It takes no
workspace and uses a fixed array inside the library instead.

Checked through the C ABI against pcv_distribution (the entry point with a
caller-provided workspace), within the tolerance of the other parity tests,
on two calls in a row: the shared array keeps the previous call's contents,
which must not leak into the next result.  This file sorts last so that a
run stopping at the first failure has already run every other test.
"""
import math

import numpy as np
import pytest

import pcv_inputs as pin

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def amp_err(got, want, m, n):
    floor = 1.0 / math.sqrt(math.comb(m + n - 1, n))
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


@pytest.mark.parametrize("m,n,seed", [(12, 6, 11), (20, 10, 12)])
def test_static_scratch_matches_workspace_entry_point(pcv, m, n, seed):
    abi = pcv.abi
    stream = torch.cuda.current_stream().cuda_stream
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    for call in range(2):                       # two calls in a row, different unitaries
        U = torch.from_numpy(pin.haar_unitary(m, seed + 100 * call)).cuda()
        p_ref = torch.empty(N, dtype=torch.float64, device="cuda")
        a_ref = torch.empty(N, dtype=torch.complex128, device="cuda")
        ws_bytes = abi.pcv_distribution_workspace(m, n)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        abi.pcv_distribution(U, m, t, p_ref, a_ref, ws, ws_bytes, stream)

        prob = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
        amp = torch.full((N,), -1.0, dtype=torch.complex128, device="cuda")
        abi.pcv_distribution_static(U, m, t, prob, amp, stream)
        torch.cuda.synchronize()
        assert amp_err(amp.cpu().numpy(), a_ref.cpu().numpy(), m, n) <= 1e-10
        assert 0.5 * (prob - p_ref).abs().sum().item() <= 1e-12
        assert abs(prob.sum().item() - 1.0) < 1e-12


@pytest.mark.parametrize("m,n,seed", [(12, 6, 21), (14, 8, 22)])
def test_static_scratch_probabilities_only(pcv, m, n, seed):
    """Probabilities only: the running amplitude sums then live inside the
    shared array too.  m=12, n=6 takes one pass over the sign vectors; at
    m=14, n=8 the tables of all 128 sign vectors exceed the array, so the
    sign vectors run in two passes that add into those sums.  Two calls in a
    row with different unitaries: nothing of the first may leak into the
    second."""
    abi = pcv.abi
    stream = torch.cuda.current_stream().cuda_stream
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    for call in range(2):
        U = torch.from_numpy(pin.haar_unitary(m, seed + 100 * call)).cuda()
        p_ref = torch.empty(N, dtype=torch.float64, device="cuda")
        ws_bytes = abi.pcv_distribution_workspace(m, n)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        abi.pcv_distribution(U, m, t, p_ref, None, ws, ws_bytes, stream)
        prob = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
        abi.pcv_distribution_static(U, m, t, prob, None, stream)
        torch.cuda.synchronize()
        assert 0.5 * (prob - p_ref).abs().sum().item() <= 1e-12
        assert (prob - p_ref).abs().max().item() <= 1e-12
        assert abs(prob.sum().item() - 1.0) < 1e-12


def test_static_scratch_rejects_problems_that_do_not_fit(pcv):
    abi = pcv.abi
    m, n = 20, 10
    U = torch.from_numpy(pin.haar_unitary(m, 3)).cuda()
    prob = torch.empty(math.comb(m + n - 1, n), dtype=torch.float64, device="cuda")
    # probabilities only: the running amplitude sums alone (320 MB) exceed the array
    with pytest.raises(abi.PcvError) as e:
        abi.pcv_distribution_static(U, m, pin.single_photon_input(m, n), prob, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.code == abi.PCV_ENOMEM
    assert "PCV_STATIC_SCRATCH_BYTES" in str(e.value)
    assert abi.pcv_distribution_static_max_bytes() == 32 << 20
