"""The headline workload certified against the CPU oracle over every output.

m = 20 modes, n = 10 photons in modes 0..9, the Haar unitary of seed
2204006022 (the one the throughput benchmark times): all 20,030,010 outputs
of S_{20,10}.  The oracle evaluates Eq. eqperm for each output with Ryser's
formula on the host cores (about 40 s on 16 cores); each GPU path is then
compared with it element by element:
  * relative amplitude error |a_gpu - a_ref| / max(|a_ref|, 1/sqrt(N)) <= 1e-10
    (the floor is the RMS amplitude of a unitary, sum_S |a(S)|^2 = 1);
  * total variation distance (Eq. bosonsampling) <= 1e-12;
  * p = |a|^2 and sum p = 1.
"""
import math

import numpy as np
import pytest

import oracle
import pcv_inputs as pin

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

M, N = 20, 10


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


@pytest.fixture(scope="module")
def problem():
    U = pin.haar_unitary(M, pin.BASE_SEED + 2)
    t = pin.single_photon_input(M, N)
    p_ref, a_ref = oracle.distribution(U, t)
    assert len(p_ref) == math.comb(M + N - 1, N) == 20_030_010
    return U, t, p_ref, a_ref


def check(prob, amp, p_ref, a_ref):
    floor = 1.0 / math.sqrt(len(a_ref))
    rel = np.abs(amp - a_ref) / np.maximum(np.abs(a_ref), floor)
    assert rel.max() <= 1e-10, f"max relative amplitude error {rel.max():.3e} at {int(rel.argmax())}"
    assert oracle.tvd(prob, p_ref) <= 1e-12
    assert abs(prob.sum() - 1.0) <= 1e-12
    assert np.allclose(prob, np.abs(amp) ** 2, rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("algo", ["auto", "factor_tc", "factor"])
def test_m20_n10_every_output_against_oracle(pcv, problem, algo):
    U, t, p_ref, a_ref = problem
    code = {"auto": pcv.PCV_ALGO_AUTO, "factor_tc": pcv.PCV_ALGO_FACTOR_TC, "factor": pcv.PCV_ALGO_FACTOR}[algo]
    prob, amp = pcv.distribution(torch.from_numpy(U).cuda(), t, algo=code)
    torch.cuda.synchronize()
    check(prob.cpu().numpy(), amp.cpu().numpy(), p_ref, a_ref)
