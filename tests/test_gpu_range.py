"""Splitting one distribution into canonical output ranges (pcv_distribution_range).

A partition of [0, N) into ranges, each computed by its own call as a rank
would, must give back pcv_distribution's arrays exactly (the same arithmetic
per output wherever its tile falls), for the tensor-core products and the
FP64 products (single pass and sign vectors in chunks), with and without
amplitudes, and at the m=20, n=10 workload.  Cuts fall inside the blocks of
outputs that share a low-side multiset, and ranges may be empty or hold one
output.  The whole distribution is itself checked against the oracle here.
"""
import math

import numpy as np
import pytest

import oracle
import pcv_inputs as pin

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


def run_parts(pcv, U, t, cuts, nbytes, want_amp):
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    probs, amps = [], []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        p, a = pcv.distribution_range(U, t, lo, hi, want_amp=want_amp, ws=ws)
        probs.append(p)
        amps.append(a)
    torch.cuda.synchronize()
    return torch.cat(probs), (torch.cat(amps) if want_amp else None)


@pytest.mark.parametrize("path", ["tc", "fp64", "fp64_chunks"])
@pytest.mark.parametrize("want_amp", [True, False])
def test_union_of_ranges_is_the_whole_distribution(pcv, path, want_amp):
    m, n = 12, 6
    abi = pcv.abi
    U = torch.from_numpy(pin.haar_unitary(m, 8201)).cuda()
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    nbytes = {"tc": abi.pcv_distribution_tc_workspace(m, n),
              "fp64": abi.pcv_distribution_batched_workspace(1, m, n),
              "fp64_chunks": abi.pcv_distribution_workspace_min(m, n)}[path]
    if path == "fp64":
        nbytes = min(nbytes, abi.pcv_distribution_tc_workspace(m, n) - 256)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    p_full, a_full = pcv.distribution(U, t, want_amp=want_amp, ws=ws)
    torch.cuda.synchronize()
    p_ref, a_ref = oracle.distribution(U.cpu().numpy(), t)
    assert oracle.tvd(p_full.cpu().numpy(), p_ref) <= 1e-12
    rng = np.random.default_rng(8202)
    for cuts in ([0, N], [0, 1, 2, N // 3, N // 3, N - 1, N],
                 sorted({0, N, *rng.integers(0, N, 5).tolist()}),
                 [pcv.abi.pcv_num_outputs(m, n) * r // 4 for r in range(5)]):
        p, a = run_parts(pcv, U, t, cuts, nbytes, want_amp)
        assert torch.equal(p, p_full), (path, cuts)
        if want_amp:
            assert torch.equal(a, a_full), (path, cuts)


def test_m20_n10_split_in_four(pcv):
    """The bench's workload split into four ranges (as four ranks would run
    it): identical to the whole distribution."""
    m, n = 20, 10
    U = torch.from_numpy(pin.haar_unitary(m, pin.BASE_SEED + 2)).cuda()
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    nbytes = pcv.abi.pcv_distribution_workspace(m, n)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    p_full, a_full = pcv.distribution(U, t, ws=ws)
    torch.cuda.synchronize()
    cuts = [N * r // 4 for r in range(5)]
    p, a = run_parts(pcv, U, t, cuts, nbytes, True)
    assert torch.equal(p, p_full) and torch.equal(a, a_full)
    assert abs(p.sum().item() - 1.0) < 1e-12


def test_range_arguments_are_checked(pcv):
    m, n = 8, 4
    U = torch.from_numpy(pin.haar_unitary(m, 8203)).cuda()
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    fake = 1 << 40                      # never dereferenced: the range is checked first
    for lo, hi in ((-1, 3), (5, 4), (0, N + 1)):
        with pytest.raises(pcv.PcvError) as e:
            pcv.abi.pcv_distribution_range(U, m, t, lo, hi, fake, None, fake, 1 << 40, 0)
        assert e.value.code == pcv.abi.PCV_EINVAL
