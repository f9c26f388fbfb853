"""The factorised full distribution with its products on the tensor cores
(PCV_ALGO_FACTOR_TC: exact digit splitting, BF16 MMA, FP32 accumulation that
never rounds) against the CPU oracle and against the FP64 factorised path.
Tolerances are the FP64 path's: relative amplitude error 1e-10 (n <= 12),
TVD <= 1e-12."""
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


def amp_err(got, want, m, n):
    floor = 1.0 / math.sqrt(math.comb(m + n - 1, n))
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def tc_dist(pcv, U, t, want_amp=True):
    prob, amp = pcv.distribution(dev(U), t, algo=pcv.PCV_ALGO_FACTOR_TC, want_amp=want_amp)
    torch.cuda.synchronize()
    return prob.cpu().numpy(), (amp.cpu().numpy() if amp is not None else None)


@pytest.mark.parametrize("m,n,t", [(2, 1, None), (3, 2, None), (6, 3, None), (7, 4, [2, 0, 1, 0, 1, 0, 0]),
                                   (9, 5, None), (12, 6, None), (11, 7, [1, 1, 2, 0, 1, 0, 1, 0, 0, 0, 1])])
def test_tc_distribution_matches_oracle(pcv, m, n, t):
    U = pin.haar_unitary(m, 7000 + 13 * m + n)
    t = pin.single_photon_input(m, n) if t is None else np.array(t, np.uint8)
    p_ref, a_ref = oracle.distribution(U, t)
    prob, amp = tc_dist(pcv, U, t)
    assert amp_err(amp, a_ref, m, n) <= 1e-10
    assert 0.5 * np.abs(prob - p_ref).sum() <= 1e-12
    assert np.allclose(prob, np.abs(amp) ** 2, rtol=1e-14, atol=0)


@pytest.mark.parametrize("m,n,t", [
    (40, 3, None),          # single-entry columns merged into the k = 1 and k = n-1 tiles (32 + 32 wide)
    (70, 2, None),          # 35 + 35 columns do not fit one tile: separate single-entry blocks
    (5, 4, [0, 4, 0, 0, 0]),    # all photons in one input mode (a repeated column)
    (2, 3, [2, 1]),          # one mode per side
    (1, 3, [3]),             # m = 1: no high side, the single-entry blocks in FP64
    (30, 4, "modes 0 2 6 29"),   # photons spread over both sides, K = 8
    (10, 8, None),           # K = 128: one warp per table entry
    (10, 9, None),           # K = 256: two warps per table entry
])
def test_tc_block_shapes_match_oracle(pcv, m, n, t):
    """Shapes that exercise how the blocks are formed: merged and separate
    single-entry columns, tile widths 16..64, one side with a single mode,
    and the FP64 fallback."""
    U = pin.haar_unitary(m, 7400 + 17 * m + n)
    if t is None:
        t = pin.single_photon_input(m, n)
    elif isinstance(t, str):
        t = pin.single_photon_input(m, n, modes=[int(v) for v in t.split()[1:]])
    else:
        t = np.array(t, np.uint8)
    p_ref, a_ref = oracle.distribution(U, t)
    prob, amp = tc_dist(pcv, U, t)
    assert amp_err(amp, a_ref, m, n) <= 1e-10
    assert 0.5 * np.abs(prob - p_ref).sum() <= 1e-12
    assert abs(prob.sum() - 1.0) <= 1e-12


def test_tc_probabilities_only(pcv):
    m, n = 10, 5
    U = pin.haar_unitary(m, 7101)
    t = pin.single_photon_input(m, n)
    p_ref, _ = oracle.distribution(U, t)
    prob, amp = tc_dist(pcv, U, t, want_amp=False)
    assert amp is None
    assert 0.5 * np.abs(prob - p_ref).sum() <= 1e-12


def test_tc_not_unitary_and_wide_range(pcv):
    # a non-unitary U whose rows differ in scale by 1e6: the per-row exponents
    # keep the relative accuracy of every output
    m, n = 8, 4
    g = np.random.default_rng(7201)
    U = (g.normal(size=(m, m)) + 1j * g.normal(size=(m, m))) * np.logspace(-3, 3, m)[:, None]
    t = pin.single_photon_input(m, n)
    _, a_ref = oracle.distribution(U, t)
    _, amp = tc_dist(pcv, U, t)
    assert np.max(np.abs(amp - a_ref) / np.maximum(np.abs(a_ref), 1e-300)) <= 1e-10


def test_tc_m20_n10_against_fp64_path_and_oracle(pcv):
    """The 20,030,010-output workload: every output against the FP64
    factorised path, sampled outputs against the oracle, and the sum rule."""
    m, n = 20, 10
    U = pin.haar_unitary(m, pin.BASE_SEED + 2)
    t = pin.single_photon_input(m, n)
    p64, a64 = pcv.distribution(dev(U), t, algo=pcv.PCV_ALGO_FACTOR)
    ptc, atc = pcv.distribution(dev(U), t, algo=pcv.PCV_ALGO_FACTOR_TC)
    torch.cuda.synchronize()
    assert abs(ptc.sum().item() - 1.0) < 1e-12
    assert 0.5 * (ptc - p64).abs().sum().item() <= 1e-12
    floor = 1.0 / math.sqrt(math.comb(m + n - 1, n))
    rel = ((atc - a64).abs() / torch.clamp(a64.abs(), min=floor)).max().item()
    assert rel <= 1e-11
    rng = np.random.default_rng(6)
    idx = np.unique(np.concatenate([[0, 1, ptc.numel() - 1], rng.integers(0, ptc.numel(), 800)]))
    occ = np.stack([pcv.unrank(m, n, int(i)) for i in idx])
    a_ref = oracle.amplitudes(U, t, occ)
    assert amp_err(atc[torch.from_numpy(idx).cuda()].cpu().numpy(), a_ref, m, n) <= 1e-10


def test_tc_workspace_and_limits(pcv):
    assert pcv.abi.pcv_distribution_tc_workspace(20, 10) > 0
    with pytest.raises(pcv.PcvError):
        pcv.abi.pcv_distribution_tc_workspace(20, 11)
    U = dev(pin.haar_unitary(12, 7301))
    with pytest.raises(pcv.PcvError):
        pcv.distribution(U, pin.single_photon_input(12, 11), algo=pcv.PCV_ALGO_FACTOR_TC)


@pytest.mark.parametrize("branch", ["tc", "fp64", "fp64_min"])
def test_auto_takes_both_branches(pcv, branch):
    """pcv_distribution (PCV_ALGO_AUTO): the tensor-core products with the
    full workspace, the FP64 products with a smaller one (single pass, and the
    minimum workspace, which runs the sign vectors in chunks); all three
    against the oracle."""
    m, n = 12, 6
    U = pin.haar_unitary(m, 7501)
    t = pin.single_photon_input(m, n)
    tc = pcv.abi.pcv_distribution_tc_workspace(m, n)
    nbytes = {"tc": tc, "fp64": min(tc - 256, pcv.abi.pcv_distribution_batched_workspace(1, m, n)),
              "fp64_min": pcv.abi.pcv_distribution_workspace_min(m, n)}[branch]
    want = pcv.PCV_ALGO_FACTOR_TC if branch == "tc" else pcv.PCV_ALGO_FACTOR
    assert pcv.abi.pcv_distribution_auto_algo(m, n, nbytes) == want
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    prob, amp = pcv.distribution(dev(U), t, ws=ws)
    torch.cuda.synchronize()
    p_ref, a_ref = oracle.distribution(U, t)
    assert amp_err(amp.cpu().numpy(), a_ref, m, n) <= 1e-10
    assert 0.5 * np.abs(prob.cpu().numpy() - p_ref).sum() <= 1e-12
