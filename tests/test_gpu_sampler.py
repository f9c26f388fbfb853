"""Exact boson sampling on the GPU against the CPU oracle's distribution:
impossible outputs never drawn, deterministic cases exact, empirical
frequencies consistent with P(S) (chi-square, seeded, significance 1e-6) and
the partial certificate P(K) (Eq. eqpk) within five standard errors."""
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


def draw(pcv, U, t, count, seed):
    n = int(np.asarray(t).sum())
    perm, uni = pin.sampler_randomness(count, n, seed)
    out = pcv.sample(torch.from_numpy(np.ascontiguousarray(U)).cuda(), t, torch.from_numpy(perm).cuda(),
                     torch.from_numpy(uni).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_hong_ou_mandel_never_gives_one_one(pcv):
    s = draw(pcv, oracle.BS_RX_HALF, np.array([1, 1], np.uint8), 20000, 1)
    assert not np.any((s[:, 0] == 1) & (s[:, 1] == 1))
    frac = np.mean(s[:, 0] == 2)
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / 20000)


def test_permutation_matrix_is_deterministic(pcv):
    m = 7
    P = np.eye(m)[[3, 0, 6, 1, 2, 5, 4]].astype(complex)
    t = pin.single_photon_input(m, 4)
    s = draw(pcv, P, t, 1000, 2)
    want = np.abs(P @ t.astype(float)).astype(np.uint8)
    assert np.all(s == want[None, :])


def _chi2_check(pcv, U, t, count, seed):
    from scipy.stats import chi2
    m = U.shape[0]
    n = int(t.sum())
    prob, _ = oracle.distribution(U, t)
    occ = oracle.enumerate_outputs(m, n)
    index = {o.tobytes(): i for i, o in enumerate(occ)}
    s = draw(pcv, U, t, count, seed)
    assert np.all(s.sum(1) == n)
    counts = np.zeros(len(occ))
    for row in s:
        counts[index[row.tobytes()]] += 1
    assert np.all(counts[prob < 1e-15] == 0)
    keep = prob * count >= 5
    exp = prob[keep] * count
    stat = np.sum((counts[keep] - exp) ** 2 / exp)
    df = int(keep.sum()) - 1
    assert stat < chi2.ppf(1 - 1e-6, df), (stat, df)


def test_frequencies_match_oracle_distribution(pcv):
    m, n = 6, 3
    _chi2_check(pcv, pin.haar_unitary(m, pin.BASE_SEED + 1), pin.single_photon_input(m, n), 200_000, 3)


def test_bunched_input(pcv):
    _chi2_check(pcv, pin.haar_unitary(4, 21), np.array([2, 0, 1, 0], np.uint8), 100_000, 4)


def test_partial_certificate_n10_m20(pcv):
    m, n = 20, 10
    U = pin.haar_unitary(m, 22)
    t = pin.single_photon_input(m, n)
    N = 60_000
    s = draw(pcv, U, t, N, 5)
    for K in (12, 15, 18):
        V = U[:K][:, :n]
        exact = oracle.perm_ryser(V.conj().T @ V).real          # P(K): all photons in the first K modes
        est = np.mean(s[:, K:].sum(1) == 0)
        assert abs(est - exact) < 5 * math.sqrt(exact * (1 - exact) / N) + 1e-4, (K, est, exact)
