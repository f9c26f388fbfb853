"""Partially distinguishable photons on the GPU (pcv_distribution_classes,
pcv_distribution_source) against the CPU oracle of oracle/distinguishable.py
and against closed forms.  Distributions must agree within TVD 1e-12 and
elementwise within 1e-12 absolute."""
import math

import numpy as np
import pytest

import oracle
import pcv_inputs as pin
from oracle import distinguishable as od

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BS = np.array([[1, 1j], [1j, 1]]) / math.sqrt(2)


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check(got, want):
    got = got.cpu().numpy() if hasattr(got, "cpu") else got
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= 1e-12
    assert 0.5 * np.abs(got - want).sum() <= 1e-12


def occ(m, modes):
    t = np.zeros(m, np.uint8)
    for c in modes:
        t[c] += 1
    return t


@pytest.mark.parametrize("split", [[[0, 1, 2]], [[0, 1], [2]], [[0], [1], [2]], [[0, 0], [1, 3]],
                                   [[0, 2], [1, 3], [4]], [[1], [0, 2, 3, 4]]])
def test_classes_match_oracle(pcv, split):
    m = 6
    U = pin.haar_unitary(m, 6001 + len(split))
    classes = [occ(m, s) for s in split]
    torch.cuda.synchronize()
    check(pcv.distribution_classes(dev(U), classes), od.class_distribution(U, classes))


def test_all_distinguishable_is_the_permanent_of_abs_u_squared(pcv):
    m, n = 7, 4
    U = pin.haar_unitary(m, 6010)
    t = pin.single_photon_input(m, n)
    classes = [occ(m, [c]) for c in range(n)]
    p = pcv.distribution_classes(dev(U), classes).cpu().numpy()
    want = np.array([od.distinguishable_closed_form(U, t, s) for s in oracle.enumerate_outputs(m, n)])
    check(p, want)


def test_classes_hom_and_empty(pcv):
    p = pcv.distribution_classes(dev(BS), [occ(2, [0]), occ(2, [1])]).cpu().numpy()
    assert np.allclose(p, [0.25, 0.5, 0.25], atol=1e-15)
    p = pcv.distribution_classes(dev(BS), [occ(2, [0, 1])]).cpu().numpy()
    assert np.allclose(p, [0.5, 0.0, 0.5], atol=1e-15)
    p = pcv.distribution_classes(dev(BS), [occ(2, []), occ(2, [])]).cpu().numpy()
    assert p.tolist() == [1.0]


def test_classes_m12_n6_mixed_sizes(pcv):
    m = 12
    U = pin.haar_unitary(m, 6020)
    classes = [occ(m, [0, 1, 2]), occ(m, [3, 4]), occ(m, [5])]
    p = pcv.distribution_classes(dev(U), classes).cpu().numpy()
    check(p, od.class_distribution(U, classes))
    assert abs(p.sum() - 1.0) <= 1e-12


@pytest.mark.parametrize("V", [0.0, 0.5, 0.9, 1.0])
def test_source_hom_visibility(pcv, V):
    p, off = pcv.source_distribution(dev(BS), [1, 1], 1.0, V)
    p = p.cpu().numpy()
    assert abs(p[off[2] + 1] - (1 - V) / 2) <= 1e-15
    assert abs(p.sum() - 1.0) <= 1e-15


@pytest.mark.parametrize("eta,V", [(1.0, 0.8), (0.7, 1.0), (0.6, 0.5), (0.0, 0.3), (1.0, 0.0)])
def test_source_matches_oracle(pcv, eta, V):
    m = 5
    U = pin.haar_unitary(m, 6030)
    t = np.array([1, 1, 0, 1, 1], np.uint8)
    p, off = pcv.source_distribution(dev(U), t, eta, V)
    check(p, od.lossy_source_distribution(U, t, eta, math.sqrt(V)))
    assert off[-1] == p.shape[0]


def test_source_bunched_input_matches_oracle(pcv):
    m = 4
    U = pin.haar_unitary(m, 6040)
    t = np.array([2, 0, 1, 0], np.uint8)
    p, _ = pcv.source_distribution(dev(U), t, 0.85, 0.6)
    check(p, od.lossy_source_distribution(U, t, 0.85, math.sqrt(0.6)))


def test_source_m8_n5(pcv):
    m, n = 8, 5
    U = pin.haar_unitary(m, 6050)
    t = pin.single_photon_input(m, n)
    p, off = pcv.source_distribution(dev(U), t, 0.9, 0.92)
    p = p.cpu().numpy()
    check(p, od.lossy_source_distribution(U, t, 0.9, math.sqrt(0.92)))
    for k in range(n + 1):   # photon number Binomial(n, eta)
        assert abs(p[off[k]:off[k + 1]].sum() - math.comb(n, k) * 0.9 ** k * 0.1 ** (n - k)) <= 1e-13


def test_source_argument_errors(pcv):
    U = dev(pin.haar_unitary(4, 6060))
    with pytest.raises(pcv.PcvError):
        pcv.source_distribution(U, [1, 1, 0, 0], 1.5, 1.0)
    with pytest.raises(pcv.PcvError):
        pcv.source_distribution(U, [1, 1, 0, 0], 1.0, -0.1)
    with pytest.raises(pcv.PcvError):
        pcv.source_distribution(dev(pin.haar_unitary(20, 6061)), [1] * 17 + [0] * 3, 1.0, 1.0)
