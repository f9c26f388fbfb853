"""Pins of the partially-distinguishable oracle (oracle/distinguishable.py)
against results fixed independently of it: the indistinguishable distribution
(one class), the permanent of |U|^2 for mutually distinguishable photons, the
Hong-Ou-Mandel values, normalisation, and the visibility of the source model."""
import math

import numpy as np
import pytest

import oracle
import pcv_inputs as pin
from oracle import distinguishable as od

BS = np.array([[1, 1j], [1j, 1]]) / math.sqrt(2)      # Eq. bs at theta = pi/2


def test_one_class_is_the_indistinguishable_distribution():
    m = 5
    U = pin.haar_unitary(m, 5001)
    t = np.array([1, 0, 2, 0, 1], np.uint8)
    p = od.class_distribution(U, [t])
    want, _ = oracle.distribution(U, t)
    assert np.max(np.abs(p - want)) <= 1e-15


def test_empty_classes_are_ignored():
    m = 4
    U = pin.haar_unitary(m, 5002)
    t = np.array([1, 1, 0, 0], np.uint8)
    z = np.zeros(m, np.uint8)
    assert np.max(np.abs(od.class_distribution(U, [z, t, z]) - oracle.distribution(U, t)[0])) <= 1e-15


@pytest.mark.parametrize("t", [[1, 1, 1, 0, 0], [2, 0, 1, 0, 0], [0, 3, 0, 0, 1]])
def test_every_photon_its_own_class_is_the_permanent_of_abs_u_squared(t):
    m = 5
    U = pin.haar_unitary(m, 5003)
    t = np.array(t, np.uint8)
    singles = []
    for c in od.photon_modes(t):
        e = np.zeros(m, np.uint8)
        e[c] = 1
        singles.append(e)
    p = od.class_distribution(U, singles)
    outs = oracle.enumerate_outputs(m, int(t.sum()))
    want = np.array([od.distinguishable_closed_form(U, t, s) for s in outs])
    assert np.max(np.abs(p - want)) <= 1e-14
    assert abs(p.sum() - 1.0) <= 1e-13


def test_hong_ou_mandel():
    a = np.array([1, 0], np.uint8)
    b = np.array([0, 1], np.uint8)
    # outputs of S_{2,2} in canonical order: (2,0), (1,1), (0,2)
    dist = od.class_distribution(BS, [a, b])
    assert np.allclose(dist, [0.25, 0.5, 0.25], atol=1e-15)
    same = od.class_distribution(BS, [a + b])
    assert np.allclose(same, [0.5, 0.0, 0.5], atol=1e-15)


@pytest.mark.parametrize("V", [0.0, 0.3, 0.9, 1.0])
def test_source_visibility(V):
    # coincidence probability (1 - V)/2 for a source of indistinguishability V
    p = od.source_distribution(BS, np.array([1, 1], np.uint8), math.sqrt(V))
    assert abs(p[1] - (1.0 - V) / 2.0) <= 1e-15
    assert abs(p.sum() - 1.0) <= 1e-15


def test_source_limits_and_normalisation():
    m = 5
    U = pin.haar_unitary(m, 5004)
    t = np.array([1, 1, 0, 1, 0], np.uint8)
    outs = oracle.enumerate_outputs(m, 3)
    assert np.max(np.abs(od.source_distribution(U, t, 1.0) - oracle.distribution(U, t)[0])) <= 1e-15
    dist = np.array([od.distinguishable_closed_form(U, t, s) for s in outs])
    assert np.max(np.abs(od.source_distribution(U, t, 0.0) - dist)) <= 1e-14
    mid = od.source_distribution(U, t, 0.7)
    assert abs(mid.sum() - 1.0) <= 1e-14 and np.all(mid >= 0)


def test_mixed_classes_sum_to_one_and_are_symmetric_in_class_order():
    m = 6
    U = pin.haar_unitary(m, 5005)
    c1 = np.array([1, 0, 1, 0, 0, 0], np.uint8)
    c2 = np.array([0, 1, 0, 0, 0, 0], np.uint8)
    c3 = np.array([0, 0, 0, 2, 0, 0], np.uint8)
    p = od.class_distribution(U, [c1, c2, c3])
    q = od.class_distribution(U, [c3, c1, c2])
    assert abs(p.sum() - 1.0) <= 1e-14
    assert np.max(np.abs(p - q)) <= 1e-15


def test_lossy_source_photon_number_is_binomial():
    # the photon number of the kept light is Binomial(n, eta) whatever the
    # interferometer and the distinguishability
    m = 4
    U = pin.haar_unitary(m, 5006)
    t = np.array([1, 1, 1, 0], np.uint8)
    for eta, q in ((0.8, 1.0), (0.5, 0.6), (1.0, 0.3)):
        p = od.lossy_source_distribution(U, t, eta, q)
        off = 0
        for k in range(4):
            N = math.comb(m + k - 1, k)
            want = math.comb(3, k) * eta ** k * (1 - eta) ** (3 - k)
            assert abs(p[off:off + N].sum() - want) <= 1e-14, (eta, q, k)
            off += N
        assert off == p.shape[0]


def test_lossless_source_block_is_the_lossless_mixture():
    m = 4
    U = pin.haar_unitary(m, 5007)
    t = np.array([1, 0, 1, 1], np.uint8)
    p = od.lossy_source_distribution(U, t, 1.0, 0.55)
    N3 = math.comb(m + 2, 3)
    assert np.max(np.abs(p[-N3:] - od.source_distribution(U, t, 0.55))) <= 1e-15
    assert np.all(p[:-N3] == 0)


def test_lossy_hom():
    # two photons, each kept with probability eta, on a 50:50 beam splitter:
    # coincidence eta^2 (1 - V)/2 with V = q^2; one photon left: eta (1 - eta)
    # in total, split evenly between the two modes
    eta, q = 0.7, 0.8
    p = od.lossy_source_distribution(BS, np.array([1, 1], np.uint8), eta, q)
    # blocks: S_{2,0} (1), S_{2,1} (2), S_{2,2} (3)
    assert abs(p[0] - (1 - eta) ** 2) <= 1e-15
    assert np.allclose(p[1:3], [eta * (1 - eta)] * 2, atol=1e-15)
    assert abs(p[4] - eta ** 2 * (1 - q * q) / 2) <= 1e-15
