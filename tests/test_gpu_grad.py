"""Gradients on the GPU (through the C ABI) against the CPU oracle: the
adjoint kernel against the Laplace-expansion gradient, the mesh kernels
against the oracle's U(phi) and central finite differences (h = 1e-6), and
the whole phases -> U -> distribution -> KL chain against finite differences
of the oracle's KL."""
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


@pytest.fixture(scope="module")
def ag():
    from paper_2204_00602_gb300 import autograd
    return autograd


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_mesh_forward_matches_oracle(ag):
    for m in (2, 5, 12, 33):
        ph = pin.mesh_phases(3, m * (m - 1), 40 + m)
        U = ag.mesh_unitary(dev(ph), m).cpu().numpy()
        for b in range(3):
            assert np.abs(U[b] - oracle.mesh(ph[b])).max() < 1e-13


def test_mesh_backward_matches_finite_differences(ag):
    m = 6
    ph = pin.mesh_phases(2, m * (m - 1), 50)
    W = pin.random_complex_matrix(m, m, 51)
    U = ag.mesh_unitary(dev(ph), m)
    G = dev(np.stack([W, 2 * W]))
    g = ag.mesh_backward(dev(ph), U, G).cpu().numpy()
    h = 1e-6
    for b, w in ((0, W), (1, 2 * W)):
        L = lambda p: float(np.real(np.sum(np.conj(w) * oracle.mesh(p))))
        for q in range(ph.shape[1]):
            e = np.zeros(ph.shape[1]); e[q] = h
            fd = (L(ph[b] + e) - L(ph[b] - e)) / (2 * h)
            assert abs(g[b, q] - fd) < 1e-8


@pytest.mark.parametrize("m,n", [(4, 1), (5, 3), (6, 4), (8, 6), (9, 8)])
def test_adjoint_matches_laplace_gradient(pcv, m, n):
    U = pin.haar_unitary(m, 60 + n)
    t = pin.single_photon_input(m, n)
    t2 = t.copy()
    if n >= 3:                                  # a bunched input as well
        t2[1] = 0; t2[0] = 2
    for tin in (t, t2):
        outs = pin.random_bunched_outputs(m, n, 12, 70 + n)
        g = pin.random_complex_matrix(1, len(outs), 80 + n)[0]
        want = oracle.grad_U_from_amp_grad(U, tin, outs, g)
        gU = torch.empty(m, m, dtype=torch.complex128, device="cuda")
        pcv.abi.pcv_amplitudes_backward(dev(U), m, tin, dev(outs), len(outs), dev(g), gU,
                                        torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = gU.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


def test_distribution_backward_batched(pcv, ag):
    m, n, B = 6, 3, 2
    Us = np.stack([pin.haar_unitary(m, 90 + b) for b in range(B)])
    t = pin.single_photon_input(m, n)
    occ = oracle.enumerate_outputs(m, n)
    g = pin.random_complex_matrix(B, len(occ), 95)
    gU = ag.distribution_backward(dev(Us), t, dev(g)).cpu().numpy()
    for b in range(B):
        want = oracle.grad_U_from_amp_grad(Us[b], t, occ, g[b])
        assert np.abs(gU[b] - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


def _oracle_kl(phases, m, t, q):
    prob, _ = oracle.distribution(oracle.mesh(phases), t)
    return oracle.kl(q, prob)


@pytest.mark.parametrize("m,n,B", [(6, 3, 3), (12, 6, 2)])
def test_mesh_kl_chain_matches_finite_differences(ag, m, n, B):
    """The differentiable-mesh workload (m=12, n=6 with all 12,376 outputs, a
    Dirichlet(1) target): forward KL against the oracle, gradient against
    central finite differences of the oracle (h = 1e-6)."""
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    q = pin.dirichlet_target(N, 100 + m)
    ph = pin.mesh_phases(B, m * (m - 1), 110 + m)
    phd = dev(ph).requires_grad_(True)
    kl = ag.mesh_kl(phd, m, t, dev(q))
    kl.sum().backward()
    grad = phd.grad.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(7)
    for b in range(B):
        assert abs(kl[b].item() - _oracle_kl(ph[b], m, t, q)) < 1e-10 * max(1, abs(kl[b].item()))
        idx = range(ph.shape[1]) if m <= 6 else rng.choice(ph.shape[1], 24, replace=False)
        for qd in idx:
            e = np.zeros(ph.shape[1]); e[qd] = h
            fd = (_oracle_kl(ph[b] + e, m, t, q) - _oracle_kl(ph[b] - e, m, t, q)) / (2 * h)
            assert abs(grad[b, qd] - fd) <= 1e-6 * max(1.0, abs(fd)), (b, qd, grad[b, qd], fd)


def test_mesh_distribution_gradient_of_a_probability(ag):
    # d p_S / d phi through MeshDistribution (generic dL/dp path)
    m, n = 5, 2
    t = pin.single_photon_input(m, n)
    ph = pin.mesh_phases(1, m * (m - 1), 120)
    phd = dev(ph).requires_grad_(True)
    p = ag.mesh_distribution(phd, m, t)
    w = dev(pin.dirichlet_target(p.shape[1], 121))
    (p[0] * w).sum().backward()
    grad = phd.grad.cpu().numpy()[0]
    wn = w.cpu().numpy()
    L = lambda x: float(np.dot(oracle.distribution(oracle.mesh(x), t)[0], wn))
    h = 1e-6
    for qd in range(ph.shape[1]):
        e = np.zeros(ph.shape[1]); e[qd] = h
        fd = (L(ph[0] + e) - L(ph[0] - e)) / (2 * h)
        assert abs(grad[qd] - fd) < 1e-8


def test_dist_stats(ag):
    p = np.stack([pin.dirichlet_target(1000, 1), pin.dirichlet_target(1000, 2)])
    q = pin.dirichlet_target(1000, 3)
    out = ag.dist_stats(dev(p), dev(q)).cpu().numpy()
    for b in range(2):
        assert abs(out[b, 0] - p[b].sum()) < 1e-14
        assert abs(out[b, 1] - oracle.tvd(p[b], q)) < 1e-14
        assert abs(out[b, 2] - oracle.kl(q, p[b])) < 1e-12
