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


def backward(pcv, U, m, tin, outs, g, ws_bytes=None):
    """pcv_amplitudes_backward through the C ABI; dL/dU as numpy."""
    n = int(np.asarray(tin).sum())
    if ws_bytes is None:
        ws_bytes = pcv.abi.pcv_amplitudes_backward_workspace(1, m, n, len(outs))
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device="cuda")
    gU = torch.empty(m, m, dtype=torch.complex128, device="cuda")
    pcv.abi.pcv_amplitudes_backward(dev(U), m, tin, dev(outs), len(outs), dev(g), gU, ws, ws_bytes,
                                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return gU.cpu().numpy()


@pytest.mark.parametrize("m,n", [(4, 1), (5, 3), (6, 4), (8, 6), (9, 8), (12, 10), (14, 12)])
def test_adjoint_matches_laplace_gradient(pcv, m, n):
    """Against the oracle's Laplace expansion (each dPerm/dA[i][j] the permanent
    of a minor, by Ryser), single-photon and bunched inputs, bunched outputs,
    up to n = 12."""
    U = pin.haar_unitary(m, 60 + n)
    t = pin.single_photon_input(m, n)
    t2 = t.copy()
    if n >= 3:                                  # a bunched input as well
        t2[1] = 0; t2[0] = 2
    for tin in (t, t2):
        outs = pin.random_bunched_outputs(m, n, 12 if n <= 10 else 4, 70 + n)
        g = pin.random_complex_matrix(1, len(outs), 80 + n)[0]
        want = oracle.grad_U_from_amp_grad(U, tin, outs, g)
        got = backward(pcv, U, m, tin, outs, g)
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("m,n", [(18, 16), (22, 20)])
def test_adjoint_large_n_split_sign_vectors(pcv, m, n):
    """n = 16 and 20: each output's sign vectors split into parts (several
    warps), summed in part order; against the oracle's Laplace gradient on
    collision-free outputs (tolerance 1e-8, as the forward path's for n > 12)."""
    U = pin.haar_unitary(m, 160 + n)
    t = pin.single_photon_input(m, n)
    outs = pin.random_outputs(m, n, 2, 170 + n)
    g = pin.random_complex_matrix(1, len(outs), 180 + n)[0]
    want = oracle.grad_U_from_amp_grad(U, t, outs, g)
    got = backward(pcv, U, m, t, outs, g)
    assert np.abs(got - want).max() <= 1e-8 * max(1.0, np.abs(want).max())


def test_adjoint_is_deterministic_and_chunks_agree(pcv):
    """The same call twice gives the same bits (fixed summation order, no
    atomics); the smallest workspace (one output per chunk) gives the same
    gradient up to the order in which chunks are added."""
    m, n = 10, 7
    U = pin.haar_unitary(m, 190)
    t = pin.single_photon_input(m, n)
    outs = pin.random_bunched_outputs(m, n, 600, 191)
    g = pin.random_complex_matrix(1, len(outs), 192)[0]
    a = backward(pcv, U, m, t, outs, g)
    b = backward(pcv, U, m, t, outs, g)
    assert np.array_equal(a, b)
    small = pcv.abi.pcv_amplitudes_backward_workspace(1, m, n, 1)
    c = backward(pcv, U, m, t, outs, g, ws_bytes=small)
    assert np.abs(c - a).max() <= 1e-13 * np.abs(a).max()
    with pytest.raises(pcv.PcvError):
        backward(pcv, U, m, t, outs, g, ws_bytes=small - 256)


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
