"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerance (Eq. eqperm amplitudes, complex FP64): the relative amplitude error
|a_gpu - a_ref| / max(|a_ref|, 1/sqrt(C(m+n-1,n))) must stay <= 1e-10 for
n <= 12 and <= 1e-8 for n <= 30; the floor is the RMS amplitude of a unitary
U (sum_S |a(S)|^2 = 1), so near-zero amplitudes (HOM-type zeros) are judged
on an absolute scale.  Full distributions: TVD (Eq. bosonsampling) <= 1e-12.
"""
import math

import numpy as np
import pytest

import golden_io
import oracle
import pcv_inputs as pin

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


def tol(n):
    return 1e-10 if n <= 12 else 1e-8


def amp_err(got, want, m, n):
    floor = 1.0 / math.sqrt(math.comb(m + n - 1, n))
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_amps(pcv, U, t, outs, **kw):
    amp, prob = pcv.amplitudes(dev(U), t, dev(outs), **kw)
    torch.cuda.synchronize()
    return amp.cpu().numpy(), prob.cpu().numpy()


# ------------------------------------------------------------ workload 1


def test_m6_n3_full_distribution_all_algorithms(pcv):
    m, n = 6, 3
    U = pin.haar_unitary(m, pin.BASE_SEED + 1)
    t = pin.single_photon_input(m, n)
    p_ref, a_ref = oracle.distribution(U, t)
    assert len(p_ref) == 56
    variants = [dict(algo=pcv.PCV_ALGO_FACTOR)] + [dict(algo=pcv.PCV_ALGO_GROUP, param=g) for g in (1, 2, 4)]
    for kw in variants:
        prob, amp = pcv.distribution(dev(U), t, **kw)
        torch.cuda.synchronize()
        prob, amp = prob.cpu().numpy(), amp.cpu().numpy()
        assert amp_err(amp, a_ref, m, n) <= tol(n), kw
        assert oracle.tvd(prob, p_ref) <= 1e-12, kw
        assert abs(prob.sum() - 1) < 1e-13


# -------------------------------------------------- explicit outputs


@pytest.mark.parametrize("n", list(range(1, 13)))
def test_group_kernel_every_threads_per_permanent(pcv, n):
    m = max(n + 2, 8)
    U = pin.haar_unitary(m, 300 + n)
    t = pin.single_photon_input(m, n)
    outs = np.concatenate([pin.random_outputs(m, n, 40, 400 + n), pin.random_bunched_outputs(m, n, 40, 500 + n)])
    a_ref = oracle.amplitudes(U, t, outs)
    for G in (1, 2, 4, 8, 16, 32):
        if G > 2 ** (n - 1):
            continue
        amp, prob = run_amps(pcv, U, t, outs, algo=pcv.PCV_ALGO_GROUP, param=G)
        assert amp_err(amp, a_ref, m, n) <= tol(n), G
        assert np.allclose(prob, np.abs(a_ref) ** 2, rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("n,splits", [(9, 1), (10, 2), (12, 1), (13, 4), (14, 2), (16, 8)])
def test_block_kernel_with_splits(pcv, n, splits):
    m = 2 * n
    U = pin.haar_unitary(m, 600 + n)
    t = pin.single_photon_input(m, n)
    outs = np.concatenate([pin.random_outputs(m, n, 6, 700 + n), pin.random_bunched_outputs(m, n, 6, 800 + n)])
    a_ref = oracle.amplitudes(U, t, outs)
    amp, _ = run_amps(pcv, U, t, outs, algo=pcv.PCV_ALGO_BLOCK, param=splits)
    assert amp_err(amp, a_ref, m, n) <= tol(n)


def test_auto_choice_and_ragged_counts(pcv):
    for m, n, cnt in [(9, 4, 1), (9, 4, 33), (16, 7, 257), (24, 12, 3), (30, 14, 5)]:
        U = pin.haar_unitary(m, 900 + cnt)
        t = pin.single_photon_input(m, n)
        outs = pin.random_bunched_outputs(m, n, cnt, 1000 + cnt)
        a_ref = oracle.amplitudes(U, t, outs)
        amp, _ = run_amps(pcv, U, t, outs)
        assert amp_err(amp, a_ref, m, n) <= tol(n), (m, n, cnt)


def test_photon_number_mismatch_and_bunched_input(pcv):
    m = 7
    U = pin.haar_unitary(m, 31)
    t = np.array([2, 0, 1, 0, 0, 1, 0], np.uint8)         # bunched input, n = 4
    outs = np.concatenate([pin.random_bunched_outputs(m, 4, 30, 32), pin.random_bunched_outputs(m, 3, 5, 33),
                           pin.random_bunched_outputs(m, 5, 5, 34), np.zeros((1, m), np.uint8)])
    a_ref = oracle.amplitudes(U, t, outs)
    for G in (1, 4, 8):
        amp, _ = run_amps(pcv, U, t, outs, algo=pcv.PCV_ALGO_GROUP, param=G)
        assert amp_err(amp, a_ref, m, 4) <= tol(4)
        assert np.all(amp[30:] == 0)


def test_zero_photons_and_empty_batch(pcv):
    m = 5
    U = pin.haar_unitary(m, 41)
    t = np.zeros(m, np.uint8)
    outs = np.array([[0] * 5, [1, 0, 0, 0, 0]], np.uint8)
    amp, prob = run_amps(pcv, U, t, outs)
    assert amp[0] == 1 and amp[1] == 0 and prob[0] == 1
    amp, prob = pcv.amplitudes(dev(U), pin.single_photon_input(m, 2), torch.zeros((0, m), dtype=torch.uint8, device="cuda"))
    assert amp.numel() == 0
    prob, amp = pcv.distribution(dev(U), t)
    torch.cuda.synchronize()
    assert prob.numel() == 1 and prob.item() == 1.0


def test_hong_ou_mandel_and_cnot(pcv):
    U = oracle.BS_RX_HALF
    outs = np.array([[1, 1], [2, 0], [0, 2]], np.uint8)
    amp, prob = run_amps(pcv, U, np.array([1, 1], np.uint8), outs)
    assert abs(amp[0]) < 1e-16 and abs(prob[1] - 0.5) < 1e-15 and abs(prob[2] - 0.5) < 1e-15
    C = golden_io.cnot_unitary()
    logical = [[0, 1, 0, 1, 0, 0], [0, 1, 0, 0, 1, 0], [0, 0, 1, 1, 0, 0], [0, 0, 1, 0, 1, 0]]
    expected = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]]
    for i, tin in enumerate(logical):
        _, prob = run_amps(pcv, C, np.array(tin, np.uint8), np.array(logical, np.uint8))
        assert abs(prob.sum() - 1 / 9) < 1e-15
        assert np.allclose(prob * 9, expected[i], atol=1e-14)


def test_single_mode(pcv):
    U = np.array([[0.6 + 0.8j]])
    for n in (1, 3, 7):
        prob, amp = pcv.distribution(dev(U), [n])
        torch.cuda.synchronize()
        assert abs(amp.cpu().numpy()[0] - U[0, 0] ** n) <= tol(n) * abs(U[0, 0] ** n)


# --------------------------------------------------- full distributions


@pytest.mark.parametrize("m,n,t", [(12, 6, None), (9, 5, [2, 0, 1, 0, 0, 1, 0, 1, 0]), (5, 7, [3, 1, 0, 2, 1]),
                                   (2, 1, None), (11, 2, None)])
def test_factorised_distribution_matches_oracle(pcv, m, n, t):
    U = pin.haar_unitary(m, 1200 + m + n)
    t = pin.single_photon_input(m, n) if t is None else np.array(t, np.uint8)
    p_ref, a_ref = oracle.distribution(U, t)
    # FP64 products, and pcv_distribution's own choice (the tensor-core
    # products where 2 <= n <= 10)
    for algo in (pcv.PCV_ALGO_FACTOR, pcv.PCV_ALGO_AUTO):
        prob, amp = pcv.distribution(dev(U), t, algo=algo)
        torch.cuda.synchronize()
        amp = amp.cpu().numpy()
        assert amp_err(amp, a_ref, m, n) <= tol(n), algo
        assert oracle.tvd(prob.cpu().numpy(), p_ref) <= 1e-12, algo


def test_factorised_distribution_in_several_chunks(pcv):
    # a workspace below the default forces several passes over the sign vectors
    m, n = 10, 7
    U = pin.haar_unitary(m, 1301)
    t = pin.single_photon_input(m, n)
    p_ref, a_ref = oracle.distribution(U, t)
    wsmin = pcv.abi.pcv_distribution_workspace_min(m, n)
    for want_amp in (True, False):
        ws = torch.empty(wsmin, dtype=torch.uint8, device="cuda")
        prob, amp = pcv.distribution(dev(U), t, want_amp=want_amp, ws=ws)
        torch.cuda.synchronize()
        assert oracle.tvd(prob.cpu().numpy(), p_ref) <= 1e-12
        if want_amp:
            assert amp_err(amp.cpu().numpy(), a_ref, m, n) <= tol(n)


def test_plain_kernels_in_distribution_mode(pcv):
    m, n = 8, 10
    U = pin.haar_unitary(m, 1401)
    t = np.array([2, 2, 1, 1, 1, 1, 1, 1], np.uint8)
    p_ref, a_ref = oracle.distribution(U, t)
    for kw in (dict(algo=pcv.PCV_ALGO_GROUP, param=8), dict(algo=pcv.PCV_ALGO_BLOCK, param=1),
               dict(algo=pcv.PCV_ALGO_BLOCK, param=2)):
        prob, amp = pcv.distribution(dev(U), t, **kw)
        torch.cuda.synchronize()
        assert amp_err(amp.cpu().numpy(), a_ref, m, n) <= tol(n), kw


# ---------------------------------------------- full-size workloads


def test_m20_n10_full_distribution_sampled_and_invariants(pcv):
    """The 20,030,010-output workload, in the launch configuration the bench
    times: sampled outputs against the oracle one by one, the sum rule, and
    the partial certificate P(K) (Eq. eqpk) against one Gram-matrix permanent."""
    m, n = 20, 10
    U = pin.haar_unitary(m, pin.BASE_SEED + 2)
    t = pin.single_photon_input(m, n)
    prob, amp = pcv.distribution(dev(U), t)
    torch.cuda.synchronize()
    assert prob.numel() == 20_030_010
    assert abs(prob.sum().item() - 1.0) < 1e-12
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, prob.numel() - 1], rng.integers(0, prob.numel(), 1500)]))
    occ = np.stack([pcv.unrank(m, n, int(i)) for i in idx])
    a_ref = oracle.amplitudes(U, t, occ)
    a_gpu = amp[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert amp_err(a_gpu, a_ref, m, n) <= tol(n)
    # P(K) for the last K modes: those outputs are the last C(K+n-1, n) entries of
    # the canonical order (their first photon is already in mode >= m-K); their
    # total equals the permanent of the Gram matrix of those rows of U.
    for K in (12, 16, 19):
        cnt = math.comb(K + n - 1, n)
        V = U[m - K:][:, :n]
        want = oracle.perm_ryser(V.conj().T @ V).real
        assert abs(prob[prob.numel() - cnt:].sum().item() - want) < 1e-12


@pytest.mark.parametrize("n", [16, 20, 24])
def test_large_n_sweep_sampled(pcv, n):
    m = n * n
    U = pin.haar_unitary(m, 1500 + n)
    t = pin.single_photon_input(m, n)
    outs = pin.random_outputs(m, n, 2 if n >= 24 else 4, 1600 + n)
    # above n = 16 the outputs are bunched multisets, where plain double
    # Ryser cancels too much to certify 1e-8: the double-double sum instead
    a_ref = oracle.amplitudes(U, t, outs, method="ryser_dd" if n >= 20 else "ryser")
    amp, _ = run_amps(pcv, U, t, outs)
    assert amp_err(amp, a_ref, m, n) <= tol(n)


def test_n30_rank_one_closed_form(pcv):
    """Perm(u v^T) = n! prod u prod v at the largest supported n.  (The CPU
    oracle's Ryser sum cancels too strongly at n = 30 to certify 1e-8 in
    double precision, so n = 30 is checked against closed forms.)"""
    n, m = 30, 34
    g = np.random.default_rng(30)
    u = np.exp(2j * np.pi * g.random(m)) * (0.8 + 0.4 * g.random(m))
    v = np.exp(2j * np.pi * g.random(m)) * (0.8 + 0.4 * g.random(m))
    U = np.outer(u, v)
    t = pin.single_photon_input(m, n)
    outs = np.concatenate([pin.random_outputs(m, n, 2, 31), pin.random_bunched_outputs(m, n, 2, 32)])
    want = []
    for s in outs:
        rows = np.repeat(np.arange(m), s)
        want.append(math.factorial(n) * np.prod(u[rows]) * np.prod(v[:n]) / math.sqrt(np.prod([math.factorial(k) for k in s])))
    want = np.array(want)
    for kw in (dict(), dict(algo=pcv.PCV_ALGO_BLOCK, param=64)):
        amp, _ = run_amps(pcv, U, t, outs, **kw)
        assert np.max(np.abs(amp - want) / np.abs(want)) <= tol(n), kw


def test_n30_block_diagonal_factorises(pcv):
    """U = U1 (+) U2 with 14 photons in the first block and 16 in the second:
    the 30-photon amplitude is the product of the two blocks' amplitudes."""
    m1 = m2 = 450
    U1, U2 = pin.haar_unitary(m1, 3001), pin.haar_unitary(m2, 3002)
    U = np.zeros((m1 + m2, m1 + m2), complex)
    U[:m1, :m1], U[m1:, m1:] = U1, U2
    t1, t2 = pin.single_photon_input(m1, 14), pin.single_photon_input(m2, 16)
    s1, s2 = pin.random_outputs(m1, 14, 1, 3003)[0], pin.random_outputs(m2, 16, 1, 3004)[0]
    want = oracle.amplitude(U1, t1, s1) * oracle.amplitude(U2, t2, s2)
    t = np.concatenate([t1, t2])
    outs = np.concatenate([s1, s2])[None, :]
    amp, _ = run_amps(pcv, U, t, outs, algo=pcv.PCV_ALGO_BLOCK, param=64)
    assert abs(amp[0] - want) <= tol(30) * max(abs(want), 1 / math.sqrt(math.comb(m1 + 13, 14) * math.comb(m2 + 15, 16)))


# ------------------------------------------- shared-row-sum tile kernel


@pytest.mark.parametrize("m,n,cnt", [(8, 1, 5), (8, 3, 300), (12, 6, 257), (20, 10, 513), (24, 12, 70),
                                     (30, 14, 33), (40, 17, 9), (64, 20, 3), (128, 8, 40)])
def test_tile_kernel(pcv, m, n, cnt):
    U = pin.haar_unitary(m, 2000 + m + n)
    t = pin.single_photon_input(m, n)
    outs = np.concatenate([pin.random_outputs(m, n, cnt, 2100 + n), pin.random_bunched_outputs(m, n, 3, 2200 + n),
                           pin.random_bunched_outputs(m, max(n - 1, 0), 2, 2300 + n)])
    a_ref = oracle.amplitudes(U, t, outs)
    amp, prob = run_amps(pcv, U, t, outs, algo=pcv.PCV_ALGO_TILE)
    assert amp_err(amp, a_ref, m, n) <= tol(n)
    assert np.all(amp[-2:] == 0)


def test_tile_kernel_bunched_input(pcv):
    m = 16
    U = pin.haar_unitary(m, 2401)
    t = np.zeros(m, np.uint8); t[[0, 3, 7]] = [3, 2, 4]        # n = 9
    outs = pin.random_bunched_outputs(m, 9, 100, 2402)
    a_ref = oracle.amplitudes(U, t, outs)
    amp, _ = run_amps(pcv, U, t, outs, algo=pcv.PCV_ALGO_TILE)
    assert amp_err(amp, a_ref, m, 9) <= tol(9)


# ------------------------------------------------- batched persistent


def test_batched_uneven_circuits(pcv):
    """Uneven batch (m in [8, 64], n in [4, min(16, m)]) in one persistent launch;
    every circuit's amplitudes against the oracle."""
    circs = pin.batched_circuits(24, 8, 64, 4, 16, 37, seed=2500)
    batch = [(dev(c["U"]), c["input_occ"], dev(c["outputs"])) for c in circs]
    amps, probs = pcv.amplitudes_batched(batch)
    torch.cuda.synchronize()
    for c, a, p in zip(circs, amps, probs):
        a_ref = oracle.amplitudes(c["U"], c["input_occ"], c["outputs"])
        assert amp_err(a.cpu().numpy(), a_ref, c["m"], c["n"]) <= tol(c["n"]), (c["m"], c["n"])
        assert np.allclose(p.cpu().numpy(), np.abs(a_ref) ** 2, rtol=1e-9, atol=1e-300)


def test_batched_repeat_is_deterministic(pcv):
    circs = pin.batched_circuits(12, 8, 40, 4, 12, 300, seed=2600)
    plan = pcv.BatchPlan([(dev(c["U"]), c["input_occ"], dev(c["outputs"])) for c in circs])
    first = [a.clone() for a in plan.run()[0]]
    second = plan.run()[0]
    torch.cuda.synchronize()
    for x, y in zip(first, second):
        assert torch.equal(x, y)


def test_batched_graph_replay(pcv):
    """The whole batched launch captured once as a CUDA graph: a replay gives
    the direct launch's bits, and after new unitaries are copied into the
    recorded tensors a replay gives their amplitudes (against the oracle)."""
    circs = pin.batched_circuits(16, 8, 40, 4, 14, 200, seed=2650)
    Us = [dev(c["U"]) for c in circs]
    plan = pcv.BatchPlan([(U, c["input_occ"], dev(c["outputs"])) for U, c in zip(Us, circs)])
    direct = [a.clone() for a in plan.run()[0]]
    plan.capture()
    replayed = plan.replay()[0]
    torch.cuda.synchronize()
    for x, y in zip(direct, replayed):
        assert torch.equal(x, y)
    new = [pin.haar_unitary(c["m"], 2700 + i) for i, c in enumerate(circs)]
    for U, Un in zip(Us, new):
        U.copy_(torch.from_numpy(Un))
    amps = plan.replay()[0]
    torch.cuda.synchronize()
    for c, Un, a in zip(circs, new, amps):
        a_ref = oracle.amplitudes(Un, c["input_occ"], c["outputs"])
        assert amp_err(a.cpu().numpy(), a_ref, c["m"], c["n"]) <= tol(c["n"])


def test_batched_skips_invalid_descriptor(pcv):
    # a descriptor with an input mode outside [0, m) gets no work; the others run
    circs = pin.batched_circuits(3, 8, 12, 3, 5, 10, seed=2700)
    plan = pcv.BatchPlan([(dev(c["U"]), c["input_occ"], dev(c["outputs"])) for c in circs])
    raw = plan.descs.cpu().numpy().copy()
    arr = (pcv.abi.pcv_batch_desc * 3).from_buffer_copy(raw.tobytes())
    arr[1].cols[0] = 200
    plan.descs = torch.from_numpy(np.frombuffer(bytes(arr), np.uint8).copy()).cuda()
    plan.amps[1].fill_(7)
    amps, _ = plan.run()
    torch.cuda.synchronize()
    assert torch.all(amps[1] == 7)
    for i in (0, 2):
        a_ref = oracle.amplitudes(circs[i]["U"], circs[i]["input_occ"], circs[i]["outputs"])
        assert amp_err(amps[i].cpu().numpy(), a_ref, circs[i]["m"], circs[i]["n"]) <= tol(circs[i]["n"])


def test_batched_distribution(pcv):
    m, n, B = 12, 6, 5
    Us = np.stack([pin.haar_unitary(m, 1700 + b) for b in range(B)])
    t = pin.single_photon_input(m, n)
    prob, amp = pcv.distribution_batched(dev(Us), t)
    torch.cuda.synchronize()
    for b in range(B):
        p_ref, a_ref = oracle.distribution(Us[b], t)
        assert amp_err(amp[b].cpu().numpy(), a_ref, m, n) <= tol(n)
        assert oracle.tvd(prob[b].cpu().numpy(), p_ref) <= 1e-12
    # a small workspace forces several passes over the sign vectors, per batch entry
    wsmin = pcv.abi.pcv_distribution_batched_workspace(B, m, n) // 4
    ws = torch.empty(wsmin, dtype=torch.uint8, device="cuda")
    prob2, _ = pcv.distribution_batched(dev(Us), t, want_amp=False, ws=ws)
    torch.cuda.synchronize()
    assert torch.allclose(prob2, prob, rtol=1e-12, atol=1e-18)


# ------------------------------------- state expansion (SLOS-style) path


@pytest.mark.parametrize("m,n,t", [(6, 3, None), (12, 6, None), (9, 5, [2, 0, 1, 0, 0, 1, 0, 1, 0]),
                                   (5, 7, [3, 1, 0, 2, 1]), (1, 4, [4]), (7, 1, None), (11, 2, None)])
def test_state_expansion_matches_oracle(pcv, m, n, t):
    U = pin.haar_unitary(m, 1800 + m + n)
    t = pin.single_photon_input(m, n) if t is None else np.array(t, np.uint8)
    p_ref, a_ref = oracle.distribution(U, t)
    prob, amp = pcv.distribution(dev(U), t, algo=pcv.PCV_ALGO_SLOS)
    torch.cuda.synchronize()
    assert amp_err(amp.cpu().numpy(), a_ref, m, n) <= tol(n)
    assert oracle.tvd(prob.cpu().numpy(), p_ref) <= 1e-12


def test_state_expansion_m20_n10_and_batch(pcv):
    m, n = 20, 10
    U = pin.haar_unitary(m, pin.BASE_SEED + 2)
    t = pin.single_photon_input(m, n)
    prob, amp = pcv.distribution(dev(U), t, algo=pcv.PCV_ALGO_SLOS)
    torch.cuda.synchronize()
    assert abs(prob.sum().item() - 1.0) < 1e-12
    rng = np.random.default_rng(6)
    idx = np.unique(np.concatenate([[0, prob.numel() - 1], rng.integers(0, prob.numel(), 800)]))
    occ = np.stack([pcv.unrank(m, n, int(i)) for i in idx])
    a_ref = oracle.amplitudes(U, t, occ)
    assert amp_err(amp[torch.from_numpy(idx).cuda()].cpu().numpy(), a_ref, m, n) <= tol(n)
    # batch of three unitaries through the C ABI
    B, m2, n2 = 3, 10, 5
    Us = np.stack([pin.haar_unitary(m2, 1900 + b) for b in range(B)])
    t2 = pin.single_photon_input(m2, n2)
    N = math.comb(m2 + n2 - 1, n2)
    p2 = torch.empty(B * N, dtype=torch.float64, device="cuda")
    a2 = torch.empty(B * N, dtype=torch.complex128, device="cuda")
    wsb = pcv.abi.pcv_distribution_slos_workspace(B, m2, n2)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    pcv.abi.pcv_distribution_slos(dev(Us), B, m2, t2, p2, a2, ws, wsb, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for b in range(B):
        p_ref, a_ref = oracle.distribution(Us[b], t2)
        assert amp_err(a2[b * N:(b + 1) * N].cpu().numpy(), a_ref, m2, n2) <= tol(n2)
