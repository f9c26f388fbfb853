"""Glynn's sum with multiplicities (PCV_ALGO_MULT) and the batched launch's
per-output routing, against the CPU oracle (Ryser over the expanded n x n
matrix) and closed forms.

Tolerance: relative amplitude error 1e-10 for n <= 12 and 1e-8 above, with
the same 1/sqrt(|S_{m,n}|) floor as the other parity tests."""
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


def tol(n):
    return 1e-10 if n <= 12 else 1e-8


def amp_err(got, want, m, n):
    floor = 1.0 / math.sqrt(math.comb(m + n - 1, n))
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_mult(pcv, U, t, outs, parts=1):
    amp, prob = pcv.amplitudes(dev(U), t, dev(outs), algo=pcv.PCV_ALGO_MULT, param=parts)
    torch.cuda.synchronize()
    return amp.cpu().numpy(), prob.cpu().numpy()


@pytest.mark.parametrize("m,n,cnt", [(3, 1, 4), (4, 2, 10), (6, 3, 56), (8, 5, 200), (12, 7, 300),
                                     (16, 10, 100), (20, 12, 60), (24, 14, 20)])
def test_bunched_outputs_match_oracle(pcv, m, n, cnt):
    U = pin.haar_unitary(m, 3000 + 31 * m + n)
    t = pin.single_photon_input(m, n)
    outs = np.concatenate([pin.random_bunched_outputs(m, n, cnt, 3100 + n),
                           pin.random_outputs(m, n, 5, 3200 + n),                 # collision-free
                           pin.random_bunched_outputs(m, n + 1, 2, 3300 + n)])    # wrong photon number
    a_ref = oracle.amplitudes(U, t, outs)
    amp, prob = run_mult(pcv, U, t, outs)
    assert amp_err(amp, a_ref, m, n) <= tol(n)
    assert np.all(amp[-2:] == 0) and np.all(prob[-2:] == 0)
    assert np.allclose(prob, np.abs(amp) ** 2, rtol=1e-14, atol=0)


def test_full_distribution_m6_n3_sums_to_one(pcv):
    # every output of S_{6,3}, bunched ones included, through the multiplicity kernel
    m, n = 6, 3
    U = pin.haar_unitary(m, pin.BASE_SEED)
    t = pin.single_photon_input(m, n)
    outs = oracle.enumerate_outputs(m, n)
    amp, prob = run_mult(pcv, U, t, outs)
    assert amp_err(amp, oracle.amplitudes(U, t, outs), m, n) <= 1e-12
    assert abs(prob.sum() - 1.0) <= 1e-13


def test_bunched_input_takes_the_input_side(pcv):
    # input (3, 2, 4) photons: 2 * 3 * 5 = 30 terms on the input side against
    # 2^8 on the collision-free output side
    m = 16
    U = pin.haar_unitary(m, 3401)
    t = np.zeros(m, np.uint8)
    t[[0, 3, 7]] = [3, 2, 4]
    outs = np.concatenate([pin.random_outputs(m, 9, 60, 3402), pin.random_bunched_outputs(m, 9, 60, 3403)])
    amp, _ = run_mult(pcv, U, t, outs)
    assert amp_err(amp, oracle.amplitudes(U, t, outs), m, 9) <= tol(9)


def test_even_multiplicities_only(pcv):
    # no odd multiplicity on either side: the pivot's middle term has weight 1
    m, n = 6, 8
    U = pin.haar_unitary(m, 3501)
    t = np.array([2, 2, 4, 0, 0, 0], np.uint8)
    outs = np.array([[0, 2, 0, 2, 2, 2], [4, 0, 0, 4, 0, 0], [0, 0, 8, 0, 0, 0], [2, 0, 2, 0, 4, 0]], np.uint8)
    amp, _ = run_mult(pcv, U, t, outs)
    assert amp_err(amp, oracle.amplitudes(U, t, outs), m, n) <= tol(n)


@pytest.mark.parametrize("parts", [1, 2, 3, 32, 200])
def test_warps_per_permanent(pcv, parts):
    m, n = 18, 13
    U = pin.haar_unitary(m, 3601)
    t = pin.single_photon_input(m, n)
    outs = pin.random_bunched_outputs(m, n, 7, 3602)
    amp, _ = run_mult(pcv, U, t, outs, parts)
    assert amp_err(amp, oracle.amplitudes(U, t, outs), m, n) <= tol(n)


def test_all_photons_in_one_mode_closed_form(pcv):
    # n photons from mode i to mode j: a = U[j][i]^n exactly (Perm of the
    # all-equal n x n matrix is n! u^n, the normalisation sqrt(n! n!)).  The
    # multiplicity sum is sum_k (-1)^k C(n,k) (n-2k)^n u^n / 2^n, whose terms
    # exceed the result by ~1e3 at n = 30, hence the n-dependent tolerance.
    m = 5
    U = pin.haar_unitary(m, 3701)
    for n in (1, 2, 7, 16, 30):
        for i, j in ((0, 0), (1, 3), (4, 2)):
            t = np.zeros(m, np.uint8)
            t[i] = n
            out = np.zeros((1, m), np.uint8)
            out[0, j] = n
            amp, _ = run_mult(pcv, U, t, out)
            want = U[j, i] ** n
            assert abs(amp[0] - want) <= tol(n) * abs(want), (n, i, j)


def test_n30_rank_one_closed_form(pcv):
    # U = u v^T (not unitary; the kernel does not need it): Perm of the
    # expanded matrix is n! prod u_r^{s_r} prod v_c^{t_c}
    m, n = 40, 30
    g = np.random.default_rng(3801)
    u = np.exp(1j * g.uniform(0, 2 * np.pi, m)) * g.uniform(0.9, 1.1, m)
    v = np.exp(1j * g.uniform(0, 2 * np.pi, m)) * g.uniform(0.9, 1.1, m)
    U = np.outer(u, v)
    t = pin.single_photon_input(m, n)
    outs = pin.random_bunched_outputs(m, n, 12, 3802)
    amp, _ = run_mult(pcv, U, t, outs)
    for k in range(outs.shape[0]):
        s = outs[k].astype(int)
        want = math.factorial(n) * np.prod(u ** s) * np.prod(v[:n]) / math.sqrt(
            np.prod([math.factorial(x) for x in s]))
        assert abs(amp[k] - want) <= 1e-8 * abs(want), k


def ref_amplitudes(U, t, outs, n):
    # at n >= 20 the plain double Ryser sum loses digits to cancellation; the
    # double-double one does not
    return oracle.amplitudes(U, t, outs, method="ryser_dd" if n >= 20 else "ryser")


def test_n20_bunched_against_oracle(pcv):
    m, n = 26, 20
    U = pin.haar_unitary(m, 3901)
    t = pin.single_photon_input(m, n)
    outs = pin.random_bunched_outputs(m, n, 6, 3902)
    amp, _ = run_mult(pcv, U, t, outs)
    assert amp_err(amp, ref_amplitudes(U, t, outs, n), m, n) <= tol(n)


# ---------------------------------------------------- batched routing


def _batch(pcv, circs, algo):
    plan = pcv.BatchPlan([(dev(c["U"]), c["input_occ"], dev(c["outputs"])) for c in circs], algo=algo)
    amps, probs = plan.run()
    torch.cuda.synchronize()
    return [a.cpu().numpy() for a in amps], [p.cpu().numpy() for p in probs]


def _bunched_circuits(seed):
    # uneven circuits whose outputs are uniform multisets (bunched), with a
    # few collision-free ones mixed in, so that both kernels get outputs
    circs = pin.batched_circuits(14, 6, 24, 3, 18, 9, seed=seed)
    for k, c in enumerate(circs):
        c["outputs"] = np.concatenate([pin.random_bunched_outputs(c["m"], c["n"], 9, seed + 50 + k),
                                       pin.random_outputs(c["m"], min(c["n"], 16), 2, seed + 90 + k)
                                       if c["n"] <= 16 else pin.random_bunched_outputs(c["m"], c["n"], 2, seed + 90 + k)])
    return circs


@pytest.mark.parametrize("route", ["AUTO", "TILE", "MULT"])
def test_batched_routes_match_oracle(pcv, route):
    circs = _bunched_circuits(4000)
    amps, probs = _batch(pcv, circs, getattr(pcv, "PCV_ALGO_" + route))
    for c, a, p in zip(circs, amps, probs):
        a_ref = oracle.amplitudes(c["U"], c["input_occ"], c["outputs"])
        assert amp_err(a, a_ref, c["m"], c["n"]) <= tol(c["n"]), (route, c["m"], c["n"])
        assert np.allclose(p, np.abs(a_ref) ** 2, rtol=1e-8, atol=1e-300)


def test_batched_auto_is_deterministic_and_agrees_with_tile(pcv):
    circs = _bunched_circuits(4100)
    plan = pcv.BatchPlan([(dev(c["U"]), c["input_occ"], dev(c["outputs"])) for c in circs])
    first = [a.clone() for a in plan.run()[0]]
    second = plan.run()[0]
    torch.cuda.synchronize()
    for x, y in zip(first, second):
        assert torch.equal(x, y)
    tile, _ = _batch(pcv, circs, pcv.PCV_ALGO_TILE)
    for c, a, b in zip(circs, first, tile):
        assert amp_err(a.cpu().numpy(), b, c["m"], c["n"]) <= tol(c["n"])


def test_batched_workload_shape_sampled(pcv):
    # the 512-circuit uneven workload's shape (m in [8, 64], n in [4, 24],
    # stars-and-bars outputs above n = 16) at reduced output counts; the n >= 20
    # circuits are checked on a few outputs each
    circs = pin.batched_circuits(40, 8, 64, 4, 24, 64, seed=pin.BASE_SEED + 3)
    amps, _ = _batch(pcv, circs, pcv.PCV_ALGO_AUTO)
    for c, a in zip(circs, amps):
        k = 64 if c["n"] <= 16 else (8 if c["n"] < 20 else 2)
        a_ref = ref_amplitudes(c["U"], c["input_occ"], c["outputs"][:k], c["n"])
        assert amp_err(a[:k], a_ref, c["m"], c["n"]) <= tol(c["n"]), (c["m"], c["n"])


def test_auto_routes_single_circuit_explicit_outputs(pcv):
    # enough outputs for the tile regime (m <= 128, n = 14: 152 x 64 outputs):
    # AUTO routes each output to the tile kernel or to the multiplicity kernel
    m, n = 30, 14
    U = pin.haar_unitary(m, 4201)
    t = pin.single_photon_input(m, n)
    outs = np.concatenate([pin.random_bunched_outputs(m, n, 6000, 4202), pin.random_outputs(m, n, 4000, 4203)])
    assert pcv.abi.pcv_amplitudes_workspace(m, n, outs.shape[0]) > 0
    auto, _ = pcv.amplitudes(dev(U), t, dev(outs))
    tile, _ = pcv.amplitudes(dev(U), t, dev(outs), algo=pcv.PCV_ALGO_TILE)
    torch.cuda.synchronize()
    auto, tile = auto.cpu().numpy(), tile.cpu().numpy()
    assert amp_err(auto, tile, m, n) <= tol(n)
    pick = np.r_[0:40, 5980:6040, 9960:10000]
    assert amp_err(auto[pick], oracle.amplitudes(U, t, outs[pick]), m, n) <= tol(n)


def test_batched_workload_full_size_sampled():
    """The 512-circuit x 4096-output uneven workload in the launch configuration
    the workload runner times (AUTO routing): every amplitude finite with
    prob = |amp|^2 <= 1; two outputs of every circuit with n <= 16 and one
    output of 16 seeded circuits with n >= 17 against the oracle."""
    import paper_2204_00602_gb300 as pcv
    g = np.random.default_rng(pin.BASE_SEED + 3)
    circs = []
    for c in range(512):                       # the workload runner's recipe
        m = int(g.integers(8, 65))
        n = int(g.integers(4, min(24, m) + 1))
        circs.append(dict(m=m, n=n, U=pin.haar_unitary(m, pin.BASE_SEED + 3 + 1000 + c),
                          input_occ=pin.single_photon_input(m, n),
                          outputs=pin.random_outputs(m, n, 4096, pin.BASE_SEED + 3 + 5000 + c)))
    amps, probs = _batch(pcv, circs, pcv.PCV_ALGO_AUTO)
    pick = np.random.default_rng(4301)
    big = [i for i, c in enumerate(circs) if c["n"] >= 17]
    checked_big = set(pick.choice(big, size=16, replace=False).tolist())
    for i, (c, a, p) in enumerate(zip(circs, amps, probs)):
        assert np.all(np.isfinite(a)) and np.all(p <= 1.0)
        assert np.allclose(p, np.abs(a) ** 2, rtol=1e-12, atol=0)
        if c["n"] <= 16:
            k = pick.choice(4096, size=2, replace=False)
        elif i in checked_big:
            k = pick.choice(4096, size=1)
        else:
            continue
        ref = ref_amplitudes(c["U"], c["input_occ"], c["outputs"][k], c["n"])
        assert amp_err(a[k], ref, c["m"], c["n"]) <= tol(c["n"]), (i, c["m"], c["n"])
