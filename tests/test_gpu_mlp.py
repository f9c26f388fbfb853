"""BF16 MLP surrogate kernels on the GPU (through the C ABI) against the CPU
reference oracle/mlp.py.  FP32-accumulated results are compared with the
FP64 reference within the accumulation bound K 2^-24 sum|a b|; BF16-stored
results within one BF16 rounding (2^-8 relative) of the reference computed
from the same BF16 inputs."""
import io
import math

import numpy as np
import pytest

import pcv_inputs as pin
from oracle import mlp as ref

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


def S():
    return torch.cuda.current_stream().cuda_stream


def bf16_dev(x):
    return torch.from_numpy(np.asarray(x, np.float32)).cuda().to(torch.bfloat16)


def to64(t):
    return t.float().cpu().numpy().astype(np.float64)


def rand(shape, seed, scale=1.0):
    return ref.bf16(np.random.default_rng(seed).standard_normal(shape) * scale)


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 200, 96), (7, 33, 64), (4096, 1024, 1024), (1024, 288, 4096)])
def test_gemm_modes(pcv, M, N, K):
    abi = pcv.abi
    A, B = rand((M, K), 1), rand((N, K), 2)
    bias = np.random.default_rng(3).standard_normal(N).astype(np.float32)
    Ad, Bd, bd = bf16_dev(A), bf16_dev(B), torch.from_numpy(bias).cuda()
    C = ref.gemm(A, B)
    bound = ref.gemm_error_bound(A, B, K)
    out = torch.empty(M, N, dtype=torch.float32, device="cuda")
    abi.pcv_gemm_bf16(Ad, K, Bd, K, M, N, K, 0, None, out, N, None, 0, None, 0, S())
    assert np.all(np.abs(out.cpu().numpy() - C) <= bound)
    abi.pcv_gemm_bf16(Ad, K, Bd, K, M, N, K, 2, bd, out, N, None, 0, None, 0, S())
    assert np.all(np.abs(out.cpu().numpy() - (C + bias)) <= bound + 1e-6 * np.abs(bias))
    pre = torch.empty(M, N, dtype=torch.float32, device="cuda")
    act = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.pcv_gemm_bf16(Ad, K, Bd, K, M, N, K, 1, bd, pre, N, act, N, None, 0, S())
    pre_ref = C + bias
    assert np.all(np.abs(pre.cpu().numpy() - pre_ref) <= bound + 1e-6 * np.abs(bias))
    g = ref.gelu(pre.cpu().numpy().astype(np.float64))
    assert np.all(np.abs(to64(act) - g) <= 2 ** -8 * np.abs(g) + 1e-6)
    # mode 3: C * gelu'(pre)
    P = np.random.default_rng(4).standard_normal((M, N)).astype(np.float32)
    outb = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.pcv_gemm_bf16(Ad, K, Bd, K, M, N, K, 3, None, None, 0, outb, N, torch.from_numpy(P).cuda(), N, S())
    want = C * ref.gelu_grad(P.astype(np.float64))
    assert np.all(np.abs(to64(outb) - want) <= 2 ** -8 * np.abs(want) + 2 * bound * np.abs(ref.gelu_grad(P)) + 1e-6)


def test_small_kernels(pcv):
    abi = pcv.abi
    g = np.random.default_rng(9)
    X = rand((100, 70), 10)
    Xd = bf16_dev(X)
    XT = torch.empty(70, 100, dtype=torch.bfloat16, device="cuda")
    abi.pcv_transpose_bf16(Xd, 100, 70, 70, XT, 100, S())
    assert np.array_equal(to64(XT), X.T)
    db = torch.empty(70, dtype=torch.float32, device="cuda")
    abi.pcv_colsum_bf16(Xd, 100, 70, 70, db, S())
    assert np.allclose(db.cpu().numpy(), X.sum(0), rtol=1e-5, atol=1e-5)
    ph = pin.mesh_phases(5, 132, 11)
    F = torch.empty(5, 288, dtype=torch.bfloat16, device="cuda")
    abi.pcv_phase_features(torch.from_numpy(ph).cuda(), 5, 132, F, 288, S())
    assert np.array_equal(to64(F), ref.features(ph, 288))
    dX = g.standard_normal((5, 288)).astype(np.float32)
    gp = torch.empty(5, 132, dtype=torch.float64, device="cuda")
    abi.pcv_phase_features_grad(torch.from_numpy(ph).cuda(), 5, 132, torch.from_numpy(dX).cuda(), 288, gp, S())
    want = dX[:, :132] * np.cos(ph) - dX[:, 132:264] * np.sin(ph)
    assert np.allclose(gp.cpu().numpy(), want, rtol=1e-12, atol=1e-12)
    pred = g.standard_normal(10000).astype(np.float32)
    tgt = g.standard_normal(10000).astype(np.float32)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dy = torch.empty(10000, dtype=torch.bfloat16, device="cuda")
    ws = torch.empty(abi.pcv_mse_workspace(), dtype=torch.uint8, device="cuda")
    abi.pcv_mse(torch.from_numpy(pred).cuda(), torch.from_numpy(tgt).cuda(), 10000, loss, dy, ws, ws.numel(), S())
    L, d = ref.mse(pred, tgt)
    assert abs(loss.item() - L) < 1e-5 * L
    assert np.all(np.abs(to64(dy) - d) <= 2 ** -8 * np.abs(d))
    w0, gr = g.standard_normal(1000).astype(np.float32), g.standard_normal(1000).astype(np.float32)
    w, m, v = (torch.from_numpy(a.copy()).cuda() for a in (w0, np.zeros(1000, np.float32), np.zeros(1000, np.float32)))
    wb = torch.empty(1000, dtype=torch.bfloat16, device="cuda")
    abi.pcv_adam(w, m, v, torch.from_numpy(gr).cuda(), 1000, 1e-3, 0.9, 0.999, 1e-8, 1, wb, S())
    rw, _, _ = ref.adam(w0.astype(np.float64), 0, 0, gr.astype(np.float64), 1e-3, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(w.cpu().numpy(), rw, rtol=0, atol=1e-6)
    assert np.array_equal(to64(wb), ref.bf16(w.cpu().numpy()))


def _net(pcv, seed=21, lr=1e-3, tc="tcgen05"):
    from paper_2204_00602_gb300 import surrogate
    Ws, bs = surrogate.init_weights(seed)
    return surrogate, surrogate.MLP(Ws, bs, lr=lr, tensor_core=tc), Ws, bs


TC = pytest.mark.parametrize("tc", ["tcgen05", "mma_sync"])


@TC
def test_mlp_forward_backward_layer_by_layer(pcv, tc):
    surrogate, net, Ws, bs = _net(pcv, tc=tc)
    B = 256
    ph = torch.from_numpy(pin.mesh_phases(B, 132, 22)).cuda()
    X = net.features(ph)
    y = net.forward(X)
    Wr = [ref.bf16(W) for W in Ws]
    # each layer from the GPU's own bf16 input
    for l in range(4):
        h = to64(net.acts[l])
        pre = ref.gemm(h, Wr[l]) + bs[l]
        bound = ref.gemm_error_bound(h, Wr[l], Wr[l].shape[1]) + 1e-6 * np.abs(bs[l])
        got = (net.pres[l] if l < 3 else y).cpu().numpy()
        assert np.all(np.abs(got - pre) <= bound), l
        if l < 3:
            gg = ref.gelu(got.astype(np.float64))
            assert np.all(np.abs(to64(net.acts[l + 1]) - gg) <= 2 ** -8 * np.abs(gg) + 1e-6)
    # backward for a random upstream gradient, layer by layer
    dy = bf16_dev(rand((B, 512), 23, 1e-3))
    net.backward(dy, want_input_grad=True)
    dY = to64(dy)
    for l in reversed(range(4)):
        h = to64(net.acts[l])
        gW = ref.gemm(dY.T, h.T)
        assert np.all(np.abs(net.gW[l].cpu().numpy() - gW) <= ref.gemm_error_bound(dY.T, h.T, B)), l
        assert np.allclose(net.gb[l].cpu().numpy(), dY.sum(0), rtol=1e-4, atol=1e-7)
        if l > 0:
            dprev = to64(net._bufs[f"dY{l - 1}"])
            full = ref.gemm(dY, Wr[l].T) * ref.gelu_grad(net.pres[l - 1].cpu().numpy().astype(np.float64))
            assert np.all(np.abs(dprev - full) <= 2 ** -8 * np.abs(full) +
                          2 * ref.gemm_error_bound(dY, Wr[l].T, Wr[l].shape[0]))
            dY = dprev
        else:
            dX = ref.gemm(dY, Wr[0].T)
            assert np.all(np.abs(net._bufs["dX0"].cpu().numpy() - dX) <= ref.gemm_error_bound(dY, Wr[0].T, 512) + 1e-9)


@TC
def test_mlp_training_reduces_loss_and_resumes_bitwise(pcv, tc):
    surrogate, net, Ws, bs = _net(pcv, lr=1e-3, tc=tc)
    B = 512
    g = np.random.default_rng(30)
    ph = torch.from_numpy(pin.mesh_phases(B, 132, 31)).cuda()
    X = net.features(ph).clone()
    tgt = torch.from_numpy(g.standard_normal((B, 512)).astype(np.float32) * 0.1 - 3.0).cuda()
    losses = [net.train_step(X, tgt).item() for _ in range(40)]
    assert losses[-1] < 0.2 * losses[0]
    # checkpoint / resume: k steps + save/load + j steps == k + j steps
    _, a, _, _ = _net(pcv, seed=40, tc=tc)
    _, b, _, _ = _net(pcv, seed=40, tc=tc)
    for _ in range(5):
        a.train_step(X, tgt)
        b.train_step(X, tgt)
    f = io.BytesIO()
    b.save(f)
    f.seek(0)
    c = surrogate.MLP.load(f, tensor_core=tc)
    for _ in range(4):
        a.train_step(X, tgt)
        c.train_step(X, tgt)
    torch.cuda.synchronize()
    for wa, wc in zip(a.W, c.W):
        assert torch.equal(wa, wc)
    for n_ in (net, a, c):
        n_.check()


@TC
def test_phase_gradient_of_the_surrogate(pcv, tc):
    # d(sum y)/dphi through the network against central differences of an FP64
    # evaluation of the same BF16 weights (no activation rounding)
    surrogate, net, Ws, bs = _net(pcv, seed=50, tc=tc)
    ph = pin.mesh_phases(2, 132, 51)
    phd = torch.from_numpy(ph).cuda()
    net.predict_phases(phd)
    dy = torch.full((2, 512), 1.0, dtype=torch.bfloat16, device="cuda")
    g = net.grad_phases(phd, dy).cpu().numpy()
    # reference: fp64 network on the same bf16 weights without activation rounding
    Wr = [ref.bf16(W) for W in Ws]

    def f(p):
        X = np.zeros((1, 288))
        X[0, :132], X[0, 132:264], X[0, 264] = np.sin(p), np.cos(p), 1.0
        h = X
        for l in range(3):
            h = ref.gelu(ref.gemm(h, Wr[l]) + bs[l])
        return float(np.sum(ref.gemm(h, Wr[3]) + bs[3]))
    h = 1e-5
    for q in range(0, 132, 11):
        e = np.zeros(132); e[q] = h
        fd = (f(ph[0] + e) - f(ph[0] - e)) / (2 * h)
        assert abs(g[0, q] - fd) <= 0.03 * max(1.0, abs(fd))


def test_exact_training_targets(pcv):
    from paper_2204_00602_gb300 import surrogate
    import oracle
    m, n = 12, 6
    outs = surrogate.output_set(m, n, 512, pin.BASE_SEED + 5)
    assert len({tuple(o) for o in outs}) == 512 and np.all(outs.sum(1) == n)
    ph = pin.mesh_phases(4, 132, 60)
    lp = surrogate.exact_log_probs(torch.from_numpy(ph).cuda(), m, pin.single_photon_input(m, n),
                                   torch.from_numpy(outs).cuda()).cpu().numpy()
    for b in range(4):
        p = np.abs(oracle.amplitudes(oracle.mesh(ph[b]), pin.single_photon_input(m, n), outs)) ** 2
        assert np.allclose(lp[b], np.log(p).astype(np.float32), rtol=1e-6, atol=1e-6)
