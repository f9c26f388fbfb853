"""Learned surrogate of the mesh's output probabilities (not in the paper).

An MLP maps the features (sin phi, cos phi) of the 132 phases of the m=12
Clements mesh to log P(S) of a fixed set of 512 outputs: 264 (+1 bias, padded
to 288) -> 1024 -> 1024 -> 1024 (GELU) -> 512.  Weights and activations are
BF16, products accumulate in FP32 on the tensor cores, master weights and
Adam state are FP32.  Every step (features, GEMMs with fused bias/GELU,
transposes, bias gradients, MSE, Adam) runs in the library's kernels; torch
only owns the buffers.  The GEMMs run on the 5th-generation tensor cores
(tcgen05 + TMEM, TMA-staged operands) by default; `tensor_core="mma_sync"`
selects the warp-level mma.sync kernel.

Training data come from the exact kernels: U(phi) by the mesh kernel, then the
512 amplitudes per phase set by the shared-row-sum tile kernel.
"""
from __future__ import annotations

import io

import numpy as np
import torch

from . import _abi as abi
from . import _stream, num_outputs, unrank
from .autograd import mesh_unitary

P_MESH = 132           # phases of the m=12 mesh
IN_PAD = 288           # 2*132 features + 1 constant, padded to a multiple of 32
DIMS = (IN_PAD, 1024, 1024, 1024, 512)


def _bf16(shape, dev):
    return torch.empty(shape, dtype=torch.bfloat16, device=dev)


def _f32(shape, dev):
    return torch.empty(shape, dtype=torch.float32, device=dev)


def init_weights(seed: int, dims=DIMS, n_features: int = 2 * P_MESH + 1):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (numpy,
    seeded); the padded input columns of the first layer are zero."""
    g = np.random.default_rng(seed)
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        fan_in = n_features if l == 0 else dims[l]
        lim = 1.0 / np.sqrt(fan_in)
        W = g.uniform(-lim, lim, size=(dims[l + 1], dims[l])).astype(np.float32)
        if l == 0:
            W[:, n_features:] = 0.0
        Ws.append(W)
        bs.append(g.uniform(-lim, lim, size=dims[l + 1]).astype(np.float32))
    return Ws, bs


class MLP:
    """Device-resident surrogate network with Adam state."""

    def __init__(self, Ws, bs, device="cuda", lr=1e-3, betas=(0.9, 0.999), eps=1e-8, tensor_core: str = "tcgen05"):
        self.dev = torch.device(device)
        if tensor_core not in ("tcgen05", "mma_sync"):
            raise ValueError("tensor_core must be 'tcgen05' or 'mma_sync'")
        self.tensor_core = tensor_core
        self.error = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.L = len(Ws)
        self.dims = [Ws[0].shape[1]] + [W.shape[0] for W in Ws]
        self.W = [torch.from_numpy(np.ascontiguousarray(W, np.float32)).to(self.dev) for W in Ws]
        self.b = [torch.from_numpy(np.ascontiguousarray(b, np.float32)).to(self.dev) for b in bs]
        self.mW = [torch.zeros_like(w) for w in self.W]
        self.vW = [torch.zeros_like(w) for w in self.W]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.Wb = [_bf16(w.shape, self.dev) for w in self.W]                       # [out, in]
        self.WTb = [_bf16((w.shape[1], w.shape[0]), self.dev) for w in self.W]     # [in, out]
        self.lr, self.betas, self.eps = lr, betas, eps
        self.step_count = 0
        self._mse_ws = torch.empty(abi.pcv_mse_workspace(), dtype=torch.uint8, device=self.dev)
        self._bufs = {}
        self.refresh_bf16()

    # ------------------------------------------------------------ helpers
    @property
    def stream(self):
        return _stream(self.dev)

    def refresh_bf16(self):
        for l in range(self.L):
            abi.pcv_f32_to_bf16(self.W[l], self.W[l].numel(), self.Wb[l], self.stream)
            o, i = self.W[l].shape
            abi.pcv_transpose_bf16(self.Wb[l], o, i, i, self.WTb[l], o, self.stream)

    def _buf(self, name, shape, dtype):
        t = self._bufs.get(name)
        if t is None or tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            t = torch.empty(shape, dtype=dtype, device=self.dev)
            self._bufs[name] = t
        return t

    def gemm(self, A, lda, B, ldb, M, N, K, mode, bias, outf, ldo, outb, ldob, pre, ldp):
        """C = A B^T with a fused epilogue on the BF16 tensor cores (tcgen05 by default)."""
        if self.tensor_core == "tcgen05":
            abi.pcv_gemm_bf16_tc(A, lda, B, ldb, M, N, K, mode, bias, outf, ldo, outb, ldob, pre, ldp, self.error,
                                 self.stream)
        else:
            abi.pcv_gemm_bf16(A, lda, B, ldb, M, N, K, mode, bias, outf, ldo, outb, ldob, pre, ldp, self.stream)

    def check(self):
        """Raise if a tcgen05 pipeline wait gave up since the last check (host sync)."""
        code = int(self.error.cpu().numpy()[0])
        if code:
            self.error.zero_()
            raise RuntimeError(f"tcgen05 GEMM pipeline wait gave up (code {code})")

    def features(self, phases: torch.Tensor) -> torch.Tensor:
        B = phases.shape[0]
        X = self._buf("X", (B, self.dims[0]), torch.bfloat16)
        abi.pcv_phase_features(phases.contiguous(), B, phases.shape[1], X, self.dims[0], self.stream)
        return X

    # ------------------------------------------------------------ forward
    def forward(self, X: torch.Tensor) -> torch.Tensor:
        """X bf16 [B, in] -> predictions fp32 [B, 512]; keeps activations for backward."""
        B = X.shape[0]
        self.acts, self.pres = [X], []
        h = X
        for l in range(self.L):
            o, i = self.W[l].shape
            if l + 1 < self.L:
                pre = self._buf(f"pre{l}", (B, o), torch.float32)
                out = self._buf(f"act{l}", (B, o), torch.bfloat16)
                self.gemm(h, i, self.Wb[l], i, B, o, i, 1, self.b[l], pre, o, out, o, None, 0)
                self.pres.append(pre)
                self.acts.append(out)
                h = out
            else:
                y = self._buf("y", (B, o), torch.float32)
                self.gemm(h, i, self.Wb[l], i, B, o, i, 2, self.b[l], y, o, None, 0, None, 0)
                return y
        raise RuntimeError("no layers")

    # ----------------------------------------------------------- backward
    def backward(self, dy_bf16: torch.Tensor, want_input_grad: bool = False, want_param_grad: bool = True):
        """dy bf16 [B, 512] -> parameter gradients (fp32) and optionally dL/dX (fp32 [B, in])."""
        B = dy_bf16.shape[0]
        if want_param_grad and B % 32:
            raise ValueError("training batch must be a multiple of 32")
        self.gW, self.gb = [None] * self.L, [None] * self.L
        dY = dy_bf16
        dX0 = None
        for l in reversed(range(self.L)):
            o, i = self.W[l].shape
            if want_param_grad:
                dYT = self._buf(f"dYT{l}", (o, B), torch.bfloat16)
                XT = self._buf(f"XT{l}", (i, B), torch.bfloat16)
                abi.pcv_transpose_bf16(dY, B, o, o, dYT, B, self.stream)
                abi.pcv_transpose_bf16(self.acts[l], B, i, i, XT, B, self.stream)
                gW = self._buf(f"gW{l}", (o, i), torch.float32)
                self.gemm(dYT, B, XT, B, o, i, B, 0, None, gW, i, None, 0, None, 0)
                gb = self._buf(f"gb{l}", (o,), torch.float32)
                abi.pcv_colsum_bf16(dY, B, o, o, gb, self.stream)
                self.gW[l], self.gb[l] = gW, gb
            if l > 0:
                dprev = self._buf(f"dY{l - 1}", (B, i), torch.bfloat16)
                self.gemm(dY, o, self.WTb[l], o, B, i, o, 3, None, None, 0, dprev, i, self.pres[l - 1], i)
                dY = dprev
            elif want_input_grad:
                dX0 = self._buf("dX0", (B, i), torch.float32)
                self.gemm(dY, o, self.WTb[0], o, B, i, o, 0, None, dX0, i, None, 0, None, 0)
        return dX0

    def adam_step(self):
        self.step_count += 1
        b1, b2 = self.betas
        for l in range(self.L):
            abi.pcv_adam(self.W[l], self.mW[l], self.vW[l], self.gW[l], self.W[l].numel(), self.lr, b1, b2, self.eps,
                         self.step_count, self.Wb[l], self.stream)
            abi.pcv_adam(self.b[l], self.mb[l], self.vb[l], self.gb[l], self.b[l].numel(), self.lr, b1, b2, self.eps,
                         self.step_count, None, self.stream)
            o, i = self.W[l].shape
            abi.pcv_transpose_bf16(self.Wb[l], o, i, i, self.WTb[l], o, self.stream)

    def loss(self, y: torch.Tensor, target: torch.Tensor, want_grad: bool = True):
        """MSE(y, target); returns (loss tensor [1] fp32, dy bf16 or None)."""
        out = self._buf("loss", (1,), torch.float32)
        dy = self._buf("dy", tuple(y.shape), torch.bfloat16) if want_grad else None
        abi.pcv_mse(y, target, y.numel(), out, dy, self._mse_ws, self._mse_ws.numel(), self.stream)
        return out, dy

    def train_step(self, X: torch.Tensor, target: torch.Tensor):
        y = self.forward(X)
        loss, dy = self.loss(y, target)
        self.backward(dy)
        self.adam_step()
        return loss

    def predict_phases(self, phases: torch.Tensor) -> torch.Tensor:
        return self.forward(self.features(phases))

    def grad_phases(self, phases: torch.Tensor, dy_bf16: torch.Tensor) -> torch.Tensor:
        """dL/dphi given dL/dy (bf16 [B, 512]) for the last forward(features(phases))."""
        dX = self.backward(dy_bf16, want_input_grad=True, want_param_grad=False)
        g = torch.empty_like(phases)
        abi.pcv_phase_features_grad(phases.contiguous(), phases.shape[0], phases.shape[1], dX, dX.shape[1], g,
                                    self.stream)
        return g

    # ------------------------------------------------------- checkpoints
    def state_dict(self):
        cpu = lambda ts: [t.detach().cpu().clone() for t in ts]
        return {"W": cpu(self.W), "b": cpu(self.b), "mW": cpu(self.mW), "vW": cpu(self.vW), "mb": cpu(self.mb),
                "vb": cpu(self.vb), "step": self.step_count, "lr": self.lr, "betas": self.betas, "eps": self.eps}

    def save(self, f):
        torch.save(self.state_dict(), f)

    @classmethod
    def load(cls, f, device="cuda", tensor_core: str = "tcgen05"):
        sd = torch.load(f, map_location="cpu")
        net = cls([w.numpy() for w in sd["W"]], [b.numpy() for b in sd["b"]], device, sd["lr"], tuple(sd["betas"]),
                  sd["eps"], tensor_core)
        for dst, src in ((net.mW, sd["mW"]), (net.vW, sd["vW"]), (net.mb, sd["mb"]), (net.vb, sd["vb"])):
            for d, s in zip(dst, src):
                d.copy_(s.to(net.dev))
        net.step_count = sd["step"]
        return net


# ---------------------------------------------------------------- data

def output_set(m: int, n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct outputs drawn by seeded uniform rank sampling from
    S_{m,n}, as uint8 occupations [count, m] in increasing rank order."""
    N = num_outputs(m, n)
    ranks = np.sort(np.random.default_rng(seed).choice(N, size=count, replace=False))
    return np.stack([unrank(m, n, int(r)) for r in ranks])


def exact_log_probs(phases: torch.Tensor, m: int, input_occ, outs_dev: torch.Tensor, chunk: int = 32768):
    """log P(S) (fp32 [B, n_out]) of the outputs for each phase set: mesh
    kernel, then the tile kernel on all unitaries of a chunk."""
    B = phases.shape[0]
    n_out = outs_dev.shape[0]
    t = np.ascontiguousarray(np.asarray(input_occ, np.uint8))
    out = torch.empty(B, n_out, dtype=torch.float32, device=phases.device)
    prob = torch.empty(min(chunk, B), n_out, dtype=torch.float64, device=phases.device)
    for s in range(0, B, chunk):
        e = min(B, s + chunk)
        U = mesh_unitary(phases[s:e], m)
        p = prob[: e - s]
        abi.pcv_amplitudes_multi(U, e - s, m, t, outs_dev, n_out, None, p, _stream(phases.device))
        abi.pcv_log_f64_to_f32(p, p.numel(), out[s:e], _stream(phases.device))
    return out


def exact_probs(phases: torch.Tensor, m: int, input_occ, outs_dev: torch.Tensor) -> torch.Tensor:
    B = phases.shape[0]
    n_out = outs_dev.shape[0]
    prob = torch.empty(B, n_out, dtype=torch.float64, device=phases.device)
    U = mesh_unitary(phases, m)
    abi.pcv_amplitudes_multi(U, B, m, np.ascontiguousarray(np.asarray(input_occ, np.uint8)), outs_dev, n_out, None,
                             prob, _stream(phases.device))
    return prob
