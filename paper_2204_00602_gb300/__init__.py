"""GB300 (sm_103a) strong simulation of linear-optical interferometers.

Output amplitudes a(S) = Perm(U_{T,S}) / sqrt(prod s! prod t!) (Eq. eqperm of
the Perceval paper, arXiv 2204.00602, Sec. 4.2) computed by hand-written
complex-FP64 Glynn kernels behind the C ABI of libpcv.so (include/pcv.h).

This module only marshals arguments: tensors live on the GPU (torch is used
for device memory and streams), every step of the computation runs in the
library's kernels, and a missing library is an ImportError.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi as abi
from ._abi import (PCV_ALGO_AUTO, PCV_ALGO_BLOCK, PCV_ALGO_FACTOR, PCV_ALGO_GROUP,  # noqa: F401
                   PCV_ALGO_FACTOR_TC, PCV_ALGO_MULT, PCV_ALGO_SLOS, PCV_ALGO_TILE, PCV_MAX_MODES,
                   PCV_MAX_PHOTONS, PcvError)

__all__ = ["amplitudes", "amplitudes_batched", "BatchPlan", "distribution", "distribution_batched",
           "distribution_range", "distribution_status", "distribution_classes", "source_distribution", "sample", "num_outputs", "unrank", "rank",
           "fp64_probe", "PcvError", "PCV_ALGO_AUTO", "PCV_ALGO_GROUP", "PCV_ALGO_BLOCK", "PCV_ALGO_FACTOR",
           "PCV_ALGO_TILE", "PCV_ALGO_SLOS", "PCV_ALGO_MULT", "PCV_ALGO_FACTOR_TC", "abi"]


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _host_occ(occ, m: int) -> np.ndarray:
    if isinstance(occ, torch.Tensor):
        occ = occ.detach().cpu().numpy()
    a = np.ascontiguousarray(np.asarray(occ, dtype=np.uint8).reshape(-1))
    if a.shape[0] != m:
        raise ValueError(f"occupation has {a.shape[0]} modes, expected {m}")
    return a


def _check_U(U: torch.Tensor) -> int:
    if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == torch.complex128 and U.dim() == 2
            and U.shape[0] == U.shape[1]):
        raise TypeError("U must be a square complex128 CUDA tensor")
    return U.shape[0]


def workspace(nbytes: int, device) -> torch.Tensor | None:
    """Device scratch for the library (torch's allocator aligns to 512 bytes)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device) if nbytes > 0 else None


def num_outputs(m: int, n: int) -> int:
    """|S_{m,n}| = C(m+n-1, n)."""
    return abi.pcv_num_outputs(m, n)


def unrank(m: int, n: int, idx: int) -> np.ndarray:
    """Occupation of canonical output `idx` (lexicographic non-decreasing mode list)."""
    occ = np.zeros(m, dtype=np.uint8)
    abi.pcv_unrank(m, n, idx, occ)
    return occ


def rank(occ) -> int:
    a = np.ascontiguousarray(np.asarray(occ, dtype=np.uint8))
    return abi.pcv_rank(a.shape[0], a)


def amplitudes(U: torch.Tensor, input_occ, outputs: torch.Tensor, *, algo: int = PCV_ALGO_AUTO,
               param: int = 0, want_prob: bool = True, ws: torch.Tensor | None = None):
    """Amplitudes (and probabilities) of explicit outputs.

    U: complex128 [m, m] CUDA; input_occ: m photon counts (host);
    outputs: uint8 [n_out, m] CUDA.  Returns (amp complex128 [n_out], prob float64 [n_out] or None).
    """
    m = _check_U(U)
    t = _host_occ(input_occ, m)
    if not (outputs.is_cuda and outputs.dtype == torch.uint8 and outputs.dim() == 2 and outputs.shape[1] == m):
        raise TypeError("outputs must be a uint8 CUDA tensor [n_out, m]")
    U = U.contiguous()
    outputs = outputs.contiguous()
    n_out = outputs.shape[0]
    amp = torch.empty(n_out, dtype=torch.complex128, device=U.device)
    prob = torch.empty(n_out, dtype=torch.float64, device=U.device) if want_prob else None
    n = int(t.sum())
    if ws is None:
        need = abi.pcv_amplitudes_ex_workspace(m, n, n_out, algo, param)
        ws = workspace(need, U.device)
    abi.pcv_amplitudes_ex(U, m, t, outputs, n_out, amp, prob, algo, param, ws,
                          0 if ws is None else ws.numel(), _stream(U.device))
    return amp, prob


class BatchPlan:
    """Device-resident descriptors, outputs and workspace of one batched call.

    circuits: list of (U complex128 [m, m] CUDA, input_occ (host), outputs uint8 [n_out, m] CUDA).
    Keeps references to every tensor the descriptors point at.
    """

    def __init__(self, circuits, want_prob: bool = True, algo: int = PCV_ALGO_AUTO):
        if not circuits:
            raise ValueError("empty batch")
        dev = circuits[0][0].device
        arr = (abi.pcv_batch_desc * len(circuits))()
        self.keep, self.amps, self.probs = [], [], []
        total = 0
        for i, (U, t, outs) in enumerate(circuits):
            m = _check_U(U)
            if m > 128:
                raise ValueError("batched circuits support m <= 128")
            t = _host_occ(t, m)
            n = int(t.sum())
            if not 1 <= n <= PCV_MAX_PHOTONS:
                raise ValueError(f"circuit {i}: n={n} outside [1, {PCV_MAX_PHOTONS}]")
            if not (outs.is_cuda and outs.dtype == torch.uint8 and outs.dim() == 2 and outs.shape[1] == m):
                raise TypeError(f"circuit {i}: outputs must be uint8 CUDA [n_out, {m}]")
            U, outs = U.contiguous(), outs.contiguous()
            amp = torch.empty(outs.shape[0], dtype=torch.complex128, device=dev)
            prob = torch.empty(outs.shape[0], dtype=torch.float64, device=dev) if want_prob else None
            d = arr[i]
            d.U, d.outputs, d.amp = U.data_ptr(), outs.data_ptr(), amp.data_ptr()
            d.prob = prob.data_ptr() if prob is not None else None
            d.n_out, d.m, d.n = outs.shape[0], m, n
            cols = np.repeat(np.arange(m), t)
            for j, c in enumerate(cols):
                d.cols[j] = int(c)
            self.keep += [U, outs]
            self.amps.append(amp)
            self.probs.append(prob)
            total += outs.shape[0]
        raw = np.frombuffer(bytes(arr), dtype=np.uint8)
        self.descs = torch.from_numpy(raw.copy()).to(dev)
        self.n_circ, self.total = len(circuits), total
        self.ws = workspace(abi.pcv_amplitudes_batched_workspace(self.n_circ, total), dev)
        self.device = dev
        self.algo = algo

    def run(self):
        abi.pcv_amplitudes_batched_ex(self.descs, self.n_circ, self.total, self.algo, self.ws,
                                      0 if self.ws is None else self.ws.numel(), _stream(self.device))
        return self.amps, self.probs

    def capture(self):
        """Record the batched launch (queue building, routing, persistent
        kernels) once as a CUDA graph; replay() then relaunches all of it with
        one call.  The graph keeps the addresses of the unitaries, outputs,
        results and workspace, so new inputs are written into those tensors
        in place before a replay.  The queue counters are reset by the
        launch's own kernels, so replays need no host work."""
        self.run()                                    # loads kernels, sets attributes
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        if getattr(self, "graph", None) is None:
            self.capture()
        self.graph.replay()
        return self.amps, self.probs


def amplitudes_batched(circuits, want_prob: bool = True, algo: int = PCV_ALGO_AUTO):
    """Amplitudes of many circuits of uneven size: per output the shared-row-sum
    tile kernel or Glynn's sum with multiplicities (algo AUTO), or all outputs
    through one of them (PCV_ALGO_TILE, PCV_ALGO_MULT).
    Returns (list of amp tensors, list of prob tensors or None)."""
    return BatchPlan(circuits, want_prob, algo).run()


def distribution_workspace_bytes(m: int, n: int, algo: int = PCV_ALGO_AUTO, param: int = 0) -> int:
    if algo == PCV_ALGO_AUTO:
        return abi.pcv_distribution_workspace(m, n)
    if algo == PCV_ALGO_FACTOR:
        return abi.pcv_distribution_batched_workspace(1, m, n)
    if algo == PCV_ALGO_SLOS:
        return abi.pcv_distribution_slos_workspace(1, m, n)
    if algo == PCV_ALGO_FACTOR_TC:
        return abi.pcv_distribution_tc_workspace(m, n)
    nb = ((m + 1) * (n + 1) * 8 + 255) // 256 * 256
    if algo == PCV_ALGO_BLOCK and param > 1:
        nb += num_outputs(m, n) * param * 16 + 256
    return nb


def distribution(U: torch.Tensor, input_occ, *, want_amp: bool = True, algo: int = PCV_ALGO_AUTO,
                 param: int = 0, ws: torch.Tensor | None = None, out=None):
    """Every output of S_{m,n} in canonical order.

    Returns (prob float64 [N], amp complex128 [N] or None), N = C(m+n-1, n).
    `out` = (prob, amp) preallocated tensors may be passed to avoid allocation.
    """
    m = _check_U(U)
    t = _host_occ(input_occ, m)
    n = int(t.sum())
    N = num_outputs(m, n)
    U = U.contiguous()
    if out is not None:
        prob, amp = out
    else:
        prob = torch.empty(N, dtype=torch.float64, device=U.device)
        amp = torch.empty(N, dtype=torch.complex128, device=U.device) if want_amp else None
    if ws is None:
        ws = workspace(distribution_workspace_bytes(m, n, algo, param), U.device)
    nbytes = 0 if ws is None else ws.numel()
    if algo == PCV_ALGO_AUTO:
        abi.pcv_distribution(U, m, t, prob, amp, ws, nbytes, _stream(U.device))
    else:
        abi.pcv_distribution_ex(U, m, t, prob, amp, algo, param, ws, nbytes, _stream(U.device))
    return prob, amp


def distribution_range(U: torch.Tensor, input_occ, begin: int, end: int, *, want_amp: bool = True,
                       ws: torch.Tensor | None = None, out=None):
    """The outputs of `distribution` with canonical index in [begin, end):
    (prob float64 [end - begin], amp complex128 [end - begin] or None), output
    i at position i - begin.  The ranges of a partition of [0, N) together
    give exactly `distribution`'s arrays."""
    m = _check_U(U)
    t = _host_occ(input_occ, m)
    n = int(t.sum())
    U = U.contiguous()
    if out is not None:
        prob, amp = out
    else:
        prob = torch.empty(end - begin, dtype=torch.float64, device=U.device)
        amp = torch.empty(end - begin, dtype=torch.complex128, device=U.device) if want_amp else None
    if ws is None:
        ws = workspace(abi.pcv_distribution_workspace(m, n), U.device)
    abi.pcv_distribution_range(U, m, t, begin, end, prob, amp, ws, 0 if ws is None else ws.numel(),
                               _stream(U.device))
    return prob, amp


def distribution_status(ws: torch.Tensor) -> int:
    """Wait for the current stream, then PCV_OK, or PcvError(PCV_ETIMEOUT) if a
    bounded wait of the tensor-core kernels gave up in the last distribution
    call that used workspace `ws`."""
    return abi.pcv_distribution_status(ws, _stream(ws.device))


def distribution_classes(U: torch.Tensor, classes, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Distribution over S_{m,n} of photon classes: `classes` is a list of
    input occupations (host, m photon counts each); photons of one class are
    identical, photons of different classes perfectly distinguishable.
    Returns prob float64 [C(m+n-1, n)] in canonical order."""
    m = _check_U(U)
    occ = np.ascontiguousarray(np.stack([_host_occ(t, m) for t in classes]) if len(classes) else
                               np.zeros((0, m), np.uint8), dtype=np.uint8)
    G = occ.shape[0]
    n = int(occ.sum())
    U = U.contiguous()
    prob = torch.empty(num_outputs(m, n), dtype=torch.float64, device=U.device)
    if ws is None:
        ws = workspace(abi.pcv_distribution_classes_workspace(m, G, occ), U.device)
    abi.pcv_distribution_classes(U, m, G, occ, prob, ws, 0 if ws is None else ws.numel(), _stream(U.device))
    return prob


def source_distribution(U: torch.Tensor, input_occ, transmittance: float = 1.0, indistinguishability: float = 1.0,
                        ws: torch.Tensor | None = None):
    """Output distribution of an imperfect source (see pcv_distribution_source):
    returns (prob float64 over S_{m,0}, ..., S_{m,n} concatenated, offsets
    list with block k at prob[offsets[k]:offsets[k+1]])."""
    m = _check_U(U)
    t = _host_occ(input_occ, m)
    n = int(t.sum())
    U = U.contiguous()
    T = abi.pcv_distribution_source_size(m, n)
    prob = torch.empty(T, dtype=torch.float64, device=U.device)
    if ws is None:
        ws = workspace(abi.pcv_distribution_source_workspace(m, t), U.device)
    abi.pcv_distribution_source(U, m, t, transmittance, indistinguishability, prob, ws,
                                0 if ws is None else ws.numel(), _stream(U.device))
    offsets = [0]
    for k in range(n + 1):
        offsets.append(offsets[-1] + num_outputs(m, k))
    return prob, offsets


def distribution_batched(U: torch.Tensor, input_occ, *, want_amp: bool = True, ws: torch.Tensor | None = None,
                         out=None):
    """Full distributions of a batch of unitaries U [B, m, m] with one input.
    Returns (prob [B, N], amp [B, N] or None)."""
    if not (U.is_cuda and U.dtype == torch.complex128 and U.dim() == 3 and U.shape[1] == U.shape[2]):
        raise TypeError("U must be a complex128 CUDA tensor [B, m, m]")
    B, m = U.shape[0], U.shape[1]
    t = _host_occ(input_occ, m)
    n = int(t.sum())
    N = num_outputs(m, n)
    U = U.contiguous()
    if out is not None:
        prob, amp = out
    else:
        prob = torch.empty(B, N, dtype=torch.float64, device=U.device)
        amp = torch.empty(B, N, dtype=torch.complex128, device=U.device) if want_amp else None
    if ws is None:
        ws = workspace(abi.pcv_distribution_batched_workspace(B, m, n), U.device)
    abi.pcv_distribution_batched(U, B, m, t, prob, amp, ws, 0 if ws is None else ws.numel(), _stream(U.device))
    return prob, amp


def sample(U: torch.Tensor, input_occ, perm: torch.Tensor, uniforms: torch.Tensor) -> torch.Tensor:
    """Exact boson samples (uint8 occupations [count, m]); perm uint8 [count, n]
    and uniforms float64 [count, n] on the device carry the randomness."""
    m = _check_U(U)
    t = _host_occ(input_occ, m)
    count = perm.shape[0]
    out = torch.empty(count, m, dtype=torch.uint8, device=U.device)
    abi.pcv_sample(U.contiguous(), m, t, perm.contiguous(), uniforms.contiguous(), count, out, _stream(U.device))
    return out


def fp64_probe(blocks: int, threads: int, iters: int, device="cuda") -> torch.Tensor:
    out = torch.empty(blocks * threads, dtype=torch.float64, device=device)
    abi.pcv_fp64_probe(out, blocks, threads, iters, _stream(torch.device(device)))
    return out
