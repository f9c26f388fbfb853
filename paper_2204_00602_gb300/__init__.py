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
                   PCV_MAX_MODES, PCV_MAX_PHOTONS, PcvError)

__all__ = ["amplitudes", "distribution", "num_outputs", "unrank", "rank", "fp64_probe", "PcvError",
           "PCV_ALGO_AUTO", "PCV_ALGO_GROUP", "PCV_ALGO_BLOCK", "PCV_ALGO_FACTOR", "abi"]


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
        need = abi.pcv_amplitudes_workspace(m, n, n_out) if algo == PCV_ALGO_AUTO else \
            (n_out * param * 16 + 256 if algo == PCV_ALGO_BLOCK and param > 1 else 0)
        ws = workspace(need, U.device)
    abi.pcv_amplitudes_ex(U, m, t, outputs, n_out, amp, prob, algo, param, ws,
                          0 if ws is None else ws.numel(), _stream(U.device))
    return amp, prob


def distribution_workspace_bytes(m: int, n: int, algo: int = PCV_ALGO_AUTO, param: int = 0) -> int:
    if algo in (PCV_ALGO_AUTO, PCV_ALGO_FACTOR):
        return abi.pcv_distribution_workspace(m, n)
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
    abi.pcv_distribution_ex(U, m, t, prob, amp, algo, param, ws, 0 if ws is None else ws.numel(),
                            _stream(U.device))
    return prob, amp


def fp64_probe(blocks: int, threads: int, iters: int, device="cuda") -> torch.Tensor:
    out = torch.empty(blocks * threads, dtype=torch.float64, device=device)
    abi.pcv_fp64_probe(out, blocks, threads, iters, _stream(torch.device(device)))
    return out
