"""Splitting the amplitude path over ranks (one process per GPU).

Every amplitude is independent, so ranks divide the work with no exchange on
the data path:

* circuits of an uneven batch: greedy longest-processing-time assignment by
  each circuit's FP64 instruction count under the batched launch's routing
  model (``circuit_cost``, ``lpt_assign``);
* outputs of one distribution or one list of explicit outputs, and phase sets
  of a mesh batch: contiguous index ranges [r N / P, (r + 1) N / P)
  (``index_range``); ``sharded_distribution`` computes a rank's range of one
  distribution with pcv_distribution_range, and ``gather_slices`` reassembles
  the ranges on every rank where the whole array is wanted (an all-gather,
  the one exchange of the split).

A reduction is needed only where a quantity is a sum over the split:

* sum p, TVD = 1/2 sum |p - q| and KL = sum q log(q / p) over an output split
  (each a sum over outputs, so the ranks' partial values add up);
* the gradient of a loss summed over a phase-set split (dL/dphi of each set
  stays on its rank; dL/dU of a shared U is summed).

``reduce_sum`` does those reductions with torch.distributed: NCCL between GPUs,
gloo in the CPU tests.  With one rank (or no process group) it returns its
input unchanged.
"""
from __future__ import annotations

import heapq

import numpy as np
import torch


def index_range(N: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank `rank` when N items are split into `world` contiguous ranges."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    return N * rank // world, N * (rank + 1) // world


def _tile_splits(n: int) -> int:
    return 1 if n <= 10 else 2 if n <= 13 else 4 if n <= 16 else 8


def output_cost(m: int, n: int, input_occ, outputs: np.ndarray) -> np.ndarray:
    """FP64 pipe instructions per output under the batched routing model:
    min(tile kernel, Glynn's sum with multiplicities on either side)."""
    t = np.asarray(input_occ, dtype=np.int64)
    tin = t[t > 0]
    d_in = len(tin)
    s = np.asarray(outputs, dtype=np.int64).reshape(-1, m)
    tile = 2.0 ** (n - 1) * (4 * n - 2 + 2 * m / (256 // _tile_splits(n)))

    def terms(mu):                       # rows: multiplicities (zeros ignored)
        prod = np.prod(mu + 1, axis=-1).astype(np.float64)
        odd = np.any(mu % 2 == 1, axis=-1)
        big = mu.max(axis=-1)
        return np.where(odd, prod / 2, prod / (big + 1) * (big // 2 + 1))

    t_out = terms(s)
    t_in = float(terms(tin[None, :])[0]) if d_in else 1.0
    d_out = (s > 0).sum(axis=1)
    cost_out = t_out * (2 * d_in + 4 * n - 1)
    cost_in = t_in * (2 * d_out + 4 * n - 1)
    return np.minimum(tile, np.minimum(cost_out, cost_in))


def circuit_cost(m: int, n: int, input_occ, outputs: np.ndarray) -> float:
    return float(output_cost(m, n, input_occ, outputs).sum())


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Greedy longest-processing-time: items by decreasing cost (ties by
    index), each to the rank with the least load so far (ties by rank).
    Returns the item indices of each rank, in increasing order."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def world_and_rank() -> tuple[int, int]:
    import torch.distributed as td
    if td.is_available() and td.is_initialized():
        return td.get_world_size(), td.get_rank()
    return 1, 0


def reduce_sum(x: torch.Tensor) -> torch.Tensor:
    """Sum of x over the ranks (in place on x, which is also returned)."""
    world, _ = world_and_rank()
    if world > 1:
        import torch.distributed as td
        td.all_reduce(x, op=td.ReduceOp.SUM)
    return x


def local_stats(p_slice: torch.Tensor, q_slice: torch.Tensor) -> torch.Tensor:
    """[3] partial (sum p, TVD, KL) of this rank's output slice, on the GPU
    (pcv_dist_stats); ``reduce_sum`` of it gives the whole distribution's."""
    from .autograd import dist_stats
    return dist_stats(p_slice.reshape(1, -1), q_slice)[0]


def sharded_stats(p_slice: torch.Tensor, q_slice: torch.Tensor) -> torch.Tensor:
    return reduce_sum(local_stats(p_slice, q_slice))


def sharded_distribution(U: torch.Tensor, input_occ, *, want_amp: bool = True, ws: torch.Tensor | None = None):
    """This rank's contiguous range of the distribution of U (one GPU per rank):
    (lo, hi, prob [hi - lo], amp [hi - lo] or None), canonical outputs lo..hi-1."""
    from . import distribution_range, num_outputs
    world, rank = world_and_rank()
    m = U.shape[0]
    n = int(np.asarray(input_occ, dtype=np.int64).sum())
    lo, hi = index_range(num_outputs(m, n), rank, world)
    prob, amp = distribution_range(U, input_occ, lo, hi, want_amp=want_amp, ws=ws)
    return lo, hi, prob, amp


def gather_slices(local: torch.Tensor, N: int) -> torch.Tensor:
    """The whole length-N array on every rank, from each rank's slice
    [index_range(N, rank, world)] (all-gather; complex values travel as pairs
    of reals)."""
    world, rank = world_and_rank()
    if world == 1:
        return local
    import torch.distributed as td
    cplx = local.is_complex()
    flat = torch.view_as_real(local).reshape(-1) if cplx else local.reshape(-1)
    per = 2 if cplx else 1
    cap = (N + world - 1) // world * per
    buf = torch.zeros(cap, dtype=flat.dtype, device=flat.device)
    buf[:flat.numel()] = flat
    parts = [torch.empty_like(buf) for _ in range(world)]
    td.all_gather(parts, buf)
    pieces = []
    for r in range(world):
        lo, hi = index_range(N, r, world)
        pieces.append(parts[r][:(hi - lo) * per])
    whole = torch.cat(pieces)
    return torch.view_as_complex(whole.reshape(-1, 2)) if cplx else whole
