"""Secondary throughput workloads (the headline m=20 n=10 distribution is bench.py).

    python -m paper_2204_00602_gb300.workloads batched [--circuits 512] [--outputs 4096] [--route auto|tile|mult]
    python -m paper_2204_00602_gb300.workloads sweep [--nmin 16] [--nmax 30] [--outputs 256]
    python -m paper_2204_00602_gb300.workloads mesh   [--batch 64]
    python -m paper_2204_00602_gb300.workloads sample [--m 60] [--n 14] [--samples 200000]
    python -m paper_2204_00602_gb300.workloads pk [--unitaries 300] [--samples 20000]
    python -m paper_2204_00602_gb300.workloads source [--m 12] [--n 6] [--eta 0.9] [--V 0.9]

batched: uneven circuits (m ~ U{8..64}, n ~ U{4..min(24, m)}, Haar U, photons in
modes 0..n-1, 4096 seeded random outputs each, collision-free for n <= 16,
uniform multisets above) in persistent launches: each output goes to the
shared-row-sum tile kernel or to Glynn's sum with multiplicities, whichever
issues fewer FP64 instructions (--route forces one of them).
sweep: one Haar unitary per n = 16..30 at m = n^2, 256 collision-free outputs,
plain Glynn block kernel (m is too large for the shared-row-sum tiles).
mesh: the differentiable m=12 n=6 mesh, 64 phase sets, forward (all 12,376
outputs) + KL + backward per step.

Each prints one JSON line: amplitudes/s, FP64 work per the kernel's
instruction count, and the fraction of the FP64 peak (152 SMs x 2 DFMA/clk x
2 flop x clock).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

import pcv_inputs as pin

from . import BatchPlan, amplitudes

SEED = pin.BASE_SEED + 3


def _peak_flops():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 2 * 2 * 2070e6


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _tile_splits(n: int) -> int:
    return 1 if n <= 10 else 2 if n <= 13 else 4 if n <= 16 else 8


def routed_fp64_instructions(m: int, n: int, outs: np.ndarray):
    """FP64 pipe instructions under the batched launch's cost model
    (single-photon input): the tile kernel's 2^{n-1} (4n - 2 + 2m/TILE) per
    output, a tile block costing as much as TILE outputs however many are live,
    or, for Glynn's sum with multiplicities, terms x (2q + 4n - 1) on the
    cheaper side.  Returns (tile-only instructions, routed instructions,
    outputs routed to the multiplicity kernel)."""
    tile = 2.0 ** (n - 1) * (4 * n - 2 + 2 * m / (256 // _tile_splits(n)))
    s = outs.astype(np.int64)
    d_out = (s > 0).sum(axis=1)
    prod = np.prod(s + 1, axis=1).astype(np.float64)
    odd = np.any(s % 2 == 1, axis=1)
    big = s.max(axis=1)
    t_out = np.where(odd, prod / 2, prod / (big + 1) * (big // 2 + 1))
    cost_out = t_out * (2 * n + 4 * n - 1)              # product side: the n input photons
    cost_in = 2.0 ** (n - 1) * (2 * d_out + 4 * n - 1)  # sign side: the n input photons
    mult = np.minimum(cost_out, cost_in)
    to_mult = mult < tile
    # a last, partly filled tile goes to the multiplicity kernel when its
    # outputs cost less there than the whole tile block (as the routing kernel does)
    tile_idx = np.flatnonzero(~to_mult)
    tsz = 256 // _tile_splits(n)
    r = len(tile_idx) % tsz
    if r and mult[tile_idx[-r:]].sum() < tile * tsz:
        to_mult[tile_idx[-r:]] = True
    n_tile_blocks = -(-int((~to_mult).sum()) // tsz)
    routed = n_tile_blocks * tsz * tile + float(mult[to_mult].sum())
    return tile * len(s), routed, int(to_mult.sum())


def batched(n_circ: int, n_out: int, reps: int = 1, route: str = "auto"):
    from . import PCV_ALGO_AUTO, PCV_ALGO_MULT, PCV_ALGO_TILE
    algo = {"auto": PCV_ALGO_AUTO, "tile": PCV_ALGO_TILE, "mult": PCV_ALGO_MULT}[route]
    g = np.random.default_rng(SEED)
    circs = []
    tile_instr = 0.0        # FP64 instructions if every output went to the tile kernel
    routed_instr = 0.0      # the same under the routing model
    n_mult = 0
    fl = 0.0                # plain Glynn flops: 6 per complex product, 2 per complex add
    for c in range(n_circ):
        m = int(g.integers(8, 65))
        n = int(g.integers(4, min(24, m) + 1))
        outs_np = pin.random_outputs(m, n, n_out, SEED + 5000 + c)
        U = torch.from_numpy(pin.haar_unitary(m, SEED + 1000 + c)).cuda()
        circs.append((U, pin.single_photon_input(m, n), torch.from_numpy(outs_np).cuda()))
        ti, ri, nm = routed_fp64_instructions(m, n, outs_np)
        tile_instr += ti
        routed_instr += ri if route == "auto" else ti
        n_mult += nm if route == "auto" else 0
        fl += n_out * 2 ** (n - 1) * (6 * (n - 1) + 2)
    # under torchrun: each rank takes its share of the circuits by greedy
    # longest-processing-time on the routed cost; no exchange on the data path
    from .sharding import circuit_cost, lpt_assign, world_and_rank
    world, rank = world_and_rank()
    if world > 1:
        costs = [circuit_cost(c[0].shape[0], int(c[1].sum()), c[1], c[2].cpu().numpy()) for c in circs]
        circs = [circs[i] for i in lpt_assign(costs, world)[rank]]
    # warm-up on one output per circuit (module load, attribute setup)
    BatchPlan([(U, t, o[:1]) for U, t, o in circs], want_prob=True, algo=algo).run()
    plan = BatchPlan(circs, want_prob=True, algo=algo)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    a, b = _events()
    a.record()
    for _ in range(reps):
        plan.run()
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3 / reps
    if world > 1:                      # the job takes as long as its slowest rank
        t = torch.tensor([sec], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        sec = float(t.item())
    amps = n_circ * n_out
    issue = _peak_flops() / 2          # DFMA-pipe instructions per second
    r = {"workload": f"batched {n_circ} uneven circuits x {n_out} outputs (m~U[8,64], n~U[4,24])",
         "route": route, "amplitudes_per_s": amps / sec, "seconds": sec, "amplitudes": amps,
         "fp64_instr_per_s": routed_instr / sec, "frac_of_fp64_issue_rate": routed_instr / sec / issue,
         "tile_only_fp64_instr": tile_instr, "routed_fp64_instr": routed_instr}
    if route == "auto":
        r["outputs_to_multiplicity_kernel"] = n_mult
    if route == "tile":
        r["fp64_tflops"] = fl / sec / 1e12
        r["frac_of_fp64_peak"] = fl / sec / _peak_flops()
    return r


def sweep(nmin: int, nmax: int, n_out: int):
    rows = []
    for n in range(nmin, nmax + 1):
        m = n * n
        U = torch.from_numpy(pin.haar_unitary(m, SEED + 100 + n)).cuda()
        t = pin.single_photon_input(m, n)
        outs = torch.from_numpy(pin.random_outputs(m, n, n_out, SEED + 200 + n)).cuda()
        amplitudes(U, t, outs[:1])
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        amplitudes(U, t, outs)
        b.record()
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        fl = n_out * 2 ** (n - 1) * (8 * n - 4)
        rows.append({"n": n, "m": m, "outputs": n_out, "seconds": sec, "amplitudes_per_s": n_out / sec,
                     "fp64_tflops_algorithmic": fl / sec / 1e12, "frac_of_fp64_peak": fl / sec / _peak_flops()})
        print(json.dumps(rows[-1]), flush=True)
    return {"workload": f"sweep n={nmin}..{nmax} at m=n^2, {n_out} outputs each", "rows": rows}


def mesh(batch: int, steps: int = 20):
    from .autograd import mesh_kl
    m, n = 12, 6
    t = pin.single_photon_input(m, n)
    N = math.comb(m + n - 1, n)
    q = torch.from_numpy(pin.dirichlet_target(N, SEED + 7)).cuda()
    ph = torch.from_numpy(pin.mesh_phases(batch, m * (m - 1), SEED + 8)).cuda().requires_grad_(True)
    for _ in range(2):
        mesh_kl(ph, m, t, q).sum().backward()
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(steps):
        ph.grad = None
        mesh_kl(ph, m, t, q).sum().backward()
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3 / steps
    return {"workload": f"mesh m=12 n=6, {batch} phase sets, all {N} outputs, KL forward+backward",
            "ms_per_step": sec * 1e3, "amplitudes_per_s_forward": batch * N / sec}


def sampling(m: int, n: int, count: int):
    """Exact boson samples per second (the paper's Boson-sampling benchmark shape
    is n=14 photons in m=60 modes)."""
    from . import sample
    U = torch.from_numpy(pin.haar_unitary(m, SEED + 60)).cuda()
    t = pin.single_photon_input(m, n)
    perm, uni = pin.sampler_randomness(count, n, SEED + 61)
    perm_d, uni_d = torch.from_numpy(perm).cuda(), torch.from_numpy(uni).cuda()
    sample(U, t, perm_d[:256], uni_d[:256])
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    sample(U, t, perm_d, uni_d)
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    return {"workload": f"exact boson sampling n={n} m={m} (Haar U, photons in modes 0..{n - 1})",
            "samples": count, "seconds": sec, "samples_per_s": count / sec}


def pk_table(m: int, n: int, n_unitaries: int, samples_per_u: int):
    """The paper's partial-certificate experiment (Sec. 4.2, Table figtablebs) on
    synthetic Haar unitaries: estimate P(K), the probability that all n photons
    leave in the first K modes, from exact samples of each unitary, average over
    the unitaries, and set it beside Eq. eqhaarpk's Haar average."""
    from . import sample
    Ks = (30, 40, 50, 55, 57)
    est = {K: [] for K in Ks}
    t = pin.single_photon_input(m, n)
    t0 = time.perf_counter()
    gpu_s = 0.0
    for u in range(n_unitaries):
        U = torch.from_numpy(pin.haar_unitary(m, SEED + 10_000 + u)).cuda()
        perm, uni = pin.sampler_randomness(samples_per_u, n, SEED + 20_000 + u)
        a, b = _events()
        a.record()
        s = sample(U, t, torch.from_numpy(perm).cuda(), torch.from_numpy(uni).cuda())
        b.record()
        occ = s.cpu().numpy()
        gpu_s += a.elapsed_time(b) / 1e3
        for K in Ks:
            est[K].append(np.mean(occ[:, K:].sum(axis=1) == 0))
    wall = time.perf_counter() - t0
    rows = []
    for K in Ks:
        e = np.array(est[K])
        haar = float(np.prod([(K + i) / (m + i) for i in range(n)]))
        rows.append({"K": K, "estimate_pct": 100 * e.mean(), "std_over_unitaries_pct": 100 * e.std(),
                     "stderr_of_mean_pct": 100 * e.std() / math.sqrt(len(e)), "haar_average_pct": 100 * haar})
    return {"workload": f"P(K) for n={n} m={m}: {n_unitaries} Haar unitaries x {samples_per_u} exact samples",
            "gpu_sampling_s": gpu_s, "wall_s": wall, "rows": rows}


def source(m: int, n: int, eta: float, V: float, reps: int = 3):
    """Output distribution of an imperfect source (transmittance eta,
    indistinguishability V): the mixture over the 2^n pure sets."""
    from . import source_distribution
    U = torch.from_numpy(pin.haar_unitary(m, SEED + 7000 + m)).cuda()
    t = pin.single_photon_input(m, n)
    p, off = source_distribution(U, t, eta, V)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(reps):
        p, off = source_distribution(U, t, eta, V)
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3 / reps
    return {"workload": f"imperfect source m={m} n={n} eta={eta} V={V}: all {off[-1]} photon-number-resolved outputs",
            "seconds": sec, "outputs": off[-1], "pure_sets": 2 ** n, "sum": float(p.sum().item())}


def batched_graph(n_circ: int = 64, n_out: int = 256, reps: int = 200):
    """Small uneven batches, where launch overhead shows: the batched launch
    issued directly each time against the same launch replayed from a CUDA
    graph (BatchPlan.capture)."""
    g = np.random.default_rng(SEED + 7)
    circs = []
    for c in range(n_circ):
        m = int(g.integers(8, 33))
        n = int(g.integers(3, min(9, m) + 1))
        outs = torch.from_numpy(pin.random_outputs(m, n, n_out, SEED + 7000 + c)).cuda()
        U = torch.from_numpy(pin.haar_unitary(m, SEED + 8000 + c)).cuda()
        circs.append((U, pin.single_photon_input(m, n), outs))
    plan = BatchPlan(circs)
    plan.run()
    plan.capture()
    torch.cuda.synchronize()
    res = {}
    for name, call in (("direct", plan.run), ("graph", plan.replay)):
        for _ in range(5):
            call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a, b = _events()
        a.record()
        for _ in range(reps):
            call()
        b.record()
        torch.cuda.synchronize()
        res[name] = {"gpu_ms_per_call": a.elapsed_time(b) / reps,
                     "host_ms_per_call": (time.perf_counter() - t0) * 1e3 / reps}
    return {"workload": f"batched {n_circ} circuits x {n_out} outputs (m~U[8,32], n~U[3,9]), direct vs CUDA graph",
            "amplitudes_per_call": n_circ * n_out, **res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["batched", "batched_graph", "sweep", "mesh", "sample", "pk", "source"])
    ap.add_argument("--eta", type=float, default=0.9)
    ap.add_argument("--V", type=float, default=0.9)
    ap.add_argument("--unitaries", type=int, default=300)
    ap.add_argument("--m", type=int, default=60)
    ap.add_argument("--n", type=int, default=14)
    ap.add_argument("--samples", type=int, default=200_000)
    ap.add_argument("--circuits", type=int, default=512)
    ap.add_argument("--outputs", type=int, default=None)
    ap.add_argument("--nmin", type=int, default=16)
    ap.add_argument("--nmax", type=int, default=30)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--route", choices=["auto", "tile", "mult"], default="auto")
    a = ap.parse_args()
    import os
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:          # torchrun: one rank per GPU
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    if a.which == "batched":
        r = batched(a.circuits, a.outputs or 4096, route=a.route)
    elif a.which == "batched_graph":
        r = batched_graph(min(a.circuits, 64), a.outputs or 256)
    elif a.which == "sweep":
        r = sweep(a.nmin, a.nmax, a.outputs or 256)
    elif a.which == "mesh":
        r = mesh(a.batch)
    elif a.which == "source":
        r = source(a.m, a.n, a.eta, a.V)
    elif a.which == "sample":
        r = sampling(a.m, a.n, a.samples)
    else:
        r = pk_table(a.m, a.n, a.unitaries, a.samples)
    if not torch.distributed.is_initialized() or torch.distributed.get_rank() == 0:
        print(json.dumps(r), flush=True)
    if torch.distributed.is_initialized():
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
