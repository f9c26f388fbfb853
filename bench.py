"""Throughput of the full output distribution, m=20 modes, n=10 photons.

One step = every amplitude and probability of the 20,030,010 outputs of a
Haar-random 20x20 unitary with photons in modes 0..9 (Eq. eqperm, Sec. 4.2),
computed by the CUDA library through its C ABI entry point pcv_distribution.
At this size that call takes the factorised Glynn sum with its complex
products on the tensor cores as exact integer digit products (--algo auto,
the default, = factor_tc here); --algo factor runs the same sum with FP64
products, which the JSON line also reports as context.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--algo auto|factor_tc|factor|group|slos]

Prints one JSON line (rank 0).  `value` is amplitudes/s over all ranks with
inputs resident in HBM; `e2e` is the same metric through the public API with
host buffers (pinned H2D of U, D2H of probabilities and amplitudes inside the
timed region).  Multi-GPU (torchrun) runs independent unitaries per rank
(weak scaling), or with --shard one distribution split into contiguous output
ranges, one per rank (pcv_distribution_range, strong scaling); neither has a
collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N_PH = 20, 10


def workload_text(m, n, count):
    return (f"full distribution m={m} n={n}, photons in modes 0..{n - 1}, Haar-random {m}x{m} complex128 "
            f"unitary (QR of seeded complex Gaussian, seed 2204006022 + 1000*rank), all {count:,} "
            "outputs, complex FP64 amplitudes and probabilities")
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2, written between timed steps

# Per-launch DRAM traffic of the dominant kernels comes from ncu records
# committed beside the profile summaries; each names the SHA-256 of the CUDA
# source it was taken from, and a record whose source has changed since is
# not used (traffic = null).
TRAFFIC_RECORDS = {"factor_tc": ("tc_product_kernel_traffic.txt", "glynn_tc.cu"),
                   "factor": ("gemm_kernel_traffic.txt", "glynn_dist.cu")}


def recorded_traffic(algo: str, m: int, n: int):
    """(bytes per launch, note) from the kernel's traffic record, or (None, why)."""
    import hashlib
    if algo not in TRAFFIC_RECORDS:
        return None, "no traffic record for this kernel"
    rec, src = TRAFFIC_RECORDS[algo]
    try:
        with open(os.path.join(ROOT, "profiles", rec)) as f:
            kv = dict(line.split(":", 1) for line in f if ":" in line and not line.startswith("#"))
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        with open(os.path.join(ROOT, "paper_2204_00602_gb300", "csrc", src), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None, "no traffic record for this kernel"
    if kv.get("source_sha256") != sha:
        return None, f"the kernel changed since its ncu traffic record ({rec})"
    if (int(kv.get("m", -1)), int(kv.get("n", -1))) != (m, n):
        return None, f"the traffic record is for another workload ({rec})"
    return float(kv["read_bytes"]) + float(kv["write_bytes"]), f"ncu record {rec} of the current source"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=250,
                    help="timed steps (250 x ~2.4 ms: about a second with the copies, long enough for several clock samples)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="auto", choices=["auto", "factor", "factor_tc", "group", "slos"],
                    help="auto: pcv_distribution's own choice (default); factor / factor_tc: factorised Glynn "
                         "with FP64 / tensor-core products; group: plain Glynn; slos: state expansion")
    ap.add_argument("--shard", action="store_true",
                    help="split ONE distribution into contiguous canonical output ranges, one per rank "
                         "(pcv_distribution_range; strong scaling) instead of one distribution per rank")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--m", type=int, default=20, help="modes (default: the m=20 n=10 workload)")
    ap.add_argument("--n", type=int, default=10, help="photons")
    args = ap.parse_args()
    global M, N_PH
    M, N_PH = args.m, args.n
    return args


def measured_bf16_peak() -> float:
    """Dense BF16 TFLOP/s measured on the GB300s (burst), else the
    recipe's fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def rank_unitary_seed(rank: int) -> int:
    """Each rank simulates its own Haar unitary (independent problems, weak scaling)."""
    import pcv_inputs as pin
    return pin.BASE_SEED + 2 + 1000 * rank


def max_over_ranks(value: float, world: int, device) -> float:
    """Slowest rank's time: the only collective of the multi-GPU bench."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as td
    t = torch.tensor([value], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.cpu().numpy()[0])


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, seconds: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank_step * steps * world / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


# ------------------------------------------------------------ CPU oracle

def oracle_sample(budget_s: float, rank_seed: int = 0):
    """Time the CPU oracle (Ryser, all host threads) on the first outputs of the
    canonical order until `budget_s` seconds of work are done."""
    import numpy as np

    import oracle
    import pcv_inputs as pin
    U = pin.haar_unitary(M, pin.BASE_SEED + 2 + rank_seed)
    t = pin.single_photon_input(M, N_PH)
    chunk = 20_000
    outs = oracle.enumerate_outputs_prefix(M, N_PH, 2_000_000)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and done + chunk <= len(outs):
        oracle.amplitudes(U, t, outs[done:done + chunk])
        done += chunk
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "amplitudes/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {done} outputs in canonical order of the m=20 n=10 workload, "
                      f"{dt:.1f} s of Ryser FP64 on the host"}, done, dt


# --------------------------------------------------------------- ours

def run_ours(args):
    import numpy as np
    import torch

    import paper_2204_00602_gb300 as pcv
    import pcv_inputs as pin
    from paper_2204_00602_gb300 import abi

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    U_h = pin.haar_unitary(M, rank_unitary_seed(0 if args.shard else rank))
    t = pin.single_photon_input(M, N_PH)
    Ntot = pcv.num_outputs(M, N_PH)
    algo = {"auto": pcv.PCV_ALGO_AUTO, "factor": pcv.PCV_ALGO_FACTOR, "factor_tc": pcv.PCV_ALGO_FACTOR_TC,
            "group": pcv.PCV_ALGO_GROUP, "slos": pcv.PCV_ALGO_SLOS}[args.algo]
    param = 32 if args.algo == "group" else 0
    U = torch.from_numpy(U_h).to(dev)
    # --shard: this rank's canonical range [lo, hi) of the one distribution
    lo, hi = (Ntot * rank // world, Ntot * (rank + 1) // world) if args.shard else (0, Ntot)
    if args.shard and args.algo not in ("auto", "factor", "factor_tc"):
        raise SystemExit("--shard runs the factorised distribution (algo auto, factor or factor_tc)")
    prob = torch.empty(hi - lo, dtype=torch.float64, device=dev)
    amp = torch.empty(hi - lo, dtype=torch.complex128, device=dev)
    ws_bytes = pcv.distribution_workspace_bytes(M, N_PH, algo, param)
    ws = pcv.workspace(ws_bytes, dev)
    # the path pcv_distribution takes with this workspace (the roofline's kernel)
    kind = args.algo
    if args.algo == "auto":
        kind = "factor_tc" if abi.pcv_distribution_auto_algo(M, N_PH, ws_bytes) == pcv.PCV_ALGO_FACTOR_TC else "factor"
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def dist_call(Uc, out):
        if args.shard:
            pcv.distribution_range(Uc, t, lo, hi, ws=ws, out=out)
        else:
            pcv.distribution(Uc, t, algo=algo, param=param, ws=ws, out=out)

    def step():
        dist_call(U, (prob, amp))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # FP64 probe: measured DFMA throughput of this GPU (context for the roofline)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    iters = 1 << 16
    pr_blocks, pr_threads = sms * 8, 256
    pcv.fp64_probe(pr_blocks, pr_threads, iters, device=dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pcv.fp64_probe(pr_blocks, pr_threads, iters, device=dev)
    e1.record(stream)
    torch.cuda.synchronize()
    probe_tflops = pr_blocks * pr_threads * iters * 16 / (e0.elapsed_time(e1) * 1e-3) / 1e12

    # ---------------- timed region (inputs resident in HBM)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    abi.pcv_profile_read()
    abi.pcv_profile_enable(True)
    launches0 = abi.pcv_launch_count()
    clocks = ClockSampler(gpu_id_for(torch, dev))
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                      # L2 flush between steps (untimed)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    launches = abi.pcv_launch_count() - launches0
    abi.pcv_profile_enable(False)
    stages = abi.pcv_profile_read()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    if args.algo in ("auto", "factor", "factor_tc"):
        abi.pcv_distribution_status(ws, stream.cuda_stream)      # raises if a bounded wait gave up
    t_dev = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    if world > 1:
        torch.distributed.barrier()
    # weak: every rank a whole distribution; strong (--shard): one between them
    value = Ntot * args.steps / t_dev if args.shard else whole_job_rate(Ntot, args.steps, world, t_dev)

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # every step: H2D of U from pinned memory, the distribution, D2H of
        # its amplitudes and probabilities to pinned memory.  The results are
        # double-buffered so that the D2H of step i runs on a copy stream
        # while step i+1 computes.
        U_pin = torch.from_numpy(U_h).pin_memory()
        dev_out = [(prob, amp), (torch.empty_like(prob), torch.empty_like(amp))]
        host_out = [(torch.empty(Ntot, dtype=torch.float64).pin_memory(),
                     torch.empty(Ntot, dtype=torch.complex128).pin_memory()) for _ in range(2)]
        U_d = torch.empty_like(U)
        copy_stream = torch.cuda.Stream(device=dev)
        computed = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        for ev in copied:
            ev.record(copy_stream)

        def e2e_step(i):
            b = i % 2
            U_d.copy_(U_pin, non_blocking=True)
            stream.wait_event(copied[b])                  # buffer b's previous D2H has finished
            dist_call(U_d, dev_out[b])
            computed[b].record(stream)
            copy_stream.wait_event(computed[b])
            with torch.cuda.stream(copy_stream):
                host_out[b][0].copy_(dev_out[b][0], non_blocking=True)
                host_out[b][1].copy_(dev_out[b][1], non_blocking=True)
            copied[b].record(copy_stream)

        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for i in range(args.steps):
            e2e_step(i)
        stream.wait_stream(copy_stream)                   # the last D2H is inside the timed region
        ee.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(es.elapsed_time(ee) / 1e3, world, dev)
        e2e = {"value": (Ntot * args.steps / te) if args.shard else whole_job_rate(Ntot, args.steps, world, te),
               "unit": "amplitudes/s",
               "h2d_bytes_per_step": U_pin.numel() * 16,
               "d2h_bytes_per_step": host_out[0][0].numel() * 8 + host_out[0][1].numel() * 16,
               "pipeline": "results double-buffered; the D2H of step i overlaps the compute of step i+1"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel (FP64 ALU bound)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_tflops = sms * 4 * sm_max * 1e6 / 1e12        # 2 DFMA/clk/SM x 2 flop
    if kind == "factor":
        ms, calls = stages["dist_products"]
        flops_per_call = (hi - lo) * (2 ** (N_PH - 1)) * 6     # 3 DFMA per output and sign vector
        kname = "gemm_kernel (factorised Glynn products, 3 DFMA per output and sign vector)"
        launches_per_call = 1
    elif kind == "factor_tc":
        # BF16 tensor-core work: 3 real products x 36 digit pairs x 2 flops per
        # output and sign vector (useful outputs only)
        ms, calls = stages["dist_products"]
        # every output goes through the tensor cores when n >= 2 and m >= 2
        # (tile padding and the pairs of merged seam groups that are not
        # outputs are computed but not counted); else the outputs with every
        # photon on one side run in FP64
        h = max(1, M // 2)
        n_tc = (hi - lo) if (N_PH >= 2 and M - h >= 1) else \
            Ntot - math.comb(M - h + N_PH - 1, N_PH) - math.comb(h + N_PH - 1, N_PH)
        flops_per_call = n_tc * (2 ** (N_PH - 1)) * 3 * 36 * 2
        kname = "tc_product_kernel (exact-digit BF16 tcgen05 products, 36 digit pairs x 3 real products)"
        launches_per_call = 1
    elif kind == "group":
        ms, calls = stages["glynn_plain"]
        flops_per_call = Ntot * (2 ** (N_PH - 1)) * (8 * N_PH - 4)
        kname = "glynn_group_kernel<10,32> (plain Glynn)"
        launches_per_call = 1
    else:
        # state expansion: one complex multiply-add (8 flops) per state and distinct occupied mode;
        # counted exactly over every level
        ms, calls = stages["glynn_plain"]
        # multisets of size k over M modes with d distinct modes: C(M, d) C(k-1, d-1)
        flops_per_call = sum(8 * d * math.comb(M, d) * math.comb(k - 1, d - 1)
                             for k in range(1, N_PH + 1) for d in range(1, min(k, M) + 1))
        kname = "slos_level_kernel (state expansion)"
        launches_per_call = N_PH
    achieved = flops_per_call * calls / (ms * 1e-3) / 1e12 if ms > 0 and flops_per_call else None
    peak_src = f"derived: {sms} SMs x 2 DFMA/clk x 2 flop x {sm_max:.0f} MHz (FP64 ALU)"
    bound = "alu"
    if kind == "factor_tc":
        peak_tflops, bound = measured_bf16_peak(), "tensor"
        peak_src = "MEASURED_PEAKS.json bf16_tflops (burst cuBLAS bf16 GEMM, measured)"
    traffic, traffic_note = recorded_traffic(kind, M, N_PH)
    roof = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops if achieved else None,
            "peak_source": peak_src,
            "fp64_probe_tflops": probe_tflops,
            "traffic": traffic, "traffic_source": traffic_note,
            "launches_per_step": launches_per_call,
            "stage_ms_per_step": {k: (v[0] / v[1] if v[1] else None) for k, v in stages.items()}}

    # context: the FP64 factorised path (its product kernel against the FP64 peak)
    fp64_ctx = None
    if kind == "factor_tc" and not args.no_e2e:
        ws_f = pcv.workspace(pcv.distribution_workspace_bytes(M, N_PH, pcv.PCV_ALGO_FACTOR), dev)
        for _ in range(2):
            pcv.distribution(U, t, algo=pcv.PCV_ALGO_FACTOR, ws=ws_f, out=(prob, amp))
        torch.cuda.synchronize()
        abi.pcv_profile_read()
        abi.pcv_profile_enable(True)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fsteps = min(args.steps, 20)                      # ~55 ms each
        f0.record(stream)
        for _ in range(fsteps):
            pcv.distribution(U, t, algo=pcv.PCV_ALGO_FACTOR, ws=ws_f, out=(prob, amp))
        f1.record(stream)
        torch.cuda.synchronize()
        abi.pcv_profile_enable(False)
        st = abi.pcv_profile_read()
        ms_f = f0.elapsed_time(f1) / fsteps
        gms, gcalls = st["dist_products"]
        gflops = Ntot * (2 ** (N_PH - 1)) * 6
        ach = gflops * gcalls / (gms * 1e-3) / 1e12 if gms > 0 else None
        fp64_peak = sms * 4 * sm_max * 1e6 / 1e12
        fp64_ctx = {"algo": "factorised Glynn, FP64 products (gemm_kernel, 3 DFMA per output and sign vector)",
                    "ms_per_step": ms_f, "value": Ntot / (ms_f * 1e-3), "unit": "amplitudes/s",
                    "product_kernel_tflops": ach, "fp64_peak_tflops": fp64_peak,
                    "frac_of_fp64_peak": ach / fp64_peak if ach else None}
        del ws_f

    # context: the same workload by photon-by-photon state expansion (not the Glynn path)
    alt = None
    if kind in ("factor", "factor_tc") and not args.no_e2e:
        ws_s = pcv.workspace(pcv.distribution_workspace_bytes(M, N_PH, pcv.PCV_ALGO_SLOS), dev)
        for _ in range(2):
            pcv.distribution(U, t, algo=pcv.PCV_ALGO_SLOS, ws=ws_s, out=(prob, amp))
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            pcv.distribution(U, t, algo=pcv.PCV_ALGO_SLOS, ws=ws_s, out=(prob, amp))
        a1.record(stream)
        torch.cuda.synchronize()
        ms_s = a0.elapsed_time(a1) / args.steps
        alt = {"algo": "state expansion (pcv_distribution_slos)", "ms_per_step": ms_s,
               "value": Ntot / (ms_s * 1e-3), "unit": "amplitudes/s", "note": "context only; not the Glynn path"}
        del ws_s

    cpu = None
    if not args.no_cpu and (world == 1 or rank == 0):
        cpu, _, _ = oracle_sample(args.cpu_seconds)

    line = {
        "metric": f"amplitudes/s (m={M} n={N_PH} full distribution, complex FP64)",
        "value": value, "unit": "amplitudes/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "dtype_note": None if kind != "factor_tc" else
        "FP64 tables, scaling and results; the complex products run as exact integer digit products "
        "on the bf16 tensor cores (no rounding; agreement with the FP64 path to 1e-11)",
        "data": "synthetic",
        "config": {"workload": workload_text(M, N_PH, Ntot), "m": M, "n": N_PH, "outputs": Ntot, "algo": kind,
                   "entry_point": "pcv_distribution" if args.algo == "auto" else "pcv_distribution_ex",
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "parallelism": f"output-range shards x{world}" if args.shard else f"replicas{world}"},
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "state_expansion": alt,
        "fp64_factor_path": fp64_ctx,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import pcv_inputs as pin
    U = pin.haar_unitary(M, pin.BASE_SEED + 2)
    t = pin.single_photon_input(M, N_PH)
    per_step = 20_000
    outs = oracle.enumerate_outputs_prefix(M, N_PH, per_step)
    for _ in range(args.warmup):
        oracle.amplitudes(U, t, outs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.amplitudes(U, t, outs)
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": f"amplitudes/s (m={M} n={N_PH} full distribution, complex FP64)",
        "value": v, "unit": "amplitudes/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_text(M, N_PH, oracle.num_outputs(M, N_PH)), "m": M, "n": N_PH,
                   "outputs": oracle.num_outputs(M, N_PH),
                   "sample_per_step": per_step},
        "cpu_baseline": {"value": v, "unit": "amplitudes/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: the first {per_step} outputs in canonical order, CPU Ryser FP64"},
        "e2e": {"value": v, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
