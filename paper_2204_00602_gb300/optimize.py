"""Phase optimisation of Clements meshes with exact gradients, and with the
learned surrogate in the loop (not in the paper; its Sec. 4.4 trains circuit
parameters with an optimiser over exact output distributions).

Problem: B independent m=12 meshes, n=6 photons in modes 0..5, a fixed set of
512 outputs and a target q (Dirichlet(1) over the set).  Each mesh minimises
L(phi) = KL(q || p(phi)) restricted to the set (= -sum q log p + const).

* exact loop: mesh kernel -> tile kernel (512 amplitudes) -> KL gradient
  kernel -> adjoint kernel -> mesh backward kernel -> FP64 Adam kernel.
* surrogate loop: the MLP predicts log p; dL/dlog p = -q is constant, so one
  MLP backward to its inputs and the sin/cos chain give dL/dphi.  Every
  `check_every` steps the exact probabilities of the set are computed and the
  surrogate's TVD on the set, 1/2 sum |p_hat - p|, is checked; above `tvd_tol`
  the loop uses exact gradients for the next `check_every` steps.  Optionally
  the network is refined online on the exact probabilities the loop computes
  anyway (``refine_steps``).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch

from . import _abi as abi
from . import _stream, workspace
from .autograd import dist_stats, mesh_backward, mesh_unitary
from .surrogate import MLP, exact_log_probs, init_weights, output_set


class MeshProblem:
    def __init__(self, B: int = 64, m: int = 12, n: int = 6, n_set: int = 512, seed: int = 2204006025,
                 device="cuda"):
        self.B, self.m, self.n = B, m, n
        self.dev = torch.device(device)
        self.t = np.zeros(m, np.uint8)
        self.t[:n] = 1
        self.outs_host = output_set(m, n, n_set, seed)
        self.outs = torch.from_numpy(self.outs_host).to(self.dev)
        self.n_set = n_set
        self.q = torch.from_numpy(np.random.default_rng(seed + 1).dirichlet(np.ones(n_set))).to(self.dev)
        self.P = m * (m - 1)
        self.amp = torch.empty(B, n_set, dtype=torch.complex128, device=self.dev)
        self.prob = torch.empty(B, n_set, dtype=torch.float64, device=self.dev)
        self.gamp = torch.empty_like(self.amp)
        self.gU = torch.empty(B, m, m, dtype=torch.complex128, device=self.dev)
        self.bws = workspace(abi.pcv_amplitudes_backward_workspace(B, m, n, n_set), self.dev)

    @property
    def stream(self):
        return _stream(self.dev)

    def probs(self, phases):
        U = mesh_unitary(phases, self.m)
        abi.pcv_amplitudes_multi(U, phases.shape[0], self.m, self.t, self.outs, self.n_set, self.amp, self.prob,
                                 self.stream)
        return U, self.prob

    def loss(self, phases):
        _, p = self.probs(phases)
        return dist_stats(p, self.q)[:, 2]

    def loss_and_grad(self, phases):
        U, p = self.probs(phases)
        B = phases.shape[0]
        abi.pcv_kl_grad(p, self.q, self.amp, self.n_set, B, 0, None, 1.0, self.gamp, self.stream)
        abi.pcv_amplitudes_backward_multi(U, B, self.m, self.t, self.outs, self.n_set, self.gamp, self.gU, self.bws,
                                          self.bws.numel(), self.stream)
        return mesh_backward(phases, U, self.gU)


class Adam64:
    def __init__(self, params: torch.Tensor, lr: float):
        self.p, self.lr = params, lr
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.t = 0

    def step(self, g: torch.Tensor):
        self.t += 1
        abi.pcv_adam_f64(self.p, self.m, self.v, g, self.p.numel(), self.lr, 0.9, 0.999, 1e-8, self.t,
                         _stream(self.p.device))


def exact_loop(problem: MeshProblem, phases0: torch.Tensor, steps: int, lr: float = 0.02):
    problem.loss_and_grad(phases0.clone())          # untimed: loads every kernel of the loop once
    phases = phases0.clone()
    opt = Adam64(phases, lr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        opt.step(problem.loss_and_grad(phases))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return phases, wall


class TrajectoryBuffer:
    """Ring buffer of (phases, log p of the set) met along the optimisation, for
    refining the surrogate online (exact probabilities are computed anyway at
    every check and every exact step)."""

    def __init__(self, size: int, n_phases: int, n_set: int, device, seed: int = 1):
        self.ph = torch.zeros(size, n_phases, dtype=torch.float64, device=device)
        self.y = torch.zeros(size, n_set, dtype=torch.float32, device=device)
        self.size, self.filled, self.head = size, 0, 0
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(seed)

    def push(self, phases: torch.Tensor, p: torch.Tensor):
        k = phases.shape[0]
        idx = (torch.arange(k, device=phases.device) + self.head) % self.size
        self.ph[idx] = phases
        self.y[idx] = torch.log(torch.clamp(p, min=1e-300)).to(torch.float32)
        self.head = (self.head + k) % self.size
        self.filled = min(self.size, self.filled + k)

    def refine(self, net: MLP, steps: int, batch: int = 512):
        bs = min(batch, self.filled) // 32 * 32          # the training kernels take multiples of 32 rows
        if bs == 0:
            return
        for _ in range(steps):
            sel = torch.randint(0, self.filled, (bs,), device=self.ph.device, generator=self.gen)
            net.train_step(net.features(self.ph[sel]), self.y[sel])


def surrogate_loop(problem: MeshProblem, net: MLP, phases0: torch.Tensor, steps: int, lr: float = 0.02,
                   check_every: int = 50, tvd_tol: float = 1e-3, refine_steps: int = 0,
                   refine_lr: float = 1e-3, buffer_size: int = 4096):
    """The gated loop.  With refine_steps > 0 the network is also trained
    online: the exact probabilities met at every check and every exact step go
    to a ring buffer, and after each check `refine_steps` Adam steps (learning
    rate refine_lr) are taken on random batches of it."""
    phases = phases0.clone()
    buf = TrajectoryBuffer(buffer_size, problem.P, problem.n_set, phases.device) if refine_steps > 0 else None
    if buf is not None:
        net.lr = refine_lr
    opt = Adam64(phases, lr)
    B = phases.shape[0]
    dy = torch.empty(B, problem.n_set, dtype=torch.bfloat16, device=phases.device)
    negq = (-problem.q).to(torch.float32)
    abi.pcv_f32_to_bf16(negq.repeat(B).contiguous(), B * problem.n_set, dy, problem.stream)
    phat = torch.empty(B, problem.n_set, dtype=torch.float64, device=phases.device)
    warm = phases0.clone()                           # untimed: loads every kernel of the loop once
    problem.loss_and_grad(warm)
    net.predict_phases(warm)
    net.grad_phases(warm, dy)
    abi.pcv_exp_f32_to_f64(net.predict_phases(warm), B * problem.n_set, phat, problem.stream)
    dist_stats(phat, phat)[:, 1].cpu()
    exact_steps, checks, tvds = 0, 0, []
    use_exact_until = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        if s % check_every == 0:
            checks += 1
            _, p = problem.probs(phases)
            y = net.predict_phases(phases)
            abi.pcv_exp_f32_to_f64(y, y.numel(), phat, problem.stream)
            tvd = float(dist_stats(p, phat)[:, 1].cpu().numpy().max())   # host read once per check
            tvds.append(tvd)
            if tvd > tvd_tol:
                use_exact_until = s + check_every
            if buf is not None:
                buf.push(phases, p)
                buf.refine(net, refine_steps)
        if s < use_exact_until:
            g = problem.loss_and_grad(phases)
            exact_steps += 1
            if buf is not None:
                buf.push(phases, problem.prob)
        else:
            net.predict_phases(phases)
            g = net.grad_phases(phases, dy)
        opt.step(g)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return phases, wall, {"exact_steps": exact_steps, "checks": checks, "max_tvd_seen": max(tvds),
                          "min_tvd_seen": min(tvds), "median_tvd_seen": float(np.median(tvds)), "tvd_tol": tvd_tol,
                          "refine_steps": refine_steps}


def anchored_loop(problem: MeshProblem, net: MLP | None, phases0: torch.Tensor, steps: int, lr: float = 0.02,
                  check_every: int = 5, tvd_tol: float = 1e-3, refine_steps: int = 0, buffer_size: int = 4096):
    """The surrogate as a correction to an exact anchor (control variate).

    Every `check_every` steps the loop takes one exact step at phi_a, keeping
    the exact probabilities p_a and gradient g_a, and the network's s_a =
    s(phi_a) and gs_a = dL_s/dphi(phi_a).  In between, the step uses
        g(phi) = g_a + gs(phi) - gs_a,
    so the network only supplies how the gradient changes away from the
    anchor; its prediction of the set is p_hat(phi) = p_a exp(s(phi) - s_a).
    Gate: at each check the previous interval's prediction is compared with
    the exact p (TVD on the set, max over the batch); above `tvd_tol` the
    next interval takes exact steps.  net = None is the same loop without the
    network (g = g_a, p_hat = p_a: the stale anchor), which shows what the
    network adds.  With refine_steps > 0 the network is trained online on the
    exact probabilities of the anchors."""
    phases = phases0.clone()
    B = phases.shape[0]
    opt = Adam64(phases, lr)
    buf = TrajectoryBuffer(buffer_size, problem.P, problem.n_set, phases.device) if (net is not None and
                                                                                     refine_steps > 0) else None
    dy = torch.empty(B, problem.n_set, dtype=torch.bfloat16, device=phases.device)
    abi.pcv_f32_to_bf16((-problem.q).to(torch.float32).repeat(B).contiguous(), B * problem.n_set, dy, problem.stream)
    e = torch.empty(B, problem.n_set, dtype=torch.float64, device=phases.device)
    warm = phases0.clone()                           # untimed: loads every kernel of the loop once
    problem.loss_and_grad(warm)
    if net is not None:
        net.predict_phases(warm)
        net.grad_phases(warm, dy)
    dist_stats(problem.prob, problem.prob)[:, 1].cpu()
    exact_steps, tvds = 0, []
    use_exact = False
    p_a = s_a = gs_a = g_a = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        if s % check_every == 0:
            g_a = problem.loss_and_grad(phases).clone()
            exact_steps += 1
            p = problem.prob
            if net is not None:
                y = net.predict_phases(phases)
                if p_a is not None:
                    abi.pcv_exp_f32_to_f64((y - s_a).contiguous(), y.numel(), e, problem.stream)
                    tvd = float(dist_stats(p, p_a * e)[:, 1].max().cpu())    # host read once per check
                else:
                    tvd = 0.0
                s_a = y.clone()
                gs_a = net.grad_phases(phases, dy).clone()
            else:
                tvd = float(dist_stats(p, p_a)[:, 1].max().cpu()) if p_a is not None else 0.0
            if s > 0:
                tvds.append(tvd)
            use_exact = tvd > tvd_tol
            p_a = p.clone()
            if buf is not None:
                buf.push(phases, p)
                buf.refine(net, refine_steps)
            g = g_a
        elif use_exact:
            g = problem.loss_and_grad(phases)
            exact_steps += 1
        elif net is not None:
            net.predict_phases(phases)
            g = g_a + (net.grad_phases(phases, dy) - gs_a)
        else:
            g = g_a
        opt.step(g)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    tv = np.array(tvds) if tvds else np.zeros(1)
    return phases, wall, {"exact_steps": exact_steps, "checks": len(tvds), "check_every": check_every,
                          "tvd_tol": tvd_tol, "intervals_within_tol": int((tv <= tvd_tol).sum()),
                          "median_tvd_seen": float(np.median(tv)), "max_tvd_seen": float(tv.max()),
                          "refine_steps": refine_steps, "network": net is not None}


def time_to_target(problem: MeshProblem, net: MLP, phases0: torch.Tensor, target: float, warm_steps: int,
                   max_exact_steps: int, lr: float = 0.02, every: int = 25):
    """Wall-clock until the mean exact loss over the batch reaches `target`:
    `warm_steps` surrogate-only steps (0 = none), then exact steps, checking the
    exact loss every `every` steps.  Returns (seconds, exact steps used, reached)."""
    phases = phases0.clone()
    B = phases.shape[0]
    dy = torch.empty(B, problem.n_set, dtype=torch.bfloat16, device=phases.device)
    abi.pcv_f32_to_bf16((-problem.q).to(torch.float32).repeat(B).contiguous(), B * problem.n_set, dy, problem.stream)
    warm = phases0.clone()
    problem.loss_and_grad(warm)
    net.predict_phases(warm)
    net.grad_phases(warm, dy)
    problem.loss(warm).cpu()
    opt = Adam64(phases, lr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(warm_steps):
        net.predict_phases(phases)
        opt.step(net.grad_phases(phases, dy))
    opt = Adam64(phases, lr)                 # fresh moments for the exact phase
    used = 0
    while used < max_exact_steps:
        if used % every == 0 and float(problem.loss(phases).cpu().numpy().mean()) <= target:
            break
        opt.step(problem.loss_and_grad(phases))
        used += 1
    reached = float(problem.loss(phases).cpu().numpy().mean()) <= target
    torch.cuda.synchronize()
    return time.perf_counter() - t0, used, reached


def make_dataset(problem: MeshProblem, n_samples: int, seed: int):
    """Uniform phases and exact log-probabilities of the set (fp32)."""
    g = np.random.default_rng(seed)
    phases = torch.from_numpy(g.uniform(0, 2 * np.pi, size=(n_samples, problem.P))).to(problem.dev)
    targets = exact_log_probs(phases, problem.m, problem.t, problem.outs)
    return phases, targets


def train(net: MLP, phases: torch.Tensor, targets: torch.Tensor, epochs: int, batch: int = 4096):
    n = phases.shape[0] - phases.shape[0] % batch
    losses = []
    for _ in range(epochs):
        for s in range(0, n, batch):
            X = net.features(phases[s:s + batch])
            loss = net.train_step(X, targets[s:s + batch])
        losses.append(float(loss.cpu().numpy()[0]))
        net.check()
    return losses


def validate(net: MLP, problem: MeshProblem, phases: torch.Tensor):
    """Per phase set: TVD on the set between exp(prediction) and the exact p."""
    _, p = problem.probs(phases)
    y = net.predict_phases(phases)
    phat = torch.empty_like(p)
    abi.pcv_exp_f32_to_f64(y, y.numel(), phat, problem.stream)
    return dist_stats(p, phat)[:, 1]


def run(samples: int, epochs: int, steps: int, B: int, seed: int = 2204006025, lr_net: float = 1e-3,
        refine: bool = True):
    problem = MeshProblem(B=B, seed=seed)
    t0 = time.perf_counter()
    ph_train, y_train = make_dataset(problem, samples, seed + 10)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    Ws, bs = init_weights(seed + 20)
    net = MLP(Ws, bs, lr=lr_net)
    t0 = time.perf_counter()
    losses = train(net, ph_train, y_train, epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    val_ph = torch.from_numpy(np.random.default_rng(seed + 30).uniform(0, 2 * np.pi, (B, problem.P))).to(problem.dev)
    val_tvd = validate(net, problem, val_ph).cpu().numpy()
    phases0 = torch.from_numpy(np.random.default_rng(seed + 40).uniform(0, 2 * np.pi, (B, problem.P))).to(problem.dev)
    loss0 = problem.loss(phases0).clone()
    ph_e, wall_e = exact_loop(problem, phases0, steps)
    loss_e = problem.loss(ph_e).clone()
    ph_s, wall_s, info = surrogate_loop(problem, net, phases0, steps)
    loss_s = problem.loss(ph_s).clone()
    refined = None
    if refine:
        # online refinement on the trajectory, from a copy of the trained network
        net_r = MLP([w.cpu().numpy() for w in net.W], [b.cpu().numpy() for b in net.b], lr=lr_net,
                    tensor_core=net.tensor_core)
        ph_r, wall_r, info_r = surrogate_loop(problem, net_r, phases0, steps, check_every=10, refine_steps=20)
        refined = {"wall_s": wall_r, "loss_mean": float(problem.loss(ph_r).cpu().numpy().mean()), **info_r,
                   "check_every": 10}
    # the surrogate as a correction to exact anchors, against the same loop
    # with a stale anchor gradient and no network
    anchored = {}
    net_a = MLP([w.cpu().numpy() for w in net.W], [b.cpu().numpy() for b in net.b], lr=lr_net,
                tensor_core=net.tensor_core)
    ph_a, wall_a, info_a = anchored_loop(problem, net_a, phases0, steps, check_every=5)
    anchored["network"] = {"wall_s": wall_a, "loss_mean": float(problem.loss(ph_a).cpu().numpy().mean()), **info_a}
    ph_n, wall_n, info_n = anchored_loop(problem, None, phases0, steps, check_every=5)
    anchored["stale_anchor"] = {"wall_s": wall_n, "loss_mean": float(problem.loss(ph_n).cpu().numpy().mean()),
                                **info_n}
    # the same loop without the TVD gate: what the network alone achieves
    ph_u, wall_u, info_u = surrogate_loop(problem, net, phases0, steps, check_every=steps + 1, tvd_tol=float("inf"))
    loss_u = problem.loss(ph_u).clone()
    # time to reach the exact loop's final loss: exact only vs surrogate warm start + exact
    target = float(loss_e.cpu().numpy().mean())
    tt = {}
    for warm in (0, steps // 4, steps):
        sec, used, ok = time_to_target(problem, net, phases0, target, warm, 4 * steps)
        tt[f"warm_{warm}"] = {"seconds": sec, "exact_steps": used, "reached": ok}
    return {
        "time_to_exact_final_loss": tt,
        "samples": samples, "epochs": epochs, "steps": steps, "batch_phase_sets": B,
        "t_data_s": t_data, "t_train_s": t_train, "train_mse_per_epoch": losses,
        "val_tvd_median": float(np.median(val_tvd)), "val_tvd_max": float(val_tvd.max()),
        "loss_initial_mean": float(loss0.cpu().numpy().mean()),
        "exact": {"wall_s": wall_e, "loss_mean": float(loss_e.cpu().numpy().mean())},
        "surrogate": {"wall_s": wall_s, "loss_mean": float(loss_s.cpu().numpy().mean()), **info},
        "speedup_wall": wall_e / wall_s,
        "surrogate_refined_online": refined,
        "anchored": anchored,
        "surrogate_ungated": {"wall_s": wall_u, "loss_mean": float(loss_u.cpu().numpy().mean()),
                              "exact_steps": info_u["exact_steps"]},
        "tensor_core": net.tensor_core,
    }


def _tvd_stats(net: MLP, problem: MeshProblem, phases: torch.Tensor):
    out = []
    for s0 in range(0, phases.shape[0], problem.B):
        out.append(validate(net, problem, phases[s0:s0 + problem.B]).cpu().numpy())
    t = np.concatenate(out)
    return {"median": float(np.median(t)), "p90": float(np.quantile(t, 0.9)), "max": float(t.max()),
            "frac_within_1e-3": float(np.mean(t <= 1e-3))}


def _fit(problem, ph, y, width: int, epochs: int, seed: int, lr_net: float = 1e-3):
    dims = (288, width, width, width, 512)
    Ws, bs = init_weights(seed, dims=dims)
    net = MLP(Ws, bs, lr=lr_net)
    t0 = time.perf_counter()
    losses = train(net, ph, y, epochs)
    torch.cuda.synchronize()
    return net, time.perf_counter() - t0, losses[-1]


def gate_curve(seed: int = 2204006025, B: int = 64, steps: int = 2000):
    """Validation TVD of the surrogate on the 512-output set against the
    training budget: samples, epochs and width on uniformly random phases, and
    training on phases near where the optimisation runs (Gaussian patches of
    width sigma around the 64 start points, and around points of the exact
    loop's trajectory), each validated on held-out phases of its own
    distribution.  Returns a list of records."""
    problem = MeshProblem(B=B, seed=seed)
    rec = []
    ph_all, y_all = make_dataset(problem, 4_000_000, seed + 10)
    val_ph = torch.from_numpy(np.random.default_rng(seed + 30).uniform(0, 2 * np.pi, (4 * B, problem.P))).to(
        problem.dev)
    for samples in (250_000, 500_000, 1_000_000, 2_000_000, 4_000_000):
        net, tt, mse = _fit(problem, ph_all[:samples], y_all[:samples], 1024, 8, seed + 20)
        rec.append({"data": "uniform", "samples": samples, "epochs": 8, "width": 1024, "train_s": tt,
                    "final_mse": mse, "tvd": _tvd_stats(net, problem, val_ph)})
    for epochs in (2, 4, 16, 32):
        net, tt, mse = _fit(problem, ph_all[:2_000_000], y_all[:2_000_000], 1024, epochs, seed + 20)
        rec.append({"data": "uniform", "samples": 2_000_000, "epochs": epochs, "width": 1024, "train_s": tt,
                    "final_mse": mse, "tvd": _tvd_stats(net, problem, val_ph)})
    for width in (256, 512, 2048):
        net, tt, mse = _fit(problem, ph_all[:2_000_000], y_all[:2_000_000], width, 8, seed + 20)
        rec.append({"data": "uniform", "samples": 2_000_000, "epochs": 8, "width": width, "train_s": tt,
                    "final_mse": mse, "tvd": _tvd_stats(net, problem, val_ph)})
    del ph_all, y_all
    # local patches: around the 64 start points, and around 41 points of the
    # exact loop's trajectory (every 50 steps)
    g = np.random.default_rng(seed + 50)
    phases0 = torch.from_numpy(np.random.default_rng(seed + 40).uniform(0, 2 * np.pi, (B, problem.P))).to(
        problem.dev)
    traj = [phases0.clone()]
    ph = phases0.clone()
    opt = Adam64(ph, 0.02)
    for st in range(steps):
        opt.step(problem.loss_and_grad(ph))
        if (st + 1) % 50 == 0:
            traj.append(ph.clone())
    traj = torch.cat(traj)
    for name, centers in (("start_points", phases0), ("trajectory", traj)):
        for sigma in (0.3, 0.1, 0.03):
            n = 2_000_000
            c = centers[torch.from_numpy(g.integers(0, centers.shape[0], n)).to(problem.dev)]
            ph_l = c + sigma * torch.from_numpy(g.standard_normal((n, problem.P))).to(problem.dev)
            y_l = exact_log_probs(ph_l, problem.m, problem.t, problem.outs)
            cv = centers[torch.from_numpy(g.integers(0, centers.shape[0], 4 * B)).to(problem.dev)]
            val_l = cv + sigma * torch.from_numpy(g.standard_normal((4 * B, problem.P))).to(problem.dev)
            net, tt, mse = _fit(problem, ph_l, y_l, 1024, 8, seed + 20)
            rec.append({"data": f"{name}, sigma {sigma}", "samples": n, "epochs": 8, "width": 1024, "train_s": tt,
                        "final_mse": mse, "tvd": _tvd_stats(net, problem, val_l),
                        "tvd_at_centers": _tvd_stats(net, problem, centers)})
            del ph_l, y_l
    return rec


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--curve", action="store_true",
                    help="the surrogate's TVD against training budget and locality (gate_curve)")
    ap.add_argument("--samples", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--no-refine", action="store_true", help="skip the online-refinement variant")
    a = ap.parse_args(argv)
    if a.curve:
        for r in gate_curve():
            print(json.dumps(r), flush=True)
        return
    print(json.dumps(run(a.samples, a.epochs, a.steps, a.batch, refine=not a.no_refine)), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
