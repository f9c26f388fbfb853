"""The surrogate in the optimisation loop against the exact-gradient loop
(small sizes; bench-size numbers come from `python -m
paper_2204_00602_gb300.optimize`).  Checks that the exact loop's gradient
descends, and measures what the trained network gains: the per-step time of a
surrogate step against an exact step, and the surrogate's TVD on the set."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_exact_loop_descends_and_surrogate_steps_are_cheaper():
    from paper_2204_00602_gb300 import optimize as opt
    from paper_2204_00602_gb300.surrogate import MLP, init_weights
    prob = opt.MeshProblem(B=16)
    ph0 = torch.from_numpy(np.random.default_rng(1).uniform(0, 2 * np.pi, (16, prob.P))).cuda()
    l0 = prob.loss(ph0).clone()
    ph, wall_exact = opt.exact_loop(prob, ph0, 100)
    l1 = prob.loss(ph)
    assert torch.all(l1 < l0)

    ph_tr, y_tr = opt.make_dataset(prob, 32768, 5)
    Ws, bs = init_weights(6)
    net = MLP(Ws, bs, lr=1e-3)
    losses = opt.train(net, ph_tr, y_tr, epochs=3)
    assert losses[-1] < losses[0]
    # surrogate-only steps (tolerance never triggers the exact fallback)
    _, wall_sur, info = opt.surrogate_loop(prob, net, ph0, 100, check_every=1000, tvd_tol=1e9)
    assert info["exact_steps"] == 0
    print(f"100 steps: exact {wall_exact:.3f} s, surrogate only {wall_sur:.3f} s")
    assert wall_sur < wall_exact
    # with the 1e-3 tolerance the loop falls back to exact gradients when the
    # surrogate is off: the exact steps are counted and reported
    _, _, info = opt.surrogate_loop(prob, net, ph0, 100, check_every=50, tvd_tol=1e-3)
    assert info["checks"] == 2 and 0 <= info["exact_steps"] <= 100


def test_online_refinement_lowers_the_surrogate_tvd():
    # refinement on the trajectory's exact probabilities (computed anyway at
    # checks and exact steps) must bring the surrogate closer to the exact
    # kernel along the path than the same network without it
    from paper_2204_00602_gb300 import optimize as opt
    from paper_2204_00602_gb300.surrogate import MLP, init_weights
    prob = opt.MeshProblem(B=16)
    ph0 = torch.from_numpy(np.random.default_rng(2).uniform(0, 2 * np.pi, (16, prob.P))).cuda()
    ph_tr, y_tr = opt.make_dataset(prob, 32768, 7)
    Ws, bs = init_weights(8)
    base = MLP(Ws, bs, lr=1e-3)
    opt.train(base, ph_tr, y_tr, epochs=2)
    copy = lambda: MLP([w.cpu().numpy() for w in base.W], [b.cpu().numpy() for b in base.b], lr=1e-3)  # noqa: E731
    _, _, plain = opt.surrogate_loop(prob, copy(), ph0, 200, check_every=10, tvd_tol=1e-3)
    _, _, refined = opt.surrogate_loop(prob, copy(), ph0, 200, check_every=10, tvd_tol=1e-3, refine_steps=20)
    assert refined["refine_steps"] == 20 and refined["checks"] == 20
    assert refined["median_tvd_seen"] < plain["median_tvd_seen"], (plain, refined)


def test_anchored_loop_limits():
    # the anchored loop with a tolerance no check meets takes exact steps
    # throughout and follows the exact loop; with no network and an infinite
    # tolerance it takes one exact step per interval and reuses its gradient
    from paper_2204_00602_gb300 import optimize as opt
    from paper_2204_00602_gb300.surrogate import MLP, init_weights
    prob = opt.MeshProblem(B=16)
    ph0 = torch.from_numpy(np.random.default_rng(3).uniform(0, 2 * np.pi, (16, prob.P))).cuda()
    ph_e, _ = opt.exact_loop(prob, ph0, 40)
    Ws, bs = init_weights(9)
    net = MLP(Ws, bs, lr=1e-3)
    ph_a, _, info = opt.anchored_loop(prob, net, ph0, 40, check_every=5, tvd_tol=-1.0)
    assert info["exact_steps"] == 40 and info["checks"] == 7
    # the same exact steps, with the network's calls in between (they do not
    # touch the exact path's buffers): compare where the two runs end
    la, le = prob.loss(ph_a), prob.loss(ph_e)
    assert torch.allclose(la, le, rtol=1e-2, atol=0), (la, le)
    ph_s, _, info = opt.anchored_loop(prob, None, ph0, 40, check_every=5, tvd_tol=float("inf"))
    assert info["exact_steps"] == 8 and not info["network"]
    assert torch.all(prob.loss(ph_s) < prob.loss(ph0))
