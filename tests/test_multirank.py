"""The multi-GPU host logic on CPU ranks (gloo, world size 2): in the bench
each rank simulates its own unitary, the slowest rank's time is the job's
time and the rate counts the work of every rank; in sharding.py both ranks
see the same LPT assignment of uneven circuits (within Graham's bound), the
partial statistics (sum p, TVD, KL) and the partial grad_U of a loss over
the outputs, reduced over the ranks, equal the whole distribution's, the
gathered ranges equal the whole arrays, and the index ranges tile [0, N)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as td
    import bench
    import pcv_inputs as pin
    td.init_process_group("gloo", rank=rank, world_size=world)
    t = 1.0 + rank                                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(t, world, torch.device("cpu"))
    U = pin.haar_unitary(6, bench.rank_unitary_seed(rank))
    gathered = [None] * world
    td.all_gather_object(gathered, U.tobytes())
    td.destroy_process_group()
    out[rank] = (slowest, gathered)


def test_two_cpu_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        slowest, gathered = out[r]
        assert slowest == 2.0
        assert gathered[0] != gathered[1]                # independent problems per rank
    import bench
    assert bench.whole_job_rate(100, 10, 2, 2.0) == 1000.0


# ------------------------------------------------ sharding (host logic)


def _shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import importlib.util
    import torch.distributed as td
    import oracle
    import pcv_inputs as pin
    # sharding.py is loaded by path: the package itself needs the CUDA library
    spec = importlib.util.spec_from_file_location(
        "pcv_sharding", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                     "paper_2204_00602_gb300", "sharding.py"))
    sh = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(sh)
    td.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    # uneven circuits: LPT by routed cost
    circs = pin.batched_circuits(64, 8, 64, 4, 24, 16, seed=pin.BASE_SEED + 3)
    costs = [sh.circuit_cost(c["m"], c["n"], c["input_occ"], c["outputs"]) for c in circs]
    mine = sh.lpt_assign(costs, world)[rank]
    allsets = [None] * world
    td.all_gather_object(allsets, mine)
    res["assign"] = allsets
    res["costs"] = costs
    # distribution statistics over an output split
    m, n = 7, 3
    U = pin.haar_unitary(m, 8101)
    p, _ = oracle.distribution(U, pin.single_photon_input(m, n))
    q = pin.dirichlet_target(p.shape[0], 8102)
    lo, hi = sh.index_range(p.shape[0], rank, world)
    ps, qs = p[lo:hi], q[lo:hi]
    # the ranges reassembled on every rank (the amplitudes as complex values)
    _, a = oracle.distribution(U, pin.single_photon_input(m, n))
    res["gathered_p"] = sh.gather_slices(torch.from_numpy(ps.copy()), p.shape[0]).numpy()
    res["gathered_a"] = sh.gather_slices(torch.from_numpy(a[lo:hi].copy()), p.shape[0]).numpy()
    res["whole"] = (p, a)
    part = torch.tensor([ps.sum(), 0.5 * np.abs(ps - qs).sum(), float(np.sum(qs * np.log(qs / ps)))],
                        dtype=torch.float64)
    res["stats"] = sh.reduce_sum(part).numpy()
    res["full"] = (p.sum(), oracle.tvd(p, q), oracle.kl(q, p))
    # a loss over the outputs: each rank's grad_U from its own outputs, summed
    # over the ranks, is the whole gradient (the all-reduce of grad_U)
    outs = oracle.enumerate_outputs(m, n)
    ga = pin.random_complex_matrix(1, outs.shape[0], 8103)[0]
    t = pin.single_photon_input(m, n)
    mine_g = oracle.grad_U_from_amp_grad(U, t, outs[lo:hi], ga[lo:hi])
    res["grad"] = sh.reduce_sum(torch.from_numpy(mine_g.copy())).numpy()
    res["grad_whole"] = oracle.grad_U_from_amp_grad(U, t, outs, ga)
    td.destroy_process_group()
    out[rank] = res


def test_two_rank_sharding_host_logic():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    r0, r1 = out[0], out[1]
    # both ranks see the same assignment; it partitions the circuits
    assert r0["assign"] == r1["assign"]
    a, b = r0["assign"]
    assert sorted(a + b) == list(range(64)) and not set(a) & set(b)
    costs = np.array(r0["costs"])
    loads = [costs[a].sum(), costs[b].sum()]
    opt_lb = max(costs.sum() / 2, costs.max())
    assert max(loads) <= (4.0 / 3.0) * opt_lb          # Graham's bound for greedy LPT
    # additive statistics: the reduced partial sums are the whole distribution's
    for r in (r0, r1):
        assert np.allclose(r["stats"], r["full"], rtol=1e-13, atol=1e-15)
        # the gathered ranges are the whole arrays, exactly
        p, a = r["whole"]
        assert np.array_equal(r["gathered_p"], p) and np.array_equal(r["gathered_a"], a)
        assert np.abs(r["grad"] - r["grad_whole"]).max() <= 1e-13 * np.abs(r["grad_whole"]).max()


def test_index_ranges_cover_exactly():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "pcv_sharding", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                     "paper_2204_00602_gb300", "sharding.py"))
    sh = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(sh)
    for N in (0, 1, 7, 20_030_010):
        for world in (1, 2, 3, 8):
            ranges = [sh.index_range(N, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == N
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in ranges) - min(h - l for l, h in ranges) <= 1
