"""Host logic of the multi-GPU bench line, on CPU with gloo (world size 2).

The path has no exchange step, so N GPUs run N independent replicas: the
timed region is bracketed by barriers, each rank times its own steps, and the
line reports every rank's grid points over the slowest rank's time.  The
reduction and that formula are checked here with two CPU ranks; the
reference arm's ranks other than 0 leave without work.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    dist.barrier()
    slowest = bench.max_over_ranks(dist, times[rank], "cpu")
    value = bench.replica_throughput(1000, 10, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, slowest, value))


def test_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]           # ms each rank timed for 10 steps of 1000 points
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 20.0
        assert value == pytest.approx(2 * 1000 * 10 / 20e-3)


def test_single_rank_is_its_own_slowest():
    import bench
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.replica_throughput(64, 100, 1, 2.0) == pytest.approx(64 * 100 / 2e-3)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload = bench.WORKLOAD
        steps = 5
        gpus = 2

    assert bench.run_reference(Args()) == 0


def test_reference_arm_line_on_rank0(monkeypatch, capsys):
    """Rank 0 times the oracle after the requested warm-up steps and prints
    one JSON line with the reference arm's keys."""
    import json
    import bench
    monkeypatch.setenv("RANK", "0")

    class Args:
        workload = "tc_fp64_nr32_n32"
        steps = 2
        warmup = 1
        gpus = 1

    assert bench.run_reference(Args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["warmup"] == 1 and line["steps"] == 2
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert "after 1 untimed steps" in line["cpu_baseline"]["sample"]


@pytest.mark.parametrize("Nr", [9, 32, 64, 256])
def test_bench_norm_weights_match_oracle(Nr):
    """The bench's stated-error norm uses its own Clenshaw-Curtis weights; they
    are the oracle's quadrature (the S14 parity norm) to round-off."""
    import numpy as np
    import bench
    from oracle.grid import Grid
    g = Grid(Nr, 0.875)
    w = bench.cc_radial_weights(Nr)
    assert np.abs(w - g.w).max() <= 1e-14
    assert abs(w.sum() - 1.0) <= 1e-14


def test_bench_weighted_norm_matches_oracle_metric():
    import numpy as np
    import torch
    import bench
    from inputs import Workload, random_state
    from oracle import Model
    wl = Workload("n", Nr=12, Ntheta=12, Nz=12, eta=0.6, Lz=1.0, Re_i=10.0)
    mdl = Model(wl)
    a = random_state(1, 3, 12, mdl.M, mdl.K)
    b = random_state(2, 3, 12, mdl.M, mdl.K)
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    ref = [float(np.sqrt(np.sum(w * np.abs(a[f] - b[f]) ** 2) / np.sum(w * np.abs(b[f]) ** 2)))
           for f in range(3)]
    got = bench.weighted_rel_l2(torch.from_numpy(a), torch.from_numpy(b), mdl.g.r,
                                bench.cc_radial_weights(12))
    assert np.allclose(got, ref, rtol=1e-13)
