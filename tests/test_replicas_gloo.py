"""The multi-process path of the bench on the CPU: two ranks over gloo
(127.0.0.1), each placing its own workload and reducing its elapsed time.

Replicas exchange nothing on the data path, so what a second process can get
wrong is host logic: the ranks must propagate different simulations, every
rank must see the slowest rank's time, and the whole-job rate must count the
updates of all ranks over that time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1903_02581_gb300 import replicas as RP  # noqa: E402
from paper_1903_02581_gb300 import workloads as W  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _signature(w):
    return [(s["beta"]["x0"], s["beta"]["sigma"], s["alpha"]["sigma"], s["lam"]) for s in w["sims"]]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for kind in ("batched", "fullscale"):
            w, name = RP.rank_workload(kind, rank)
            sigs = [None] * world
            dist.all_gather_object(sigs, _signature(w))
            out[kind] = (name, sigs)
        # rank r pretends its timed region took 1 + r seconds
        dist.barrier()
        out["slowest"] = RP.slowest(1.0 + rank)
        out["rate"] = RP.job_rate(world, 32, 16_777_216, 100, out["slowest"])
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_place_distinct_work_and_reduce_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        name, sigs = res[r]["batched"]
        assert name == "batched-32x128x32"
        assert sigs[0] != sigs[1]                           # disjoint blocks of the sweep
        assert not set(sigs[0]) & set(sigs[1])
        assert sigs[0] == _signature(W.batched())           # rank 0 runs the one-GPU workload
        _, fs = res[r]["fullscale"]
        assert fs[0][0][1] == 2.0 and fs[1][0][1] == 1.0    # packet widths cycle over the ranks
        assert res[r]["slowest"] == 2.0                     # every rank sees the slowest time
        assert res[r]["rate"] == pytest.approx(2 * 32 * 16_777_216 * 100 / 2.0)


def test_single_process_helpers():
    assert RP.slowest(3.5) == 3.5                           # no process group: the value itself
    assert RP.job_rate(1, 1, 10, 4, 2.0) == 20.0
    with pytest.raises(ValueError):
        RP.job_rate(1, 1, 10, 4, 0.0)
    with pytest.raises(ValueError):
        RP.rank_workload("other", 0)
    w3, _ = RP.rank_workload("fullscale", 3)
    assert w3["sims"][0]["beta"]["sigma"] == 2.0
    # a shard's sweep keeps the one-GPU recipe: half the simulations without Coulomb
    w1 = W.batched(shard=1)
    assert [s["lam"] for s in w1["sims"]] == [0.0] * 16 + [1.0] * 16
    assert all(-4.0 <= s["beta"]["x0"] - 3.0 <= 4.0 and 1.0 <= s["beta"]["sigma"] <= 3.0 for s in w1["sims"])
