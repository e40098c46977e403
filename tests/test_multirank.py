"""The N > 1 bench path on CPU with two gloo ranks: replicas on distinct seeded frames,
the job time is the slowest rank's, and only rank 0 reports (no GPU)."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    el, ions, q = bench.make_workload(2, 6, rank)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    dist.barrier()
    out[rank] = (float(ions.sum()), slowest, el.n)
    dist.destroy_process_group()


def test_two_rank_replicas_and_timing():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (s0, t0, n0), (s1, t1, n1) = out[0], out[1]
    assert n0 == n1            # the same electrode on every rank
    assert s0 != s1            # each rank solves its own seeded frame
    assert t0 == t1 == 11.0    # the job time is the slowest rank's


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_other_ranks_do_nothing(capsys):
    import bench

    class A:
        cells, ions, warmup, steps, gpus = 2, 6, 0, 0, 2
    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""
