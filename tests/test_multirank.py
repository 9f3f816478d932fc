"""The multi-GPU path is replicas (one process per GPU, no collective on the
data path): its host-side logic -- process-group setup, barriers, the max over
ranks of the timed region, the whole-job aggregate, rank 0 alone running the
reference arm -- checked with world_size 2 over gloo on the CPU."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_setup(argparse.Namespace(impl="theseus"))
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.5 + r, w)          # rank 1 is the slow one: 2.5 ms
    value = bench.weak_value(w, 1000, 4, slowest)
    bench.barrier(w)
    dist.destroy_process_group()
    out.put((r, w, slowest, value))


def test_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    for _, _, slowest, value in got:
        assert slowest == 2.5                              # both ranks see the slowest time
        assert value == 2 * 1000 * 4 / 2.5e-3              # every rank's rows over that time


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(impl="reference", n_dim=1000, n_fact=1000, warmup=0, steps=1, cpu_sample_rows=1000,
                              gpus=2)
    assert bench.reference_arm(args, world=2, rank=1) is None
    assert capsys.readouterr().out == ""
