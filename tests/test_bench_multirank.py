"""The multi-rank host logic of bench.py on CPU: two gloo ranks, max-over-ranks timing, the
whole-job value of independent replicas, and rank 0 alone running the reference arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        # rank r took (r+1) ms per step and 10 (r+1) ms in the cost+SGM stages
        step, stage = bench.max_over_ranks([1.0 + rank, 10.0 * (1 + rank)], ws, "cpu")
        value = bench.ms_per_lf(stage, 5, ws)

        class A:
            steps, warmup, workload = 1, 0, "tiny"
        ref = bench.run_reference(A, ws, rank) if rank != 0 else "skipped on rank 0"
        dist.barrier()
        q.put((rank, env, step, stage, value, ref))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_max_and_only_rank0_reports():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=100) for _ in ps)
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, env, step, stage, value, ref in out:
        assert env == (2, rank, rank)
        assert step == 2.0 and stage == 20.0            # the slowest rank decides
        assert value == pytest.approx(20.0 / (5 * 2))   # 2 replicas x 5 light fields in 20 ms
    assert out[1][5] is None                            # rank 1 does no reference work
