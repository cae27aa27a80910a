"""The multi-process path of the benchmark on CPU: two gloo ranks shard the
targets without overlap and combine the measurement (slowest time, summed
counts) the way the GPU runs do."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2405_12866_gb300 import ranks
    r, w, local = ranks.dist_env()
    seeds = ranks.target_seeds(r, 5) + ranks.warmup_seeds(r, 3)
    mx, sm = ranks.combine([10.0 + r], [3 + r, 100 * (r + 1)])
    out.put((r, w, local, seeds, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_combine():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, mx0, sm0), (r1, w1, l1, s1, mx1, sm1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert not set(s0) & set(s1) and len(set(s0)) == len(set(s1)) == 8
    assert mx0 == mx1 == [11.0]
    assert sm0 == sm1 == [7.0, 300.0]


def test_single_process_combine_is_identity():
    from paper_2405_12866_gb300 import ranks
    assert ranks.combine([1.5], [2, 3]) == ([1.5], [2.0, 3.0])
    with pytest.raises(ValueError):
        ranks.target_seeds(0, 200000)
    with pytest.raises(ValueError):
        ranks.warmup_seeds(0, 60000)
