"""Multi-process host logic (replicas / batch sharding) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1401_4969_gb300 import replicas as R


def test_batch_share_covers_every_problem_once():
    for batch in (1, 2, 3, 7, 256, 257):
        for world in (1, 2, 3, 4, 8):
            seen = []
            sizes = []
            for rank in range(world):
                b, e = R.batch_share(batch, rank, world)
                seen.extend(range(b, e))
                sizes.append(e - b)
            assert seen == list(range(batch))
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.batch_share(4, 2, 2)


def test_env_ranks_defaults_and_torchrun_values():
    assert R.env_ranks({}) == (0, 0, 1)
    assert R.env_ranks({"RANK": "3", "LOCAL_RANK": "1", "WORLD_SIZE": "4"}) == (3, 1, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" 10 + 5 r ms for a share of a 5-problem batch of 1000 unknowns each
        b, e = R.batch_share(5, rank, world)
        rate, ms = R.whole_job_rate(1000.0 * (e - b), 10.0 + 5.0 * rank, dist)
        out.put((rank, rate, ms, R.max_over_ranks(float(rank), dist), R.sum_over_ranks(1.0, dist)))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms, mx, sm in res:
        assert ms == 15.0                       # the slowest rank's time
        assert rate == pytest.approx(5000.0 / 0.015)  # every rank's units over that time
        assert mx == 1.0 and sm == 2.0
