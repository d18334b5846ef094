"""Multi-process host logic of the benchmark's stream sharding, on CPU with
gloo: every rank owns its own stream (distinct seeds, no pixel exchange),
the slowest rank's time defines the job's time, and the job's throughput
counts every rank's pixels."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import torch.distributed as dist

    import bench
    import oracle
    from cogsynth import Scene
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.stream_seed(3, rank)
    sc = Scene(48, 32, seed, kind="dynamic", n_train=12, fg_frac=0.05)
    fr, _ = sc.frames(0, 20)
    o = oracle.Oracle(oracle.default_params(48, 32, 3))
    o.train(fr[:12])
    t0 = time.perf_counter()
    masks = [o.apply(fr[12 + i])[0] for i in range(8)]
    ms = (time.perf_counter() - t0) * 1e3 + 5.0 * rank      # rank 1 is made slower
    got = bench.max_over_ranks([ms], world)[0]
    digest = float(np.sum(np.stack(masks).astype(np.int64) * np.arange(len(masks[0]))) % 1000003)
    q.put((rank, seed, ms, got, digest, bench.job_mpixel_per_s(48 * 32, 8, got, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_streams_and_take_the_slowest_time():
    import multiprocessing as mp
    oracle = pytest.importorskip("oracle")
    oracle.build_oracle()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, ms0, got0, d0, v0), (r1, s1, ms1, got1, d1, v1) = res
    assert s0 != s1                                  # each rank its own stream
    assert got0 == got1 == max(ms0, ms1)            # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 48 * 32 * 8 / (max(ms0, ms1) / 1e3) / 1e6)
    assert d0 != d1                                  # different streams, different masks
