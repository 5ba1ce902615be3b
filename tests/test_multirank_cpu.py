"""The bench's N > 1 logic on CPU with two gloo ranks: each rank runs its own
replica box (seed + rank), the job time is the slowest rank's and the value
counts every rank's particles.  No GPU and no collective on the data path."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1209_0461_gb300 import synth
    w = synth.WORKLOADS["pm32_fp64"]
    r = bench.replica(w, rank)
    parts = synth.particles(r)
    local_ms = 10.0 + 5.0 * rank
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    out[rank] = (r.seed, float(parts["pos64"][0, :4].sum()), ms, bench.whole_job_rate(r.npart, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    (s0, p0, ms0, v0), (s1, p1, ms1, v1) = out[0], out[1]
    assert s1 == s0 + 1 and p0 != p1            # independent replica boxes
    assert ms0 == ms1 == 15.0                    # the slowest rank's time on every rank
    assert np.isclose(v0, 2 * 32 ** 3 / 0.015) and v0 == v1
