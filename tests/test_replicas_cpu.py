"""The N-GPU bench path on the CPU: one process per rank over gloo (world
size 2).  The path runs independent replicas (no data-path collective), so
what the ranks share is the whole-job reduction -- the slowest rank's time
and the summed work -- and each rank must draw its own replica's inputs."""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as tdist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs, units = bench._reduce(True, seconds=1.5 + rank, count=1000 * (rank + 1), device="cpu")
        # each rank's replica: its own photons of the tiny configuration
        sc, _ = bench.make_scene("tiny", rank)
        ph = sc.photons(1, "cpu")
        out[rank] = (secs, units, float(ph.pos[:64].double().sum()))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_rank_reduction_and_replica_seeds():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    for r in range(world):
        secs, units, _ = res[r]
        assert secs == 2.5            # max over ranks (1.5, 2.5)
        assert units == 3000.0        # 1000 + 2000
    # replicas draw different inputs
    assert not np.isclose(res[0][2], res[1][2])


def test_single_rank_reduction_is_identity():
    import bench
    assert bench._reduce(False, 0.25, 7) == (0.25, 7.0)
