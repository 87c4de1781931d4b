"""Host logic of the multi-GPU (replica) mode of bench.py on two CPU ranks over gloo.

Each rank fits its own recording (weak scaling): the ranks' seeds differ, the job time is the maximum
over ranks, and the job throughput counts every rank's units.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + rank  # rank 1 is the slow one
        job_s = bench.max_over_ranks(seconds)
        cfg = synth.WORKLOADS["glm_n50_t20k"]
        w = synth.make_workload("glm_n50_t20k", seed=bench.rank_seed(cfg["seed"], rank), n_bins=4000)
        value = bench.job_throughput(w["n"], w["n_bins"], 3, world, job_s)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), job_s=job_s, value=value, offs=w["offs"], bins=w["bins"])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    assert float(r[0]["job_s"]) == float(r[1]["job_s"]) == 2.0        # max over ranks
    assert float(r[0]["value"]) == pytest.approx(50 * 4000 * 3 * world / 2.0)
    # independent recordings: same network size, different spikes
    assert len(r[0]["offs"]) == len(r[1]["offs"])
    assert not (len(r[0]["bins"]) == len(r[1]["bins"]) and np.array_equal(r[0]["bins"], r[1]["bins"]))


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.rank_seed(7, 0) == 7
