"""The multi-GPU path of the benchmark is replicas (every rank compresses and
decompresses its own copy of the workload; blocks never cross ranks, so no
data-path collective exists).  Its host logic -- the slowest rank's times and
the whole-job rate -- runs here on two gloo ranks on the CPU, and two oracle
replicas of the same field give the same container, as independent units must.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # rank r is slower in compression, rank 0 in decompression
    local = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]
    tc, td = bench.rank_max(torch, dist, local, torch.device("cpu"))
    rate = bench.job_rate(world, 1e9, tc + td)
    # each rank compresses its own replica with the oracle
    import sys
    sys.path.insert(0, root)
    from oracle import oracle as O
    from paper_2309_09778_gb300 import gen
    x = gen.signed_lognormal((12, 20, 24), 3.0, 5, 2.0, 0.05)
    st, blob = O.compress(x, 1e-3)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([tc, td, rate, st], np.float64))
    with open(os.path.join(out_dir, f"r{rank}.bin"), "wb") as f:
        f.write(blob)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path, O):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [np.load(tmp_path / f"r{i}.npy") for i in range(world)]
    for v in r:
        assert v[0] == 15.0 and v[1] == 20.0        # the slowest rank's compress and decompress times
        assert v[2] == pytest.approx(2 * 1e9 / (35.0 * 1e6))
        assert v[3] == 0
    assert (tmp_path / "r0.bin").read_bytes() == (tmp_path / "r1.bin").read_bytes()
