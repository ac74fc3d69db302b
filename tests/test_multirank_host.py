"""Replica (N > 1) path of bench.py on CPU with two gloo ranks: the job time is
the slowest rank's, every rank runs its own disorder realisation, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import syk_inputs as si

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, device="cpu")
        q, J = bench.replica_terms(si, 16, 4.0, rank)
        os.environ["RANK"] = str(rank)
        ref = bench.reference_arm(type("A", (), {"N": 16, "k": 4.0, "steps": 1, "warmup": 1, "gpus": world})()) \
            if rank != 0 else "rank0"
        out.put((rank, t, np.asarray(J).tolist(), ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, t, J, ref = out.get(timeout=120)
        res[rank] = (t, J, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 1.5  # the slowest rank's time on every rank
    assert res[0][1] != res[1][1]  # each rank its own realisation
    import syk_inputs as si

    for r in (0, 1):
        assert np.allclose(res[r][1], si.sample_sparse_syk(16, 4.0, r=r)[1])
    assert res[1][2] is None  # the reference arm does no work off rank 0
