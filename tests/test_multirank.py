"""The N > 1 benchmark path on CPU with gloo, world size 2: each rank takes a
disjoint frequency chunk of an N-times longer sweep (replicas over
frequencies, no collective on the data path), and the step time is the
maximum over ranks."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.workload(rank, world)
    f = torch.tensor(m.freqs)
    gathered = [torch.zeros_like(f) for _ in range(world)]
    dist.all_gather(gathered, f)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)      # stand-in step times
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((torch.cat(gathered).numpy(), float(t[0]), m.n_tri))
    dist.destroy_process_group()


def test_two_ranks_split_the_sweep():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allf, tmax, ntri = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = np.geomspace(100.0, 1e10, 64)
    assert np.array_equal(np.sort(allf), ref)       # disjoint and complete
    assert len(allf) == 64 and tmax == 2.0
