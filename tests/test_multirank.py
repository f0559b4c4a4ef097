"""The N > 1 benchmark path on CPU with gloo, world size 2: each rank takes a
disjoint frequency chunk of an N-times longer sweep (replicas over
frequencies, no collective on the data path), the step time is the
maximum over ranks, and the ranks' R and L gather into the one-rank sweep's
frequency order."""
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
    # stand-in R, L [n_f][2][2] of this rank's frequencies, a known function of f
    R = np.stack([np.full((2, 2), f) for f in m.freqs])
    L = np.stack([np.full((2, 2), 1.0 / f) for f in m.freqs])
    Ra, La = bench.gather_sweep(R, L, world)
    if rank == 0:
        out.put((torch.cat(gathered).numpy(), float(t[0]), m.n_tri, Ra, La))
    dist.destroy_process_group()


def test_two_ranks_split_the_sweep():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allf, tmax, ntri, Ra, La = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = np.geomspace(100.0, 1e10, 64)
    assert np.array_equal(np.sort(allf), ref)       # disjoint and complete
    assert len(allf) == 64 and tmax == 2.0
    # the gathered sweep is the one-rank sweep, in its frequency order
    assert Ra.shape == (64, 2, 2)
    assert np.array_equal(Ra[:, 0, 0], ref) and np.array_equal(La[:, 1, 1], 1.0 / ref)


def test_package_slices_split_over_ranks():
    """The package workloads' frequency slice (bench.spread): N per rank of the
    first N * world frequencies, or of N * world spread over the sweep with
    both ends included; the ranks' slices are disjoint and make up the slice
    one rank would solve at N * world."""
    import bench
    freqs = np.geomspace(1e3, 1e10, 64)
    for even in (False, True):
        for world in (1, 2, 4):
            parts = [bench.spread(freqs, 2, world, r, even) for r in range(world)]
            assert all(len(p) == 2 for p in parts)
            allf = np.sort(np.concatenate(parts))
            assert len(np.unique(allf)) == 2 * world
            assert np.array_equal(allf, np.sort(bench.spread(freqs, 2 * world, 1, 0, even)))
    assert np.array_equal(bench.spread(freqs, 2), freqs[:2])
    assert np.array_equal(bench.spread(freqs, 2, even=True), freqs[[0, 63]])
    assert np.array_equal(bench.spread(freqs, 0), freqs)
