"""The N > 1 path on CPU: two gloo ranks use bench.py's rank setup and
reductions; rays shard by range (no collective in the data path), and the
sum of the ranks' tallies equals the single-process tally (oracle)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    from oracle import oracle as O
    from paper_2601_04370_gb300 import workloads as W
    ws, r, local, pg = bench.dist_setup(None)
    assert (ws, r) == (world, rank) and pg is not None
    bench.barrier(pg)
    assert bench.allmax(pg, float(rank + 1)) == float(world)
    assert bench.allsum(pg, float(rank + 1)) == float(world * (world + 1) // 2)
    # weak-scaling workload: every rank its own seed
    _, C0 = bench.workload(0, n_rays=1000)
    _, Cr = bench.workload(rank, n_rays=1000)
    assert (Cr.seed == C0.seed) == (rank == 0)
    # sharding by ray range: each rank traces its half, the sum is the full tally
    D, C = W.tiny(n_rays=2000)
    n = C.total_rays
    lo, hi = rank * n // world, (rank + 1) * n // world
    part = torch.tensor(O.trace(D, C, rays=(lo, hi), nthreads=1)["tally"].reshape(-1))
    pg.all_reduce(part)
    np.save(os.path.join(out_dir, f"sum{rank}.npy"), part.numpy())
    pg.destroy_process_group()


def test_two_gloo_ranks_shard_rays(tmp_path):
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2601_04370_gb300 import workloads as W
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    D, C = W.tiny(n_rays=2000)
    full = O.trace(D, C, nthreads=1)["tally"].reshape(-1)
    for r in range(2):
        s = np.load(tmp_path / f"sum{r}.npy")
        assert np.allclose(s, full, rtol=1e-12, atol=1e-15)
