"""Multi-rank harness on CPU (gloo, world size 2): every rank evaluates its own
shard of parameter sets with no data-path collective; only the timing is
reduced (max over ranks).  Each rank's results must equal a single-process run
of its shard, and the shards must be disjoint."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    import torch.distributed as dist
    w, r, _ = bench.dist_setup("gloo")
    assert (w, r) == (world, rank)
    wl = bench.workload("mcmc_batch", seed_offset=rank)
    idx = np.array([0, 1])
    t = wl["t"][900:1100]
    p = {k: np.asarray(v)[idx] for k, v in wl["params"].items()}
    u = np.array([oracle.q_to_u(a, b) for a, b in zip(p.pop("q1"), p.pop("q2"))])
    p["u1"], p["u2"] = u[:, 0].copy(), u[:, 1].copy()
    flux = oracle.lightcurve(p, t, wl["exptime"][idx], wl["nsuper"], nthreads=1)
    fake_ms = 10.0 + rank
    mx = bench.allreduce_max(fake_ms, w)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), flux)
    np.save(os.path.join(out_dir, f"params{rank}.npy"), wl["params"]["k"])
    with open(os.path.join(out_dir, f"max{rank}.txt"), "w") as fh:
        fh.write(repr(mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_collectives(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    import bench
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    ks = [np.load(tmp_path / f"params{r}.npy") for r in range(world)]
    assert not np.intersect1d(ks[0], ks[1]).size          # disjoint shards
    for r in range(world):
        assert float(open(tmp_path / f"max{r}.txt").read()) == 11.0
        wl = bench.workload("mcmc_batch", seed_offset=r)
        idx = np.array([0, 1])
        p = {k: np.asarray(v)[idx] for k, v in wl["params"].items()}
        u = np.array([oracle.q_to_u(a, b) for a, b in zip(p.pop("q1"), p.pop("q2"))])
        p["u1"], p["u2"] = u[:, 0].copy(), u[:, 1].copy()
        ref = oracle.lightcurve(p, wl["t"][900:1100], wl["exptime"][idx], wl["nsuper"], nthreads=1)
        np.testing.assert_array_equal(np.load(tmp_path / f"rank{r}.npy"), ref)
    assert bench.aggregate_value(2, 1000, 10, 5.0) == 2 * 1000 * 10 / 5e-3
