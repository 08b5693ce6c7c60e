"""Multi-process host logic on CPU (gloo, world size 2): the guide-histogram
exchange of a training pass, the record gather of the vMF guide and the
job-throughput reduction of the benchmark.

Each rank bins its own share of the records with the oracle's histogram update;
the summed histogram must equal, bit for bit, the histogram of all records
binned in one process (integer counts: the sum is exact in any order)."""
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


def _records(n, n_cells, seed=11):
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, n_cells, n).astype(np.uint32)
    v = rng.normal(size=(n, 3))
    om = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    w = rng.exponential(1.0, n).astype(np.float32)
    w[::17] = 0.0  # zero-weight records add nothing
    return cell, om, w


def _worker(rank, world, port, n_cells, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2311_12818_gb300 import dist as D
        from paper_2311_12818_gb300 import inputs as I
        cell, om, w = _records(20000, n_cells)
        mine = np.arange(cell.size) % world == rank
        g = O.Guide(n_cells, I.guide_edges())
        g.update(cell[mine], om[mine], w[mine], 16)
        counts = torch.from_numpy(g.counts.view(np.int64).copy())
        D.sum_histograms(counts)
        np.save(os.path.join(out_dir, "counts%d.npy" % rank), counts.numpy())
        t, u = D.job_throughput(10.0 + rank, 100.0 * (rank + 1))
        np.save(os.path.join(out_dir, "tp%d.npy" % rank), np.array([t, u]))
    finally:
        dist.destroy_process_group()


def test_histogram_exchange_and_throughput_reduction(tmp_path):
    from oracle import oracle as O
    from paper_2311_12818_gb300 import inputs as I
    n_cells, world = 16, 2
    mp.start_processes(_worker, args=(world, _free_port(), n_cells, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    cell, om, w = _records(20000, n_cells)
    ref = O.Guide(n_cells, I.guide_edges())
    ref.update(cell, om, w, 16)
    for r in range(world):
        got = np.load(tmp_path / ("counts%d.npy" % r)).view(np.uint64)
        assert np.array_equal(got, ref.counts)
        t, u = np.load(tmp_path / ("tp%d.npy" % r))
        assert t == 11.0 and u == 300.0
    assert ref.counts.sum() > 0


def _vmf_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2311_12818_gb300 import dist as D
        cell, om, w = _records(6000, 8, seed=23)
        k = (np.arange(cell.size) % 3 + 1).astype(np.uint8)
        tau = (np.arange(cell.size) % 2).astype(np.uint8)
        # rank r holds a contiguous share of unequal size (rank order = record order)
        cut = 2500
        sl = slice(0, cut) if rank == 0 else slice(cut, cell.size)
        mine = [torch.from_numpy(a[sl].copy()) for a in (cell.astype(np.int64), om, w, k, tau)]
        got = D.allgather_records(mine)
        g = O.VmfGuide(8).build(got[0].numpy().astype(np.uint32), got[1].numpy(), got[2].numpy(),
                                got[3].numpy(), got[4].numpy(), 16)
        np.savez(os.path.join(out_dir, "vmf%d.npz" % rank), cs=g.cell_start, key=g.key, lobe=g.lobe, prefix=g.prefix)
    finally:
        dist.destroy_process_group()


def test_vmf_records_gather_builds_the_same_guide_on_every_rank(tmp_path):
    from oracle import oracle as O
    world = 2
    mp.start_processes(_vmf_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    cell, om, w = _records(6000, 8, seed=23)
    k = (np.arange(cell.size) % 3 + 1).astype(np.uint8)
    tau = (np.arange(cell.size) % 2).astype(np.uint8)
    ref = O.VmfGuide(8).build(cell, om, w, k, tau, 16)
    for r in range(world):
        z = np.load(tmp_path / ("vmf%d.npz" % r))
        assert np.array_equal(z["cs"], ref.cell_start) and np.array_equal(z["key"], ref.key)
        assert np.array_equal(z["lobe"], ref.lobe) and np.array_equal(z["prefix"], ref.prefix)
