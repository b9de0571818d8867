"""Multi-rank host logic on the CPU (gloo, world size 2, no GPU).

(1) k-points dealt round-robin to ranks: each rank computes its k-points (the
oracle stands in for the per-rank work), the results are gathered and must
equal the single-process results. (2) One k-point's triangle dealt as 2-D
block-cyclic tiles: the union of the ranks' tiles must cover the triangle
exactly once and reproduce the single-process H and S.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1602_06589_gb300 import partition


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small_batch():
    from workloads import make_system, kpoint_list

    lat = np.diag([9.0, 9.5, 10.0])
    sysm = make_system(77, lat, [(3, 1.7), (2, 1.5)], [2, 1])
    kps = [(0.1, 0.2, 0.3), (0.0, 0.0, 0.0), (0.25, -0.1, 0.05), (0.4, 0.4, 0.1), (-0.2, 0.3, 0.0)]
    kvs = [kpoint_list(lat, k, n) for k, n in zip(kps, (40, 33, 47, 29, 38))]
    return sysm, kvs


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysm, kvs = _small_batch()
    # (1) k-point sharding
    mine = partition.kpoints_of_rank(len(kvs), rank, world)
    res = {}
    for k in mine:
        H, S = oracle.build_HS(sysm, kvs[k])
        res[k] = (H, S)
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    # (2) block-cyclic tiles of k-point 0
    n = kvs[0].shape[0]
    tile = 8
    tiles = partition.tiles_of_rank(n, tile, rank, world)
    rows, cols = [], []
    for bi, bj in tiles:
        for j in range(bj * tile, min(n, (bj + 1) * tile)):
            for i in range(bi * tile, min(n, (bi + 1) * tile)):
                if i <= j:
                    rows.append(i)
                    cols.append(j)
    He, Se = oracle.HS_entries(sysm, kvs[0], rows, cols)
    part = (np.array(rows), np.array(cols), He, Se)
    parts = [None] * world
    dist.all_gather_object(parts, part)
    if rank == 0:
        np.save(os.path.join(out_dir, "ok.npy"), np.array([1]))
        import pickle

        with open(os.path.join(out_dir, "res.pkl"), "wb") as f:
            pickle.dump((gathered, parts), f)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_helpers():
    assert partition.kpoints_of_rank(5, 1, 2) == [1, 3]
    assert partition.grid_shape(2) == (1, 2) and partition.grid_shape(4) == (2, 2)
    n, tile = 50, 8
    seen = {}
    for r in range(4):
        for t in partition.tiles_of_rank(n, tile, r, 4):
            assert t not in seen
            seen[t] = r
    nb = (n + tile - 1) // tile
    assert len(seen) == nb * (nb + 1) // 2


def test_two_ranks_gloo(tmp_path):
    import pickle

    import oracle

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    gathered, parts = pickle.load(open(tmp_path / "res.pkl", "rb"))
    sysm, kvs = _small_batch()
    merged = {}
    for d in gathered:
        merged.update(d)
    assert sorted(merged) == list(range(len(kvs)))
    for k, kv in enumerate(kvs):
        H, S = oracle.build_HS(sysm, kv)
        assert np.array_equal(merged[k][0], H) and np.array_equal(merged[k][1], S)
    n = kvs[0].shape[0]
    H, S = oracle.build_HS(sysm, kvs[0])
    Hc = np.zeros_like(H)
    Sc = np.zeros_like(S)
    count = np.zeros(H.shape, int)
    for rows, cols, He, Se in parts:
        Hc[rows, cols] = He
        Sc[rows, cols] = Se
        count[rows, cols] += 1
    iu = np.triu_indices(n)
    assert np.all(count[iu] == 1) and count.sum() == len(iu[0])
    assert np.array_equal(Hc[iu], H[iu]) and np.array_equal(Sc[iu], S[iu])
