"""Multi-process velocity sharding on CPU (gloo, world size 2 and 3): each rank
searches its v_idx range, rank 0 merges, and the merge equals one search of
the whole lattice byte for byte (candidates, ids, and a top-K cut)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2509_26279_gb300 import shard
from paper_2509_26279_gb300 import workloads as W
from tests import cases


def as_records(r):
    """Oracle result -> (CANDIDATE_DTYPE records, ids)."""
    c = np.zeros(len(r.cands), shard.CANDIDATE_DTYPE)
    for a, b in [("v_idx", "v_idx"), ("bx", "bx"), ("by", "by"), ("count", "distinct"), ("raw", "raw"),
                 ("id_len", "id_len"), ("id_off", "id_off")]:
        c[a] = r.cands[b]
    return c, np.asarray(r.ids, np.uint32)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, k, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cat, grid, n_min = case
        nv = grid.nvx * grid.nvy
        fn = lambda vb, ve: as_records(oracle.stack(cat, grid, n_min, vb, ve, k))
        res = shard.search_sharded(fn, nv, max_candidates=k)
        if rank == 0:
            c, i = res
            np.savez(out_path, c=c.view(np.uint8), i=i)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def run_sharded(case, world, k, tmp_path):
    out = str(tmp_path / f"merged_{world}_{k}.npz")
    mp.start_processes(_worker, args=(world, free_port(), case, k, out), nprocs=world, join=True,
                       start_method="spawn")
    d = np.load(out)
    return d["c"].view(shard.CANDIDATE_DTYPE), d["i"]


@pytest.mark.parametrize("world,k", [(2, 0), (3, 0), (2, 7)])
def test_sharded_search_equals_single(world, k, tmp_path):
    w = W.tiny()
    case = (W.load(w), w.grid, 5)
    c, i = run_sharded(case, world, k, tmp_path)
    ref_c, ref_i = as_records(oracle.stack(case[0], w.grid, 5, 0, None, k))
    assert len(ref_c) == (k if k else len(ref_c)) and len(ref_c) >= 7
    assert c.tobytes() == ref_c.tobytes()
    assert np.array_equal(i, ref_i)


def test_merge_edge_cases():
    cat, grid, n_min = cases.random_tiny(3)
    nv = grid.nvx * grid.nvy
    ref = as_records(oracle.stack(cat, grid, n_min))
    for world in (1, 4, nv + 3):                      # more ranks than velocities: empty shards
        parts = [as_records(oracle.stack(cat, grid, n_min, b, e)) if e > b else
                 (np.zeros(0, shard.CANDIDATE_DTYPE), np.zeros(0, np.uint32))
                 for b, e in shard.velocity_ranges(nv, world)]
        c, i = shard.merge(parts)
        assert c.tobytes() == ref[0].tobytes() and np.array_equal(i, ref[1])
    assert shard.velocity_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    c, i = shard.merge([])
    assert len(c) == 0 and len(i) == 0
