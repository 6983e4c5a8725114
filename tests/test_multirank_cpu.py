"""The path shards by history id (each rank runs its own contiguous id
range, with no exchange on the data path); the ranks' int64 tallies and
counters summed with an all-reduce are bit-identical to one rank running
every history.  Checked with two gloo ranks on the CPU, the oracle standing
in for each rank's device work, on the id ranges the product's sharding
helper (paper_2403_06362_gb300.shard, which bench.py uses) assigns."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

from paper_2403_06362_gb300 import shard
from paper_2403_06362_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {}
    for geom in ("slab", "box"):
        L = O.Lcg(m=63, pad=0, g=W.LCG_G, c=1)
        if geom == "slab":
            p = W.slab_small(W.SEED_STRIDE, n_histories=4000)[0]
            lo, hi = shard.rank_range(rank, world, p["n_histories"])
            r = O.slab_run(L, W.to_oracle_problem(p, O), lo, hi)
        else:
            b = W.box_problem(n_histories=1500, mesh=8)
            lo, hi = shard.rank_range(rank, world, b["n_histories"])
            r = O.box_run(L, W.to_oracle_box(b, O), lo, hi)
        t = torch.from_numpy(r["tally"].copy())
        c = torch.from_numpy(r["counts"][:13].astype(np.int64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        out[geom] = (t.numpy(), c.numpy())
    # the microbenchmark's weak-scaling blocks: the ranks' streams are the
    # consecutive blocks of one rank's double-size run
    lo, hi = shard.weak_range(rank, 512)
    st = O.seed_hash(63, W.HASH_SEED, lo, hi - lo)
    fs, _, dg = O.lcg_draw(63, W.LCG_G, W.LCG_C, st, 8)
    parts = [torch.zeros(2 * 512, dtype=torch.int64) for _ in range(2)]
    parts[0][lo:hi] = torch.from_numpy(fs.view(np.int64))
    parts[1][lo:hi] = torch.from_numpy(dg.view(np.int64))
    for x in parts:
        dist.all_reduce(x, op=dist.ReduceOp.SUM)
    out["streams"] = (parts[0].numpy().view(np.uint64), parts[1].numpy().view(np.uint64))
    if rank == 0:
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_single_rank_result(oracle):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    L = oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)
    whole = oracle.slab_run(L, W.to_oracle_problem(W.slab_small(W.SEED_STRIDE, n_histories=4000)[0], oracle))
    assert np.array_equal(got["slab"][0], whole["tally"])
    assert np.array_equal(got["slab"][1], whole["counts"][:13].astype(np.int64))
    wb = oracle.box_run(L, W.to_oracle_box(W.box_problem(n_histories=1500, mesh=8), oracle))
    assert np.array_equal(got["box"][0], wb["tally"])
    assert np.array_equal(got["box"][1], wb["counts"][:13].astype(np.int64))
    st, _, dg = oracle.lcg_draw(63, W.LCG_G, W.LCG_C, oracle.seed_hash(63, W.HASH_SEED, 0, 1024), 8)
    assert np.array_equal(got["streams"][0], st) and np.array_equal(got["streams"][1], dg)


def test_rank_ranges_tile_the_ids():
    for world in (1, 2, 3, 8):
        for total in (0, 1, 7, 4000, 10**8 + 3):
            r = [shard.rank_range(k, world, total) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == total
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    assert shard.weak_range(3, 2**26) == (3 * 2**26, 4 * 2**26)
