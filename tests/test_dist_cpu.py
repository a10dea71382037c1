"""Multi-rank host logic on CPU (gloo, world size 2): the row and problem
partitions used when each GPU takes a shard, the absence of any data-path
exchange (each rank's fold-in of its rows equals the same rows of the
unsharded fold-in), and the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_2508_07605_b300.shard import allreduce_increments, lpt_partition, row_range


@pytest.mark.parametrize("m,world", [(0, 2), (1, 2), (7, 2), (4096, 3), (1000003, 8)])
def test_row_ranges_tile_the_rows(m, world):
    ranges = [row_range(m, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == m
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [r1 - r0 for r0, r1 in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_lpt_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0.0, 1.0, 1000)
    parts = lpt_partition(costs, 4)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(1000))
    loads = [costs[p].sum() for p in parts]
    # LPT bound: makespan <= 4/3 OPT, and OPT >= max(mean load, largest job)
    opt_lb = max(costs.sum() / 4, costs.max())
    assert max(loads) <= 4 / 3 * opt_lb + 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    prob = synth.make_sparse_problem(seed=3, m=301, n_cpu=4, n_gpu=16, rank=8, density=0.2,
                                     k=8, lam=0.05, n_heldout=8)
    V = np.random.default_rng(1).standard_normal((prob.n, 8)) / 2
    r0, r1 = row_range(prob.m, rank, world)
    rp = prob.row_ptr[r0:r1 + 1] - prob.row_ptr[r0]
    cl = prob.col[prob.row_ptr[r0]:prob.row_ptr[r1]]
    vl = prob.val[prob.row_ptr[r0]:prob.row_ptr[r1]]
    U, _ = orc.half_step(rp, cl, vl, V, prob.lam)
    # timing reduction as bench.py does it: maximum over ranks
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    parts = [None] * world
    dist.all_gather_object(parts, (r0, r1, U))
    if rank == 0:
        Ufull, _ = orc.half_step(prob.row_ptr, prob.col, prob.val, V, prob.lam)
        got = np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])])
        np.save(os.path.join(out_dir, "diff.npy"), np.abs(got - Ufull).max(keepdims=True))
        np.save(os.path.join(out_dir, "tmax.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_fold_in_shards_without_exchange(tmp_path, orc):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    assert float(np.load(tmp_path / "diff.npy").ravel()[0]) == 0.0
    assert float(np.load(tmp_path / "tmax.npy").ravel()[0]) == float(world)



def _stream_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    rng = np.random.default_rng(11)
    n, k, lam = 48, 6, 0.05
    off = synth.make_sparse_problem(seed=5, m=90, n_cpu=3, n_gpu=16, rank=4, density=0.4, k=k,
                                    lam=lam, n_heldout=8)
    U_off = rng.standard_normal((off.m, k)) / 2
    new = synth.make_sparse_problem(seed=6, m=41, n_cpu=3, n_gpu=16, rank=4, density=0.2, k=k,
                                    lam=lam, n_heldout=8)

    def shard(p, r0, r1):
        return (p.row_ptr[r0:r1 + 1] - p.row_ptr[r0], p.col[p.row_ptr[r0]:p.row_ptr[r1]],
                p.val[p.row_ptr[r0]:p.row_ptr[r1]])

    st = orc.StreamState(n, k, lam)
    o0, o1 = row_range(off.m, rank, world)
    st.add(*shard(off, o0, o1), U_off[o0:o1])                 # this rank's offline shard
    sums = [torch.from_numpy(st.G), torch.from_numpy(st.b), torch.from_numpy(st.cnt)]
    allreduce_increments(sums, None)                          # the totals of every shard
    st.solve()
    base = [t.clone() for t in sums]
    n0, n1 = row_range(new.m, rank, world)
    Un, _ = st.ingest(*shard(new, n0, n1))                    # fold-in against the common V
    allreduce_increments(sums, base)
    st.solve()
    parts = [None] * world
    dist.all_gather_object(parts, (n0, Un, st.V.copy()))
    if rank == 0:
        ref = orc.StreamState(n, k, lam)
        ref.add(off.row_ptr, off.col, off.val, U_off)
        U_all = np.concatenate([p[1] for p in sorted(parts, key=lambda p: p[0])])
        ref.add(new.row_ptr, new.col, new.val, U_all)
        fold = orc.half_step(new.row_ptr, new.col, new.val,
                             orc.StreamState(n, k, lam).add(off.row_ptr, off.col, off.val,
                                                            U_off).copy(), lam)[0]
        dv = max(np.abs(p[2] - ref.V).max() for p in parts)
        du = np.abs(U_all - fold).max()
        np.save(os.path.join(out_dir, "stream.npy"), np.array([dv, du]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_streaming_refit_equals_one_process(tmp_path, orc):
    """The refit's exchange: two ranks each add their shard's terms, sum their
    increments by all-reduce, and solve the V one process gets from all rows."""
    world = 2
    mp.spawn(_stream_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    dv, du = np.load(tmp_path / "stream.npy")
    assert dv <= 1e-11 and du <= 1e-12, (dv, du)
