"""The host side of an N-rank run on CPU (gloo, world size 2): specimen shards cover every
specimen once with no overlap, a shard becomes a case of its own, and the timing reduction
takes the maximum over ranks."""
import os

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2602_15149_b300 import workloads as W


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        case = W.batched(nspec=12, n_min=200, n_max=600, seed=5)
        mine = bench.shard_specimens(12, rank, ws)
        sub = W.subset(case, mine)
        t = bench.max_over_ranks(1.0 + rank)  # rank 1 is the slow one
        n = bench.sum_over_ranks(sub.n)
        out[rank] = (mine, sub.n, int(sub.specimen_id.max()) + 1, t, n, case.n)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_specimens_and_reduce_times():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, 29517, out), nprocs=ws, join=True)
        res = dict(out)
    shards = [res[r][0] for r in range(ws)]
    assert sorted(shards[0] + shards[1]) == list(range(12)) and not set(shards[0]) & set(shards[1])
    assert res[0][1] + res[1][1] == res[0][5]        # every particle on exactly one rank
    assert res[0][2] == len(shards[0]) and res[1][2] == len(shards[1])  # specimens renumbered 0 .. k-1
    assert res[0][3] == res[1][3] == 2.0              # maximum over ranks
    assert res[0][4] == res[1][4] == res[0][5]        # particle count summed over ranks


def test_subset_keeps_loads_and_materials():
    case = W.batched(nspec=6, n_min=200, n_max=600, seed=2)
    sub = W.subset(case, [1, 4])
    sel = np.isin(case.specimen_id, [1, 4])
    assert sub.n == int(sel.sum())
    assert np.array_equal(sub.X0, case.X0[sel])
    assert len(sub.specimen_loads) == 2 and all(b.mask.shape[0] == sub.n for b in sub.specimen_loads)
    assert all(b.mask.shape[0] == sub.n for b in sub.bcs)
    assert np.array_equal(sub.material_id, case.material_id[sel])


def _rank_steps(rank, ws, port, out):
    """One rank of an N-rank batched run: it takes its specimens, steps them alone (here with the CPU oracle,
    the library's stand-in on a host without a GPU) and sends its displacements to rank 0 for the check."""
    from tests.oracle_cases import make_oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        case = W.batched(nspec=8, n_min=200, n_max=500, seed=9)
        mine = bench.shard_specimens(8, rank, ws)
        sub = W.subset(case, mine)
        o = make_oracle(sub)
        o.step(40)
        ids = np.nonzero(np.isin(case.specimen_id, mine))[0]
        got = [None] * ws
        dist.all_gather_object(got, (ids, o.read("U"), [o.time(s) for s in range(len(mine))]))
        if rank == 0:
            out["gathered"] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_step_their_specimens_like_the_whole_batch():
    """Specimens are independent (own neighbour rows, materials, loads and clocks), so two ranks stepping
    half the batch each reproduce the single run of the whole batch bit for bit, with no exchange on the
    data path: the gathered displacements and clocks equal those of one oracle run of all eight specimens."""
    from tests.oracle_cases import make_oracle

    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_steps, args=(ws, 29531, out), nprocs=ws, join=True)
        got = out["gathered"]
    case = W.batched(nspec=8, n_min=200, n_max=500, seed=9)
    whole = make_oracle(case)
    whole.step(40)
    U = whole.read("U")
    seen = np.zeros(case.n, bool)
    for rank, (ids, u, times) in enumerate(got):
        assert np.array_equal(u, U[ids]), rank
        seen[ids] = True
        for k, s in enumerate(bench.shard_specimens(8, rank, ws)):
            assert times[k] == whole.time(s)
    assert seen.all()
