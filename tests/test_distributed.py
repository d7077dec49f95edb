"""Host-side sharding of independent B&B nodes across ranks: two gloo ranks
on the CPU bound disjoint shares (with the oracle) and the gathered results
equal one process bounding every node."""
import os
import socket

import numpy as np
import pytest

from paper_1510_02065_gb300 import distributed as dd
from paper_1510_02065_gb300 import instances as I


def test_shard_partitions():
    units = list(range(11))
    got = sorted(i for r in range(3) for i, _ in dd.shard(units, r, 3))
    assert got == units
    assert [i for i, _ in dd.shard(units, 1, 3)] == [1, 4, 7, 10]
    with pytest.raises(ValueError):
        dd.shard(units, 3, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _bound_nodes(idx_nodes, F, D, iters):
    from oracle import oracle as O
    out = []
    for i, (fac, loc) in idx_nodes:
        Fp, Dp, Bl, cst = O.subproblem(F, D, fac, loc)
        out.append((i, int(O.State(Fp, Dp, B_lin=Bl, lb_const=cst).run(iters)[-1])))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    F, D = I.clustered_euclid(10, seed=4)
    nodes = I.subproblem_nodes(10, 7, kmin=1, kmax=4)
    local = _bound_nodes(dd.shard(nodes, rank, world), F, D, 3)
    res = dd.gather_results(local, len(nodes))
    q.put((rank, res))
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    F, D = I.clustered_euclid(10, seed=4)
    nodes = I.subproblem_nodes(10, 7, kmin=1, kmax=4)
    ref = [v for _, v in _bound_nodes(list(enumerate(nodes)), F, D, 3)]
    assert got[0] == ref and got[1] == ref
