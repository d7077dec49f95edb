"""Sharding of independent bound work across ranks (one process per GPU; the
paper runs one host thread per GPU, each with its own subtrees, Sec. 6).

CPU: the round-robin partition, and two gloo ranks bounding disjoint shares
with the oracle whose gathered results equal one process bounding every node
(the host logic alone).

GPU (two gloo ranks, both on the one GPU of this machine; their kernels are
independent and never wait for each other): every rank bounds its share
through librlt2 -- a batch of B&B nodes (distributed.bound_nodes_sharded), a
branch-and-bound search over subtrees with the incumbent exchanged between
rounds (bnb.BranchAndBound(group=...)), and a stream of bound requests with
one server per rank (serve.serve_sharded) -- and the gathered results equal
one process (rlt2_batch_bound, the single-process search, each request
bounded alone) and the oracle / the brute-force optimum.
"""
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


def _run_ranks(target, world, *args):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return got


def test_two_gloo_ranks_equal_one_process():
    got = _run_ranks(_worker, 2)
    F, D = I.clustered_euclid(10, seed=4)
    nodes = I.subproblem_nodes(10, 7, kmin=1, kmax=4)
    ref = [v for _, v in _bound_nodes(list(enumerate(nodes)), F, D, 3)]
    assert got[0] == ref and got[1] == ref


# ------------------------------------------------------------ through librlt2

def _gpu_worker(rank, world, port, q, what):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1510_02065_gb300 import bnb, rlt2, serve
    rlt2.lib()
    if what == "nodes":
        F, D = I.clustered_euclid(16, seed=4)
        nodes = I.subproblem_nodes(16, 13, kmin=1, kmax=9)
        res = dd.bound_nodes_sharded(F, D, nodes, 6)
    elif what == "bnb":
        F, D = I.uniform_symmetric(9, seed=5)
        r = bnb.BranchAndBound(F, D, iters=8, root_iters=12, group=dist.group.WORLD, sync_every=4).solve()
        res = (r["optimum"], r["proven"], None if r["perm"] is None else [int(x) for x in r["perm"]],
               r["nodes_per_rank"], r["ranks"])
    else:
        reqs = []
        for rid in range(7):
            F, D = I.clustered_euclid(8 + rid, seed=rid)
            reqs.append(serve.Request(rid=rid, F=F, D=D, iters=6 + rid, arrival=0.0))
        srv = serve.BoundServer(mem_budget=1 << 30, max_slots=3, passes_per_round=2)
        res = serve.serve_sharded(srv, reqs, realtime=False)["results"]
    q.put((rank, res))
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build, rlt2
    build.build()
    rlt2.lib()
    return t


@pytest.mark.gpu
def test_sharded_nodes_equal_one_batch_and_oracle(gpu):
    from paper_1510_02065_gb300 import rlt2
    got = _run_ranks(_gpu_worker, 2, "nodes")
    F, D = I.clustered_euclid(16, seed=4)
    nodes = I.subproblem_nodes(16, 13, kmin=1, kmax=9)
    one, _ = rlt2.rlt2_batch_bound(F, D, nodes, 6)
    ref = [v for _, v in _bound_nodes(list(enumerate(nodes)), F, D, 6)]
    assert got[0] == got[1] == [int(x) for x in one] == ref


@pytest.mark.gpu
def test_distributed_branch_and_bound_proves_the_optimum(gpu):
    from paper_1510_02065_gb300 import bnb
    from tests.layout import brute_force_qap
    got = _run_ranks(_gpu_worker, 2, "bnb")
    F, D = I.uniform_symmetric(9, seed=5)
    opt = brute_force_qap(F, D)
    single = bnb.BranchAndBound(F, D, iters=8, root_iters=12).solve()
    assert single["optimum"] == opt
    for rank in (0, 1):
        optimum, proven, perm, per_rank, ranks = got[rank]
        assert optimum == opt and proven and ranks == 2
        assert perm is None or bnb.qap_cost(F, D, np.array(perm)) == opt
    assert got[0] == got[1]


@pytest.mark.gpu
def test_one_server_per_rank_equals_requests_alone(gpu):
    from paper_1510_02065_gb300 import rlt2
    got = _run_ranks(_gpu_worker, 2, "serve")
    for rid in range(7):
        F, D = I.clustered_euclid(8 + rid, seed=rid)
        with rlt2.Context(F, D) as c:
            c.iterate(6 + rid)
            alone = c.bound()[1]
        assert got[0][rid] == got[1][rid] == (alone, None), rid
