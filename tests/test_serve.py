"""The continuous-batching server: every result in the mix equals the request
bounded alone; admission respects the memory budget; oversize requests are
rejected, not crashed."""
import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2
from paper_1510_02065_gb300.serve import BoundServer, Request

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build
    build.build()
    rlt2.lib()
    return t


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        N = int(rng.integers(5, 12))
        F, D = I.clustered_euclid(N, seed=100 + r)
        reqs.append(Request(rid=r, F=F, D=D, iters=int(rng.integers(2, 9)),
                            arrival=float(rng.integers(0, 12))))
    return reqs


@pytest.mark.parametrize("store", [rlt2.RLT2_STORE_TILES, rlt2.RLT2_STORE_CLASSES])
def test_mix_equals_alone_and_budget_holds(gpu, orc, store):
    reqs = _requests(1, 14)
    biggest = max(rlt2.rlt2_state_bytes(r.N, False, r.iters + 1, store) for r in reqs)
    budget = int(2.5 * biggest)
    srv = BoundServer(mem_budget=budget, max_slots=6, passes_per_round=2, store=store)
    stats = srv.serve(reqs, realtime=False)
    assert stats["completed"] == len(reqs) and stats["rejected"] == 0
    assert srv.peak_bytes <= budget
    assert stats["mean_resident"] > 1.0          # requests really shared launches
    for r in reqs:
        with rlt2.Context(r.F, r.D) as ctx:
            ctx.iterate(r.iters)
            assert ctx.bound()[1] == r.lb, r.rid
    for r in reqs[:4]:
        assert orc.State(r.F, r.D).run(r.iters)[-1] == r.lb


def test_oversize_request_is_rejected(gpu):
    F, D = I.clustered_euclid(9, seed=0)
    small = Request(rid=0, F=F, D=D, iters=3)
    F2, D2 = I.clustered_euclid(14, seed=1)
    big = Request(rid=1, F=F2, D=D2, iters=3)
    srv = BoundServer(mem_budget=rlt2.rlt2_state_bytes(9, False, 4) + 1024)
    stats = srv.serve([small, big], realtime=False)
    assert stats["completed"] == 1 and stats["rejected"] == 1
    assert big.error and small.lb is not None


def test_realtime_latency_stats(gpu):
    reqs = _requests(2, 6)
    for r in reqs:
        r.arrival = r.arrival * 0.01
    stats = BoundServer(mem_budget=1 << 30).serve(reqs, realtime=True)
    assert stats["completed"] == 6
    assert 0 < stats["p50_latency"] <= stats["p99_latency"]
    assert stats["throughput"] > 0


def test_group_rejects_mixed_stores(gpu):
    F, D = I.clustered_euclid(7, seed=1)
    a = rlt2.Context(F, D)
    b = rlt2.Context(F, D, store=rlt2.RLT2_STORE_CLASSES)
    try:
        with pytest.raises(rlt2.Rlt2Error) as e:
            rlt2.rlt2_group_create([a.ctx, b.ctx])
        assert e.value.code == rlt2.RLT2_E_INVAL
    finally:
        a.close()
        b.close()


def test_cancelled_request_leaves_and_others_are_unaffected(gpu):
    """A request cancelled mid-run (its client gives up after 2 of 8 passes)
    and one cancelled while queued leave without a bound; every other result
    equals the request bounded alone."""
    reqs = _requests(3, 8)
    for r in reqs:
        r.iters = 8
    reqs[2].cancel_after = 2
    srv = BoundServer(mem_budget=1 << 40, max_slots=3, passes_per_round=1)
    srv.cancel(reqs[6].rid)
    stats = srv.serve(reqs, realtime=False)
    assert reqs[2].error == "cancelled" and reqs[2].lb is None
    assert reqs[6].error == "cancelled" and reqs[6].lb is None
    assert stats["completed"] == len(reqs) - 2
    for r in reqs:
        if r.error is None:
            with rlt2.Context(r.F, r.D) as ctx:
                ctx.iterate(r.iters)
                assert ctx.bound()[1] == r.lb, r.rid
