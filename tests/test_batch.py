"""Branch-and-bound nodes: residual instances and batched bounding.

* rlt2_subproblem (host code of the library) against the oracle's own
  derivation, entry by entry (CPU, no GPU);
* rlt2_batch_bound (one graph launch for all nodes) against one context per
  node on the same residual instance, and against the oracle, bit for bit.
"""
import numpy as np
import pytest

from paper_1510_02065_gb300 import build
from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2


@pytest.fixture(scope="module")
def L():
    build.build()
    return rlt2.lib()


@pytest.mark.parametrize("seed", range(6))
def test_subproblem_matches_oracle(L, orc, seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(5, 14))
    F, D = I.clustered_euclid(N, seed=seed)
    if seed % 2:
        F = rng.integers(0, 9, size=(N, N)).astype(np.int32)   # asymmetric
        np.fill_diagonal(F, 0)
    k = int(rng.integers(0, N - 2))
    fac = rng.choice(N, size=k, replace=False)
    loc = rng.choice(N, size=k, replace=False)
    Fp, Dp, Bl, cst = rlt2.rlt2_subproblem(F, D, fac, loc)
    Fo, Do, Blo, csto = orc.subproblem(F, D, fac, loc)
    assert (Fp == Fo).all() and (Dp == Do).all() and (Bl == Blo).all() and cst == csto


def test_subproblem_rejects_repeats(L):
    F, D = I.uniform_symmetric(6, seed=0)
    with pytest.raises(rlt2.Rlt2Error):
        rlt2.rlt2_subproblem(F, D, [1, 1], [2, 3])
    with pytest.raises(rlt2.Rlt2Error):
        rlt2.rlt2_subproblem(F, D, [1, 7], [2, 3])


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rlt2.lib()
    return t


@pytest.mark.gpu
@pytest.mark.parametrize("store", [rlt2.RLT2_STORE_TILES, rlt2.RLT2_STORE_CLASSES, rlt2.RLT2_STORE_PAIRS])
def test_batch_equals_single_contexts_and_oracle(gpu, orc, store):
    F, D = I.clustered_euclid(12, seed=3)
    nodes = []
    rng = np.random.default_rng(5)
    for s in range(10):
        k = int(rng.integers(0, 8))           # residual sizes 4..12, ragged
        nodes.append((rng.choice(12, size=k, replace=False), rng.choice(12, size=k, replace=False)))
    iters = 7
    lbs, ms = rlt2.rlt2_batch_bound(F, D, nodes, iters, store=store)
    assert ms > 0
    for b, (fac, loc) in enumerate(nodes):
        Fp, Dp, Bl, cst = rlt2.rlt2_subproblem(F, D, fac, loc)
        with rlt2.Context(Fp, Dp, B_lin=Bl, lb_const=cst, store=store) as ctx:
            ctx.iterate(iters)
            assert ctx.bound()[1] == lbs[b], b
        st = orc.State(Fp, Dp, B_lin=Bl, lb_const=cst, paired=store == rlt2.RLT2_STORE_PAIRS)
        assert st.run(iters)[-1] == lbs[b], b


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("store", [rlt2.RLT2_STORE_TILES, rlt2.RLT2_STORE_CLASSES, rlt2.RLT2_STORE_PAIRS])
def test_batch_two_column_slots(gpu, store):
    """Nodes of a 34-facility instance with N' = 34, 33, 32 (two column slots
    per lane in the group's D->C kernel) and one with N' = 30 in the same
    range: the batch gives every node the bound of its own single context."""
    N = 34
    F, D = I.clustered_euclid(N, seed=12)
    nodes = [(np.array([], np.int32), np.array([], np.int32)), (np.array([5]), np.array([9])),
             (np.array([0, 17]), np.array([33, 2])), (np.array([1, 2, 3, 4]), np.array([8, 6, 4, 2]))]
    iters = 3
    lbs, _ = rlt2.rlt2_batch_bound(F, D, nodes, iters, store=store)
    for b, (fac, loc) in enumerate(nodes):
        Fp, Dp, Bl, cst = rlt2.rlt2_subproblem(F, D, fac, loc)
        with rlt2.Context(Fp, Dp, B_lin=Bl, lb_const=cst, store=store) as ctx:
            ctx.iterate(iters)
            assert ctx.bound()[1] == lbs[b], (b, N - len(fac))


@pytest.mark.gpu
def test_batch_of_one_and_zero_passes(gpu):
    F, D = I.uniform_symmetric(9, seed=2)
    lbs, _ = rlt2.rlt2_batch_bound(F, D, [(np.array([], np.int32), np.array([], np.int32))], 4)
    with rlt2.Context(F, D) as ctx:
        ctx.iterate(4)
        assert ctx.bound()[1] == lbs[0]
    fac, loc = np.array([2]), np.array([5])
    lbs0, _ = rlt2.rlt2_batch_bound(F, D, [(fac, loc)], 0)
    assert lbs0[0] == rlt2.rlt2_subproblem(F, D, fac, loc)[3]


@pytest.mark.gpu
def test_batch_rejects_too_small_residual(gpu):
    F, D = I.uniform_symmetric(6, seed=1)
    with pytest.raises(rlt2.Rlt2Error):
        rlt2.rlt2_batch_bound(F, D, [(np.arange(4), np.arange(4))], 2)   # N' = 2


@pytest.mark.gpu
def test_batch_shapes_autotuned_and_forced_agree(gpu):
    """Nodes with N' <= 16 and larger ones in one batch (two D->C ranges): the
    autotuned run (tuning passes first) and forced shapes give the same
    bounds; the shapes used are reported per range."""
    F, D = I.clustered_euclid(20, seed=9)
    rng = np.random.default_rng(9)
    nodes = []
    for s in range(12):
        k = int(rng.integers(1, 12))          # N' from 9 to 19: both ranges present
        nodes.append((rng.choice(20, size=k, replace=False), rng.choice(20, size=k, replace=False)))
    nodes.append((np.array([4]), np.array([7])))   # N' = 19
    nodes.append((np.arange(8), np.arange(8)[::-1].copy()))   # N' = 12
    lb_auto, _, shapes = rlt2.rlt2_batch_bound(F, D, nodes, 6, return_lanes=True)
    (l0, w0), (l1, w1) = shapes
    assert l0 == 32 and w0 in (4, 16, 32) and l1 in (16, 32) and w1 in (4, 16, 32)
    for kw in (dict(lanes=32), dict(cta_warps=4), dict(cta_warps=16), dict(cta_warps=32)):
        lb, _, got = rlt2.rlt2_batch_bound(F, D, nodes, 6, return_lanes=True, **kw)
        assert list(lb) == list(lb_auto), kw
        assert got[0][0] == got[1][0] == 32, (kw, got)
        if "cta_warps" in kw:
            assert got[0][1] == got[1][1] == kw["cta_warps"], (kw, got)
    with pytest.raises(rlt2.Rlt2Error):       # half-warps do not cover the N' = 19 rows
        rlt2.rlt2_batch_bound(F, D, nodes, 2, lanes=16)
    big = [(f, l) for f, l in nodes if 20 - len(f) > 16]
    _, _, shapes_big = rlt2.rlt2_batch_bound(F, D, big, 5, return_lanes=True)
    assert shapes_big[1] == (0, 0) and shapes_big[0][0] == 32
