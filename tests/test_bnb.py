"""Branch-and-bound on the RLT2 bound (the method's use of the bound, Sec. 6).

GPU: the search proves the brute-force optimum on small instances (uniform,
grid and clustered structure, N = 8 and 9), with and without strong
branching and with the initial incumbent given far above the optimum; the
returned assignment attains the reported cost.  CPU: the host parts (the
objective and the local-search incumbent) against brute force.
"""
import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import bnb
from tests.layout import brute_force_qap, qap_cost


def test_objective_and_local_search_ub():
    for seed in range(3):
        F, D = I.uniform_symmetric(7, seed=seed)
        rng = np.random.default_rng(seed)
        for _ in range(5):
            p = rng.permutation(7)
            assert bnb.qap_cost(F, D, p) == qap_cost(F, D, p)
        opt = brute_force_qap(F, D)
        ub, perm = bnb.local_search_ub(F, D, starts=4, seed=seed)
        assert ub >= opt and bnb.qap_cost(F, D, perm) == ub


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build, rlt2
    build.build()
    rlt2.lib()
    return t


CASES = [("uniform", lambda: I.uniform_symmetric(8, seed=3)),
         ("grid", lambda: I.grid_manhattan(9, rows=3, cols=3, seed=1)),
         ("clustered", lambda: I.clustered_euclid(9, seed=2))]


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", CASES)
def test_proves_brute_force_optimum(gpu, name, make):
    F, D = make()
    opt = brute_force_qap(F, D)
    res = bnb.BranchAndBound(F, D, iters=8, root_iters=20, strong_depth=1).solve()
    assert res["proven"] and res["optimum"] == opt, (name, res)
    assert res["root_lb"] <= opt
    if res["perm"] is not None:
        assert bnb.qap_cost(F, D, res["perm"]) == opt


@pytest.mark.gpu
def test_without_strong_branching_and_with_a_poor_incumbent(gpu):
    F, D = I.clustered_euclid(8, seed=5)
    opt = brute_force_qap(F, D)
    res = bnb.BranchAndBound(F, D, iters=6, root_iters=10, strong_depth=0, ub=10 * opt + 100).solve()
    assert res["proven"] and res["optimum"] == opt
    assert bnb.qap_cost(F, D, res["perm"]) == opt
    assert res["nodes_bounded"] > 0


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", CASES)
def test_warm_started_search_proves_the_same_optimum(gpu, name, make):
    """Children started from their parent's dual state (rlt2_child, advanced
    as one group per node) lead to the same proven optimum."""
    F, D = make()
    opt = brute_force_qap(F, D)
    res = bnb.BranchAndBound(F, D, iters=6, root_iters=20, strong_depth=1, warm=True).solve()
    assert res["proven"] and res["optimum"] == opt and res["warm"], (name, res)
    if res["perm"] is not None:
        assert bnb.qap_cost(F, D, res["perm"]) == opt
