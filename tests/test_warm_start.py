"""Warm-started children of branch-and-bound nodes (rlt2_child).

A child fixing facility f to location l starts from its parent's dual state
restricted to pi(f) = l (LB + b_fl, B + two C terms, C + three D terms, D
restricted).  On the GPU the derived state and every later pass equal the
oracle's child bit for bit, for the tile and the pair store and in RLT1 mode,
down to a grandchild; bad requests are refused.
"""
import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2
from tests.layout import compact_y, compact_z

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


def same(ctx, st, where):
    N = st.N
    assert ctx.bound()[1] == st.LB, where
    assert (ctx.state(0) == st.b.reshape(-1)).all(), "B " + where
    assert (ctx.state(1) == compact_y(st.c)).all(), "C " + where
    if st.d is not None:
        z = ctx.state(2).reshape(-1, N - 2, N - 2)
        assert (z == compact_z(st.d)).all(), "D " + where


@pytest.mark.parametrize("store", [rlt2.RLT2_STORE_TILES, rlt2.RLT2_STORE_PAIRS])
@pytest.mark.parametrize("name,f,l", [("uniform_n8", 3, 5), ("grid_n12", 0, 11), ("grid_n12", 7, 2)])
def test_child_and_grandchild_equal_oracle(gpu, orc, name, f, l, store):
    F, D, _ = I.instance(name)
    paired = store == rlt2.RLT2_STORE_PAIRS
    st = orc.State(F, D, paired=paired)
    with rlt2.Context(F, D, store=store) as par:
        par.iterate(3)
        st.run(3)
        ch = par.child(f, l)
        och = st.child(f, l)
        try:
            assert och.LB >= st.LB
            same(ch, och, "derived child")
            for t in range(3):
                ch.iterate(1)
                och.iterate()
                same(ch, och, "child pass %d" % (t + 1))
            g = ch.child(1, 0)
            og = och.child(1, 0)
            try:
                same(g, og, "derived grandchild")
                g.iterate(2)
                og.run(2)
                same(g, og, "grandchild after 2 passes")
            finally:
                g.close()
                og.close()
        finally:
            ch.close()
            och.close()


def test_rlt1_child(gpu, orc):
    F, D = I.clustered_euclid(10, seed=4)
    st = orc.State(F, D, rlt1_only=True)
    with rlt2.Context(F, D, rlt1_only=True) as par:
        par.iterate(2)
        st.run(2)
        with par.child(4, 6) as ch:
            och = st.child(4, 6)
            same(ch, och, "rlt1 child")
            ch.iterate(2)
            och.run(2)
            same(ch, och, "rlt1 child after 2 passes")
            och.close()


def test_child_requests_refused(gpu):
    F, D = I.uniform_symmetric(6, seed=2)
    with rlt2.Context(F, D) as par:
        par.iterate(1)
        for f, l in ((-1, 0), (0, 6), (6, 1)):
            with pytest.raises(rlt2.Rlt2Error) as e:
                par.child(f, l)
            assert e.value.code == rlt2.RLT2_E_INVAL
    with rlt2.Context(F, D, store=rlt2.RLT2_STORE_CLASSES) as par:
        with pytest.raises(rlt2.Rlt2Error) as e:
            par.child(0, 0)
        assert e.value.code == rlt2.RLT2_E_INVAL
    F3, D3 = I.uniform_symmetric(3, seed=1)
    with rlt2.Context(F3, D3) as par:
        with pytest.raises(rlt2.Rlt2Error) as e:
            par.child(0, 0)
        assert e.value.code == rlt2.RLT2_E_INVAL
