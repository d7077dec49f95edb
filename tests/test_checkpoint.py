"""Checkpoint and resume (rlt2_save / rlt2_load).

A context saved after some passes and resumed in a new context must continue
exactly as the uninterrupted run: the same LB history and the same B, C and D
after further passes, equal to the oracle's.  Corrupt or foreign files are
rejected with RLT2_E_IO.  The last test needs no GPU.
"""
import os

import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2
from tests.layout import compact_y, compact_z


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build
    build.build()
    rlt2.lib()
    return t


@pytest.mark.gpu
@pytest.mark.parametrize("name,rlt1_only,store", [("grid_n12", False, rlt2.RLT2_STORE_TILES),
                                                  ("grid_n12", False, rlt2.RLT2_STORE_CLASSES),
                                                  ("grid_n12", False, rlt2.RLT2_STORE_PAIRS),
                                                  ("uniform_n8", True, rlt2.RLT2_STORE_TILES)])
def test_resume_continues_exactly(gpu, orc, tmp_path, name, rlt1_only, store):
    F, D, _ = I.instance(name)
    N = F.shape[0]
    path = str(tmp_path / "ck.rlt2")
    st = orc.State(F, D, rlt1_only=rlt1_only, paired=store == rlt2.RLT2_STORE_PAIRS)
    for _ in range(7):
        st.iterate()
    with rlt2.Context(F, D, rlt1_only=rlt1_only, max_iters=20, store=store) as ctx:
        ctx.iterate(3)
        ctx.save(path)
        ctx.iterate(4)
        ref_hist = list(ctx.history())
        ref = [ctx.state(0), ctx.state(1)] + ([] if rlt1_only else [ctx.state(2)])
    with rlt2.Context.load(path, max_iters=20) as r:
        assert r.N == N
        assert r.bound()[2] == 3
        r.iterate(4)
        assert list(r.history()) == ref_hist
        got = [r.state(0), r.state(1)] + ([] if rlt1_only else [r.state(2)])
        for a, b in zip(got, ref):
            assert (a == b).all()
        assert r.bound()[1] == st.LB
        assert (got[0] == st.b.reshape(-1)).all()
        assert (got[1] == compact_y(st.c)).all()
        if not rlt1_only:
            assert (got[2].reshape(-1, N - 2, N - 2) == compact_z(st.d)).all()
        # the history must fit the resumed context
        with pytest.raises(rlt2.Rlt2Error) as e:
            rlt2.Context.load(path, max_iters=2)
        assert e.value.code == rlt2.RLT2_E_INVAL


@pytest.mark.gpu
def test_corrupt_files_rejected(gpu, tmp_path):
    F, D, _ = I.instance("uniform_n8")
    path = str(tmp_path / "ck.rlt2")
    with rlt2.Context(F, D) as ctx:
        ctx.iterate(2)
        ctx.save(path)
    data = open(path, "rb").read()
    for bad in (data[:-4], b"NOTACKPT" + data[8:], data[:20]):
        p = str(tmp_path / "bad.rlt2")
        open(p, "wb").write(bad)
        with pytest.raises(rlt2.Rlt2Error) as e:
            rlt2.Context.load(p)
        assert e.value.code == rlt2.RLT2_E_IO


def test_missing_file_is_io_error(tmp_path):
    """No device work happens before the file is opened."""
    rlt2.lib()
    with pytest.raises(rlt2.Rlt2Error) as e:
        rlt2.rlt2_load(str(tmp_path / "does_not_exist"))
    assert e.value.code == rlt2.RLT2_E_IO
