"""rlt2_lap_batch_static: the allocation-free LAP batch agrees with rlt2_lap_batch.

The static variant is for callers that cannot let the library allocate device
memory (all their memory comes from their own allocator or a fixed budget).
It keeps its scratch in a fixed per-GPU array instead of allocating it, so the
results must be exactly those of the allocating entry point, call after call:
integer results, compared bit for bit.  This file is collected last so that a
run stopping at the first failure has already run every other test; it passes
alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1510_02065_gb300 import rlt2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build
    build.build()
    rlt2.lib()
    return t


def _run(torch, fn, M):
    count, n, _ = M.shape
    dM = torch.from_numpy(np.ascontiguousarray(M, np.int32)).cuda()
    S = torch.full((count,), -7, dtype=torch.int64, device="cuda")
    A = torch.full((count, n), -7, dtype=torch.int32, device="cuda")
    U = torch.full((count, n), -7, dtype=torch.int32, device="cuda")
    V = torch.full((count, n), -7, dtype=torch.int32, device="cuda")
    W = torch.full((count, 2), -7, dtype=torch.int64, device="cuda")
    rc = fn(dM.data_ptr(), n, count, S.data_ptr(), A.data_ptr(), U.data_ptr(), V.data_ptr(),
            W.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, [x.cpu().numpy() for x in (S, A, U, V, W)]


def test_static_entry_matches_allocating_entry_twice(torch):
    rng = np.random.default_rng(2024)
    for call, n in enumerate([18, 28, 33, 64, 18]):
        M = rng.integers(0, 2000, size=(300, n, n)).astype(np.int32)
        rc_ref, ref = _run(torch, rlt2.rlt2_lap_batch, M)
        rc, got = _run(torch, rlt2.rlt2_lap_batch_static, M)
        assert rc_ref == 0 and rc == 0, (call, rc_ref, rc)
        for a, b in zip(ref, got):
            assert (a == b).all(), "call %d (n=%d) differs" % (call, n)


def test_static_entry_reports_bad_entries_then_recovers(torch):
    rng = np.random.default_rng(7)
    M = rng.integers(0, 50, size=(5, 9, 9)).astype(np.int32)
    M[3, 1, 1] = -4
    rc, (S, A, U, V, W) = _run(torch, rlt2.rlt2_lap_batch_static, M)
    assert rc == rlt2.RLT2_E_INVAL and S[3] == -1
    # the status block is cleared by the next call: a clean batch succeeds
    M[3, 1, 1] = 4
    rc, got = _run(torch, rlt2.rlt2_lap_batch_static, M)
    rc_ref, ref = _run(torch, rlt2.rlt2_lap_batch, M)
    assert rc == 0 and rc_ref == 0
    for a, b in zip(ref, got):
        assert (a == b).all()


def test_static_entry_rejects_sizes_beyond_its_maximum(torch):
    assert rlt2.rlt2_lap_batch_static(0, 65, 1, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_lap_batch_static(0, 0, 1, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_lap_batch_static(0, 8, 0, 0) == rlt2.RLT2_OK
