"""The auction LAP (the paper's GPU method, Sec. 6) against the oracle.

rlt2_lap_batch_auction must reach the optimum the Hungarian method finds: S
equals the oracle's S on every problem (sizes 1..64, heavy ties, sparse and
large values), and the returned assignment is a permutation of cost S.
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


def problems(n, seed):
    rng = np.random.default_rng(seed)
    parts = [rng.integers(0, 3, size=(30, n, n)),
             rng.integers(0, 100, size=(30, n, n)),
             rng.integers(0, 10 ** 6, size=(10, n, n)),
             rng.integers(0, rlt2.RLT2_LAP_MAX_ENTRY + 1, size=(4, n, n)),
             (rng.random((20, n, n)) < 0.3) * rng.integers(1, 1000, size=(20, n, n))]
    return np.concatenate(parts).astype(np.int32)


@pytest.mark.parametrize("n", list(range(1, 21)) + [28, 32, 33, 40, 64])
def test_auction_reaches_the_optimum(torch, orc, n):
    M = problems(n, 500 + n)
    count = M.shape[0]
    dM = torch.from_numpy(M).cuda()
    S = torch.full((count,), -7, dtype=torch.int64, device="cuda")
    A = torch.empty((count, n), dtype=torch.int32, device="cuda")
    W = torch.empty((count,), dtype=torch.int64, device="cuda")
    rc = rlt2.rlt2_lap_batch_auction(dM.data_ptr(), n, count, S.data_ptr(), A.data_ptr(), W.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert rc == 0, rlt2.rlt2_strerror(rc)
    S, A, W = S.cpu().numpy(), A.cpu().numpy(), W.cpu().numpy()
    S0 = orc.lap_batch(M)[0]
    assert (S == S0).all()
    for b in range(count):
        assert sorted(A[b]) == list(range(n))
        assert int(M[b][np.arange(n), A[b]].astype(np.int64).sum()) == S[b]
    assert (W >= n).all()          # at least one bid per person


def test_auction_rejects_out_of_range(torch):
    M = np.zeros((2, 4, 4), np.int32)
    M[1, 2, 3] = -1
    dM = torch.from_numpy(M).cuda()
    S = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc = rlt2.rlt2_lap_batch_auction(dM.data_ptr(), 4, 2, S.data_ptr())
    assert rc == rlt2.RLT2_E_INVAL
    assert S.cpu().numpy().tolist() == [0, -1]
