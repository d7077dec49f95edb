"""Parity of the CUDA Hungarian kernel (rlt2_lap_batch) with the oracle.

Bit-exact on integers: optimal value S, assignment, row and column potentials
and the work counts (steps, relaxations), for every size 1..64 (one and two
column slots per lane, packed and unpacked reductions) and value ranges with
many ties.
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


def gpu_lap(torch, M):
    count, n, _ = M.shape
    dM = torch.from_numpy(np.ascontiguousarray(M, np.int32)).cuda()
    S = torch.full((count,), -7, dtype=torch.int64, device="cuda")
    A = torch.empty((count, n), dtype=torch.int32, device="cuda")
    U = torch.empty((count, n), dtype=torch.int32, device="cuda")
    V = torch.empty((count, n), dtype=torch.int32, device="cuda")
    W = torch.empty((count, 2), dtype=torch.int64, device="cuda")
    rc = rlt2.rlt2_lap_batch(dM.data_ptr(), n, count, S.data_ptr(), A.data_ptr(), U.data_ptr(),
                             V.data_ptr(), W.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, S.cpu().numpy(), A.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy(), W.cpu().numpy()


def matrices(n, seed):
    rng = np.random.default_rng(seed)
    parts = [rng.integers(0, 3, size=(40, n, n)),                 # heavy ties
             rng.integers(0, 100, size=(40, n, n)),
             rng.integers(0, 10 ** 6, size=(20, n, n)),            # packed keys, large values
             rng.integers(0, rlt2.RLT2_LAP_MAX_ENTRY + 1, size=(10, n, n)),  # unpacked path
             (rng.random((20, n, n)) < 0.3) * rng.integers(1, 1000, size=(20, n, n))]
    if n > 1:
        parts.append(np.broadcast_to(rng.integers(0, 50, size=(1, n, 1)) +
                                     rng.integers(0, 50, size=(1, 1, n)), (4, n, n)).copy())
    return np.concatenate(parts).astype(np.int32)


@pytest.mark.parametrize("n", list(range(1, 37)) + [40, 47, 48, 63, 64])
def test_lap_parity(torch, orc, n):
    M = matrices(n, 1000 + n)
    rc, S, A, U, V, W = gpu_lap(torch, M)
    assert rc == 0, rlt2.rlt2_strerror(rc)
    S0, A0, U0, V0, W0 = orc.lap_batch(M)
    assert (S == S0).all()
    assert (A == A0).all()
    assert (U == U0).all() and (V == V0).all()
    assert (W[:, 0] == W0[:, 0]).all() and (W[:, 1] == W0[:, 1]).all()


def test_lap_out_of_range_entry_is_reported(torch, orc):
    rng = np.random.default_rng(3)
    M = rng.integers(0, 50, size=(9, 7, 7)).astype(np.int32)
    M[4, 2, 3] = -1
    M[6, 0, 0] = rlt2.RLT2_LAP_MAX_ENTRY + 1
    rc, S, A, U, V, W = gpu_lap(torch, M)
    assert rc == rlt2.RLT2_E_INVAL
    assert S[4] == -1 and S[6] == -1
    ok = [0, 1, 2, 3, 5, 7, 8]
    S0, A0, _, _, _ = orc.lap_batch(M[ok])
    assert (S[ok] == S0).all() and (A[ok] == A0).all()


def test_lap_extreme_values(torch, orc):
    for n in (5, 33, 64):
        M = np.full((3, n, n), rlt2.RLT2_LAP_MAX_ENTRY, np.int32)
        M[1] = 0
        M[2, :, :] = np.arange(n)[None, :] * 8000000
        rc, S, A, U, V, W = gpu_lap(torch, M)
        assert rc == 0
        S0, A0, U0, V0, _ = orc.lap_batch(M)
        assert (S == S0).all() and (A == A0).all() and (U == U0).all() and (V == V0).all()


def test_lap_packing_limit(torch, orc):
    """Entries at the largest value the packed keys take (a batch whose largest
    entry is below 2^25 / 3) and one above it (the unpacked keys), for sizes
    with a free column slot (the sentinel of the packed lane form) and without."""
    lim = (1 << 25) // 3 - 1
    rng = np.random.default_rng(11)
    for top in (lim, lim + 1):
        for n in (2, 5, 31, 32, 33, 63, 64):
            M = np.empty((6, n, n), np.int64)
            M[0] = top
            M[1] = rng.integers(0, top + 1, size=(n, n))
            M[2] = rng.integers(top - 3, top + 1, size=(n, n))
            M[3] = np.arange(n)[None, :] * (top // max(n - 1, 1))
            M[4] = (rng.random((n, n)) < 0.5) * top
            M[5] = top - np.add.outer(np.arange(n), np.arange(n)) % 7
            M = M.astype(np.int32)
            rc, S, A, U, V, W = gpu_lap(torch, M)
            assert rc == 0, rlt2.rlt2_strerror(rc)
            S0, A0, U0, V0, W0 = orc.lap_batch(M)
            assert (S == S0).all() and (A == A0).all(), (top, n)
            assert (U == U0).all() and (V == V0).all(), (top, n)
            assert (W[:, 0] == W0[:, 0]).all() and (W[:, 1] == W0[:, 1]).all(), (top, n)


def test_lap_empty_batch(torch):
    rc = rlt2.rlt2_lap_batch(0, 4, 0, 0)
    assert rc == 0
