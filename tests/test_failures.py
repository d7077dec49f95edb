"""Failure detection without a GPU fault.

* A bounded device-side wait that nothing completes gives up and reports
  RLT2_E_TIMEOUT; the device stays usable (the next LAP batch is exact).
* A device allocation beyond the GPU's memory reports RLT2_E_OOM (a batch of
  two 63-facility residual nodes needs about 0.48 TB); the library stays usable.
* Bad inputs are refused before any device work (CPU).
"""
import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2


def test_bad_inputs_refused_on_the_host():
    rlt2.lib()
    F, D = I.uniform_symmetric(5, seed=0)
    Fb = F.copy()
    Fb[1, 2] = -1
    for args in ((Fb, D), (F[:2, :2], D[:2, :2])):
        with pytest.raises(rlt2.Rlt2Error) as e:
            rlt2.Context(*args)
        assert e.value.code == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_selftest_timeout(0) == rlt2.RLT2_E_INVAL


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
def test_bounded_wait_gives_up_and_device_stays_usable(gpu, orc):
    assert rlt2.rlt2_selftest_timeout(1 << 12) == rlt2.RLT2_E_TIMEOUT
    M = np.random.default_rng(0).integers(0, 50, size=(8, 9, 9)).astype(np.int32)
    dM = gpu.from_numpy(M).cuda()
    S = gpu.empty(8, dtype=gpu.int64, device="cuda")
    assert rlt2.rlt2_lap_batch(dM.data_ptr(), 9, 8, S.data_ptr()) == 0
    assert (S.cpu().numpy() == orc.lap_batch(M)[0]).all()


@pytest.mark.gpu
def test_allocation_failure_reported(gpu):
    F, D = I.uniform_symmetric(64, seed=1)
    nodes = [(np.array([0]), np.array([5])), (np.array([3]), np.array([1]))]
    with pytest.raises(rlt2.Rlt2Error) as e:
        rlt2.rlt2_batch_bound(F, D, nodes, 1)
    assert e.value.code == rlt2.RLT2_E_OOM
    F8, D8 = I.uniform_symmetric(8, seed=0)
    with rlt2.Context(F8, D8) as ctx:      # still usable
        ctx.iterate(2)
        assert ctx.bound()[1] > 0
