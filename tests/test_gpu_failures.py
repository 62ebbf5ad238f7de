"""Failure detection without a GPU fault: bad arguments and non-finite
input are reported as error codes (see test_gpu_parity.py); a bounded device
wait that nothing satisfies gives up after its limit, reports
CP_ERR_TIMEOUT, and leaves the context usable."""
import ctypes
import time

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04801_gb300 as cp

    return cp


def test_bounded_wait_gives_up(cp):
    lib = cp.load()
    ws = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    rc = lib.cubical_persistence_debug_wait_timeout(ctypes.c_void_p(ws.data_ptr()), ws.numel(), 50_000, None)
    dt = time.perf_counter() - t0
    assert rc == -5  # CP_ERR_TIMEOUT
    assert dt < 5.0
    # the context is still usable afterwards
    img = workloads.uniform((40, 30), 5)
    got = cp.persistence(torch.from_numpy(img).cuda()).numpy()
    want = oracle.persistence(img)
    assert np.array_equal(got["birth_cell"], want["birth_cell"])
    assert lib.cubical_persistence_debug_wait_timeout(ctypes.c_void_p(ws.data_ptr()), 100, 50_000, None) == -1


def test_nonfinite_volume_fails_cleanly(cp):
    vol = workloads.blurred((20, 30, 40), 2.0, 6)
    vol[7, 11, 13] = np.nan
    with pytest.raises(cp.CpError) as e:
        cp.persistence(torch.from_numpy(vol).cuda())
    assert e.value.code == -2
    vol[7, 11, 13] = np.inf
    with pytest.raises(cp.CpError) as e:
        cp.persistence(torch.from_numpy(vol).cuda())
    assert e.value.code == -2
    vol[7, 11, 13] = 0.5  # and a clean call afterwards
    got = cp.persistence(torch.from_numpy(vol).cuda()).numpy()
    assert len(got) == len(oracle.persistence(vol))
