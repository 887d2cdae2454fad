"""The bounded device-side waits report QK_ERR_DEVICE_TIMEOUT.

Every tcgen05 kernel of the library waits on mbarriers with a clock limit;
a wait that gives up records a code in the caller's error word and raises
the CTA's abort flag so that the other roles leave too.  The self-test entry
point makes such a wait run out on purpose (an mbarrier that nothing
arrives at, a short limit) and checks that a second waiter with the normal
limit leaves through the abort flag.  No kernel faults, traps or hangs.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QK_ERR_DEVICE_TIMEOUT = -7


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib, qmckl
    buildlib.build()
    return qmckl.load()


@pytest.mark.parametrize("limit", [1000, 200000])
def test_short_wait_gives_up_and_aborts_the_other(lib, limit):
    info = np.zeros(4, dtype=np.int32)
    st = lib.qk_selftest_wait_timeout(limit, info.ctypes.data)
    assert st == QK_ERR_DEVICE_TIMEOUT
    assert info[0] == 1                  # the error word holds the wait's code
    assert info[1] == 1                  # the long waiter left through the abort flag
    assert limit <= info[2] < limit + 10**6
    assert info[3] < 2 * 10**9           # far below its own ~4e9-cycle limit
    # the context is still usable afterwards
    x = torch.arange(8, device="cuda", dtype=torch.float32)
    assert float((x * 2).sum()) == 56.0


def test_selftest_rejects_bad_limits(lib):
    assert lib.qk_selftest_wait_timeout(0, None) == -3
    assert lib.qk_selftest_wait_timeout(10**9, None) == -3
