"""Failure detection without a GPU fault: a bounded device wait that runs out (an mbarrier that
nothing arrives at, a limit of a few hundred microseconds) is reported as MPC_ERR_TIMEOUT, the
context aborts for good, and the device stays usable for other contexts."""
import hashlib

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


def test_an_expired_wait_is_reported_and_aborts_the_context(mpc):
    ctx = mpc.Context(hashlib.sha256(b"timeout").digest())
    x = np.arange(100, dtype=np.uint64)
    gx = ctx.share_input(1, x)
    assert ctx.lib.mpc_test_wait_expires(ctx.h, 1_000_000) == mpc.MPC_ERR_TIMEOUT
    assert "bounded device wait" in ctx.lib.mpc_last_error(ctx.h).decode()
    assert ctx.status() == mpc.MPC_ERR_ABORT
    with pytest.raises(mpc.MpcError) as ei:          # sticky: every later call is refused
        ctx.reconstruct(gx, 100)
    assert ei.value.code == mpc.MPC_ERR_ABORT
    # the device still works: a new context shares and opens
    other = mpc.Context(hashlib.sha256(b"timeout-after").digest())
    assert np.array_equal(other.reconstruct(other.share_input(1, x), 100), x)


def test_the_wait_limit_is_checked(mpc):
    ctx = mpc.Context(hashlib.sha256(b"timeout-args").digest())
    assert ctx.lib.mpc_test_wait_expires(ctx.h, 0) == mpc.MPC_ERR_ARG
    assert ctx.lib.mpc_test_wait_expires(ctx.h, 10 ** 9) == mpc.MPC_ERR_ARG
    assert ctx.status() == mpc.MPC_OK
