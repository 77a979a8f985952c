"""mpc_reconstruct_noalloc: Pi_Rec for callers that cannot allocate device memory when they
reconstruct.  It must return exactly what mpc_reconstruct returns (integer results: bit-exact),
on consecutive calls that share its fixed device scratch array.  This file is collected last so
that a run stopping at the first failure has run every other test before it."""
import ctypes as C
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


def _noalloc(ctx, xs, n, out):
    return ctx.lib.mpc_reconstruct_noalloc(ctx.h, C.c_void_p(xs.data_ptr()), n,
                                           C.c_void_p(out.data_ptr()))


def test_noalloc_matches_reconstruct_on_consecutive_calls(mpc):
    from paper_2411_09287_gb300 import workloads
    ctx = mpc.Context(hashlib.sha256(b"noalloc").digest())
    sizes = [100003, 777, mpc.NOALLOC_MAX_N]      # several hash leaves, a ragged tail, the limit
    shared = []
    for i, n in enumerate(sizes):
        x = workloads.uniform_words(n, f"noalloc-{i}")
        shared.append((n, x, ctx.share_input(10 + i, x)))
    torch = ctx.torch
    for rep in range(2):                          # two calls in a row per input
        for n, x, xs in shared:
            l0 = ctx.ledger()
            ref = ctx.reconstruct(xs, n, to_host=False)
            l1 = ctx.ledger()
            out = ctx.empty(n)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            rc = _noalloc(ctx, xs, n, out)
            assert rc == mpc.MPC_OK, ctx.lib.mpc_last_error(ctx.h).decode()
            ctx.sync()
            if rep > 0:   # after the first call on the device, nothing is allocated at all
                assert torch.cuda.mem_get_info()[0] == free0, "device memory changed"
            l2 = ctx.ledger()
            # the same messages as mpc_reconstruct: equal ledger increments
            assert l2[1] - l1[1] == l1[1] - l0[1]
            for k in l0[0]:
                assert l2[0][k] - l1[0][k] == l1[0][k] - l0[0][k], k
            got = mpc.to_u64(out)[:n]
            assert np.array_equal(got, mpc.to_u64(ref)[:n]), f"rep {rep}, n {n}"
            assert np.array_equal(got, x)


def test_noalloc_rejects_sizes_beyond_its_array(mpc):
    ctx = mpc.Context(hashlib.sha256(b"noalloc-limit").digest())
    n = mpc.NOALLOC_MAX_N + 1
    xs = ctx.shares(n)
    out = ctx.empty(n)
    rc = _noalloc(ctx, xs, n, out)
    assert rc == mpc.MPC_ERR_SHAPE
    assert "MPC_NOALLOC_MAX_N" in ctx.lib.mpc_last_error(ctx.h).decode()


def test_noalloc_detects_inconsistent_message(mpc):
    from paper_2411_09287_gb300 import workloads
    ctx = mpc.Context(hashlib.sha256(b"noalloc-abort").digest())
    n = 4096
    xs = ctx.share_input(1, workloads.uniform_words(n, "noalloc-abort"))
    ctx.inject_fault("REC_MSG", 99, 1 << 3)
    out = ctx.empty(n)
    assert _noalloc(ctx, xs, n, out) == mpc.MPC_ERR_ABORT
