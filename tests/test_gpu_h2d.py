"""Asynchronous copies (mpc_h2d_async / mpc_d2h_async / mpc_h2d_wait): a sharing of inputs
uploaded on the copy stream equals the sharing of the same inputs passed as host memory, word for
word, with the uploads of the next step in flight while the current one runs; an opened result
downloaded on the copy stream equals the one read back by Pi_Rec; an upload waits for the work
enqueued before it that reads its buffer; bad arguments are refused."""
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


def test_uploaded_inputs_share_like_host_inputs(mpc):
    import torch
    seed = hashlib.sha256(b"h2d").digest()
    n = 1 << 20
    g = np.random.default_rng(5)
    xs = [g.integers(0, 2 ** 63, n, dtype=np.uint64) for _ in range(3)]
    ref = mpc.Context(seed)
    want = [mpc.to_u64(ref.share_input(10 + k, x)) for k, x in enumerate(xs)]
    ctx = mpc.Context(seed)
    hosts = [torch.from_numpy(x.view(np.int64)).pin_memory() for x in xs]
    dev = [ctx.empty(n) for _ in range(2)]
    ctx.h2d_async(dev[0], hosts[0], 0)
    got = []
    for k in range(3):
        ctx.h2d_wait(k % 2)
        if k + 1 < 3:
            ctx.h2d_async(dev[(k + 1) % 2], hosts[k + 1], (k + 1) % 2)
        got.append(mpc.to_u64(ctx.share_input(10 + k, dev[k % 2][:n])))
        torch.cuda.synchronize()
    for k in range(3):
        assert np.array_equal(got[k], want[k]), k


def test_upload_arguments_are_checked(mpc):
    import torch
    ctx = mpc.Context(hashlib.sha256(b"h2d-args").digest())
    h = torch.zeros(16, dtype=torch.int64).pin_memory()
    d = ctx.empty(16)
    for bad in (-1, mpc.H2D_SLOTS):
        with pytest.raises(mpc.MpcError):
            ctx.h2d_async(d, h, bad)
        with pytest.raises(mpc.MpcError):
            ctx.h2d_wait(bad)
    ctx.h2d_wait(3)   # a slot never used: nothing to wait for


def test_downloaded_result_equals_host_read(mpc):
    import torch
    ctx = mpc.Context(hashlib.sha256(b"d2h").digest())
    n = 1 << 18
    x = np.random.default_rng(6).integers(0, 2 ** 63, n, dtype=np.uint64)
    xs = ctx.share_input(1, x)
    dev = ctx.reconstruct(xs, n, to_host=False)      # Pi_Rec into device memory
    host = torch.empty(n, dtype=torch.int64).pin_memory()
    ctx.d2h_async(host, dev[:n], 2)                  # ordered after Pi_Rec on the context stream
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy().view(np.uint64), ctx.reconstruct(xs, n))
    assert np.array_equal(host.numpy().view(np.uint64), x)


def test_upload_waits_for_earlier_readers(mpc):
    # a buffer still read by work on the context stream is overwritten only after that work:
    # the sharing enqueued before the upload sees the old words, the one after sees the new
    import torch
    seed = hashlib.sha256(b"h2d-war").digest()
    n = 1 << 24
    g = np.random.default_rng(7)
    old, new = (g.integers(0, 2 ** 63, n, dtype=np.uint64) for _ in range(2))
    ref = mpc.Context(seed)
    want_old = mpc.to_u64(ref.share_input(20, old))
    want_new = mpc.to_u64(ref.share_input(21, new))
    del ref
    ctx = mpc.Context(seed)
    dev = ctx.empty(n)
    dev.copy_(torch.from_numpy(old.view(np.int64)))
    torch.cuda.synchronize()
    s_old = ctx.share_input(20, dev[:n])              # reads dev on the context stream
    hnew = torch.from_numpy(new.view(np.int64)).pin_memory()
    ctx.h2d_async(dev, hnew, 1)
    ctx.h2d_wait(1)
    s_new = ctx.share_input(21, dev[:n])
    torch.cuda.synchronize()
    assert np.array_equal(mpc.to_u64(s_old), want_old)
    assert np.array_equal(mpc.to_u64(s_new), want_new)
