"""CUDA-graph capture of the communication-free online path of a layer (row a9): input sharing
from device memory and the secure product Pi_Inner + Pi_Trunc enqueue no host synchronisation,
so they can be captured once and replayed; every replay reproduces the eager run bit for bit
(same call ids, so the same pseudo-random masks).  The host-side ledger and pending-product
bookkeeping are recorded when the graph is captured, not on replay."""
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


@pytest.mark.parametrize("path", [0, 1])
def test_captured_layer_replays_bit_exact(mpc, path):
    import torch
    from paper_2411_09287_gb300 import workloads
    M, N, K, t = 128, 96, 200, 13
    seed = hashlib.sha256(b"graph").digest()
    X, W = workloads.gemm_shape(M, N, K, "graph")
    ctx_e = mpc.Context(seed, gemm_path=path)
    Xd, Wd = mpc.from_u64(ctx_e, X.reshape(-1)), mpc.from_u64(ctx_e, W.reshape(-1))

    def layer(ctx, out):
        gx = ctx.share_input(1, Xd, out=out[0])
        gw = ctx.share_input(2, Wd, out=out[1])
        ctx.matmul(3, gx, gw, M, N, K, t, zpre=out[2], zout=out[3], pq=out[4])

    def buffers(ctx):
        return [ctx.shares(M * K), ctx.shares(K * N), ctx.shares(M * N), ctx.shares(M * N),
                ctx.empty(12 * M * N)]

    eager = buffers(ctx_e)
    layer(ctx_e, eager)
    torch.cuda.synchronize()

    ctx_g = mpc.Context(seed, gemm_path=path)
    cap = buffers(ctx_g)
    s = torch.cuda.Stream()
    ctx_g.set_stream(s)
    with torch.cuda.stream(s):
        layer(ctx_g, cap)          # warm-up outside the graph (tensor maps, attributes)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        layer(ctx_g, cap)
    for _ in range(2):
        for b in cap:
            b.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(eager, cap):
            assert torch.equal(a, b)
