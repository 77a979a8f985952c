"""A full-size layer of config C3 (4096 x 4096 x 4096 over Z_2^64, uniform 64-bit words,
Pi_Trunc^13, both verification batches, Pi_Rec) on the tensor-core path with the default tuning:
one truncation chunk of 2^24 outputs.  bench.py's default layer, 8192^3, runs the same code in
four chunks and checks 16 sampled outputs the same way on every run; the chunked paths are
compared with the oracle at small sizes in test_gpu_trunc_blocks.py.  The oracle cannot run this
layer whole, so the test checks what holds at any size: the verification accepts, and on sampled
outputs the reconstructed pre-truncation product equals X W mod 2^64 (each computed one by one
with Python integers); a product with one flipped bit is rejected by the same verification."""
import hashlib

import numpy as np
import pytest

from paper_2411_09287_gb300 import workloads

pytestmark = pytest.mark.gpu

N4 = 4096


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


def test_full_size_layer_sampled_outputs(mpc):
    X, W = workloads.gemm_square(N4)
    ctx = mpc.Context(hashlib.sha256(b"fullsize-C3").digest(), gemm_path=mpc.GEMM_LIMB_TC)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, N4, N4, N4, 13)
    rc, _ = ctx.verify_matmul(4, gx, gw, zpre, pq, N4, N4, N4, 13, 3)
    assert rc == mpc.MPC_OK
    zp = ctx.reconstruct(zpre, N4 * N4)
    g = np.random.default_rng(7)
    for _ in range(48):
        a, b = int(g.integers(0, N4)), int(g.integers(0, N4))
        ref = sum(int(X[a, k]) * int(W[k, b]) for k in range(N4)) % (1 << 64)
        assert int(zp[a * N4 + b]) == ref, (a, b)
    # the corners of the output
    for a, b in ((N4 - 1, N4 - 1), (0, N4 - 1), (N4 - 1, 0)):
        ref = sum(int(X[a, k]) * int(W[k, b]) for k in range(N4)) % (1 << 64)
        assert int(zp[a * N4 + b]) == ref, (a, b)
    del ctx, gx, gw, zpre, zout, pq
    import torch
    torch.cuda.empty_cache()


def test_full_size_layer_rejects_a_flipped_bit(mpc):
    X, W = workloads.gemm_square(N4)
    ctx = mpc.Context(hashlib.sha256(b"fullsize-C3-bad").digest(), gemm_path=mpc.GEMM_LIMB_TC)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, N4, N4, N4, 13)
    # corrupt P1's m component of one product entry (an additive attack on the product)
    E = N4 * N4
    idx = 2 * E + 12345
    bad = zpre.clone()
    bad[idx:idx + 1] ^= 1 << 20
    rc, _ = ctx.verify_matmul(4, gx, gw, bad, pq, N4, N4, N4, 13, 3)
    assert rc == mpc.MPC_ERR_VERIFY
