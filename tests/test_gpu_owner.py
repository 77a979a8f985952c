"""Input sharing by any party, Pi_<.>^{l,k} (Sec. 2), through mpc_share_input_from.

Each test compares the GPU with the oracle:
- the shares, bit for bit, from host and from device input;
- the ledger: P0 sends m_x twice, P1 or P2 sends it once;
- a product of inputs owned by different parties, which verifies and opens;
- a corrupted message to P1, which makes Pi_Rec abort.
"""
import hashlib

import numpy as np
import pytest

from oracle import protocols as OP
from oracle import verify as OV
from oracle.shares import Session
from paper_2411_09287_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


@pytest.mark.parametrize("owner", [0, 1, 2])
def test_share_input_owner_matches_oracle(mpc, owner):
    from test_gpu_parity import assert_ledger, assert_shared_equal, gpu_shared
    seed = hashlib.sha256(f"owner-{owner}".encode()).digest()
    n = 777
    x = workloads.uniform_words(n, "owner-x")
    y = workloads.uniform_words(n, "owner-y")
    ctx, sess = mpc.Context(seed), Session(seed)
    gx = ctx.share_input(9, x, owner=owner)
    ox = OP.share_input(sess, x, 9, owner=owner)
    assert_shared_equal(gpu_shared(mpc, gx, (n,)), ox, "share")
    assert_ledger(mpc, ctx, sess)
    gx_dev = ctx.share_input(9, mpc.from_u64(ctx, x), owner=owner)
    assert np.array_equal(mpc.to_u64(gx_dev), mpc.to_u64(gx))
    OP.share_input(sess, x, 9, owner=owner)             # the same messages in the oracle's ledger
    other = (owner + 1) % 3
    gy, oy = ctx.share_input(10, y, owner=other), OP.share_input(sess, y, 10, owner=other)
    gz, oz = ctx.mult(11, gx, gy, n), OP.mult(sess, ox, oy, 11)
    assert_shared_equal(gpu_shared(mpc, gz, (n,)), oz, "mult")
    rc, _ = ctx.verify_mult(12, gx, gy, gz, n, 11)
    assert rc == mpc.MPC_OK and OV.mult_verify(sess, ox, oy, oz, 12)
    assert_ledger(mpc, ctx, sess)
    assert np.array_equal(ctx.reconstruct(gz, n), x * y)


def test_owner_two_corrupted_message_to_p1_aborts(mpc):
    ctx = mpc.Context(hashlib.sha256(b"owner-fault").digest())
    x = workloads.uniform_words(100, "owner-fault")
    ctx.inject_fault("MX_COPY_P1", 4, 1 << 3)
    gx = ctx.share_input(1, x, owner=2)
    with pytest.raises(mpc.MpcError) as ei:
        ctx.reconstruct(gx, 100)
    assert ei.value.code == mpc.MPC_ERR_ABORT


def test_owner_out_of_range_rejected(mpc):
    ctx = mpc.Context(hashlib.sha256(b"owner-arg").digest())
    with pytest.raises(mpc.MpcError) as ei:
        ctx.share_input(1, workloads.uniform_words(10, "owner-arg"), owner=3)
    assert ei.value.code == mpc.MPC_ERR_ARG
