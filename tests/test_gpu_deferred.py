"""Deferred verification of a multiplication circuit, through mpc_verify_mult_calls.

The circuit is a chain of Pi_Mult gates z_(l+1) = z_l y_l, and all of its triples are checked in
one batch before any output is opened. Each test compares, against the oracle's Pi_MultVerify on
the concatenated triples:
- the shares;
- the transcript;
- the outcome.

It also checks two more things:
- an output stays refused until every gate's call is verified;
- a fault in one middle gate is rejected.
"""
import hashlib

import numpy as np
import pytest

from oracle import protocols as OP
from oracle import verify as OV
from oracle.shares import Session, Shared
from paper_2411_09287_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


def _concat(parts):
    return Shared(*(np.concatenate([getattr(p, f) for p in parts]) for f in Shared.FIELDS))


def _run_chain(mpc, ctx, sess, x, ys, fault_layer=None):
    n = x.size
    zg, zo = ctx.share_input(1, x), OP.share_input(sess, x, 1)
    gpu, ora = [], []
    for layer, y in enumerate(ys):
        yg, yo = ctx.share_input(10 + layer, y), OP.share_input(sess, y, 10 + layer)
        if layer == fault_layer:
            ctx.inject_fault("MZ1", 7, 1 << 9)
            sess.arm_fault("MZ1", 7, 1 << 9)
        zg2, zo2 = ctx.mult(100 + layer, zg, yg, n), OP.mult(sess, zo, yo, 100 + layer)
        gpu.append((zg, yg, zg2, n, 100 + layer))
        ora.append((zo, yo, zo2))
        zg, zo = zg2, zo2
    return gpu, ora, zg, zo


def _chain_inputs(n, depth):
    x = workloads.uniform_words(n, "deferred-x")
    return x, [workloads.uniform_words(n, f"deferred-y{layer}") for layer in range(depth)]


def test_deferred_chain_matches_oracle(mpc):
    from test_gpu_parity import assert_shared_equal, check_trace, gpu_shared
    n, depth = 1000, 8
    seed = hashlib.sha256(b"deferred").digest()
    x, ys = _chain_inputs(n, depth)
    ctx, sess = mpc.Context(seed), Session(seed)
    gpu, ora, zg, zo = _run_chain(mpc, ctx, sess, x, ys)
    assert_shared_equal(gpu_shared(mpc, zg, (n,)), zo, "chain output")
    with pytest.raises(mpc.MpcError) as ei:
        ctx.reconstruct(zg, n)
    assert ei.value.code == mpc.MPC_ERR_PENDING
    # the first half of the gates alone: the second half's calls stay pending
    half = depth // 2
    rc, tr = ctx.verify_mult_calls(400, gpu[:half], trace=True)
    otr = []
    ok = OV.mult_verify(sess, *(_concat([t[i] for t in ora[:half]]) for i in range(3)), 400,
                        trace=otr)
    assert ok and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [mpc.default_R(n * half)])
    with pytest.raises(mpc.MpcError) as ei:
        ctx.reconstruct(zg, n)
    assert ei.value.code == mpc.MPC_ERR_PENDING
    rc, tr = ctx.verify_mult_calls(500, gpu[half:], trace=True)
    otr = []
    ok = OV.mult_verify(sess, *(_concat([t[i] for t in ora[half:]]) for i in range(3)), 500,
                        trace=otr)
    assert ok and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [mpc.default_R(n * (depth - half))])
    want = x.copy()
    for y in ys:
        want = want * y
    assert np.array_equal(ctx.reconstruct(zg, n), want)


def test_deferred_ragged_calls_equal_one_concatenated_batch(mpc):
    """Calls of different lengths: the transcript equals mpc_verify_mult's on the concatenation."""
    from test_gpu_parity import check_trace
    seed = hashlib.sha256(b"deferred-ragged").digest()
    lens = [129, 1, 700, 64]
    ctx, sess = mpc.Context(seed), Session(seed)
    gpu, ora = [], []
    for i, m in enumerate(lens):
        a = workloads.uniform_words(m, f"ragged-a{i}")
        b = workloads.uniform_words(m, f"ragged-b{i}")
        ga, gb = ctx.share_input(20 + 2 * i, a), ctx.share_input(21 + 2 * i, b)
        oa, ob = OP.share_input(sess, a, 20 + 2 * i), OP.share_input(sess, b, 21 + 2 * i)
        gpu.append((ga, gb, ctx.mult(200 + i, ga, gb, m), m, 200 + i))
        ora.append((oa, ob, OP.mult(sess, oa, ob, 200 + i)))
    rc, tr = ctx.verify_mult_calls(700, gpu, R=3, trace=True)
    otr = []
    ok = OV.mult_verify(sess, *(_concat([t[i] for t in ora]) for i in range(3)), 700, R=3,
                        trace=otr)
    assert ok and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [3])


@pytest.mark.parametrize("fault_layer", [1, 4])
def test_deferred_chain_rejects_a_fault_in_one_gate(mpc, fault_layer):
    n, depth = 300, 6
    seed = hashlib.sha256(f"deferred-fault-{fault_layer}".encode()).digest()
    x, ys = _chain_inputs(n, depth)
    ctx, sess = mpc.Context(seed), Session(seed)
    gpu, ora, _, _ = _run_chain(mpc, ctx, sess, x, ys, fault_layer)
    rc, _ = ctx.verify_mult_calls(500, gpu)
    try:
        ook = OV.mult_verify(sess, *(_concat([t[i] for t in ora]) for i in range(3)), 500)
        oabort = False
    except OP.Abort:
        ook, oabort = False, True
    assert rc in (mpc.MPC_ERR_VERIFY, mpc.MPC_ERR_ABORT)
    assert not ook
    assert (rc == mpc.MPC_ERR_ABORT) == oabort
    assert ctx.status() == mpc.MPC_ERR_ABORT


def test_deferred_rejects_bad_arguments(mpc):
    ctx = mpc.Context(hashlib.sha256(b"deferred-args").digest())
    x = workloads.uniform_words(10, "deferred-args")
    gx = ctx.share_input(1, x)
    gz = ctx.mult(2, gx, gx, 10)
    with pytest.raises(mpc.MpcError):
        ctx.verify_mult_calls(3, [])
    with pytest.raises(mpc.MpcError):
        ctx.verify_mult_calls(3, [(gx, gx, gz, 10, 1 << 50)])   # call id out of range
    with pytest.raises(mpc.MpcError):
        ctx.verify_mult_calls(3, [(gx, gx, gz, 10, 7)])         # no such pending mpc_mult call
    with pytest.raises(mpc.MpcError):
        ctx.verify_mult_calls(3, [(gx, gx, gz, 10, 2), (gx, gx, gz, 10, 2)])   # listed twice
    with pytest.raises(mpc.MpcError):                           # still pending: refused
        ctx.reconstruct(gz, 10)
    rc, _ = ctx.verify_mult_calls(3, [(gx, gx, gz, 10, 2)])
    assert rc == mpc.MPC_OK
    assert np.array_equal(ctx.reconstruct(gz, 10), x * x)
    with pytest.raises(mpc.MpcError):                           # verified: no longer pending
        ctx.verify_mult_calls(4, [(gx, gx, gz, 10, 2)])
