"""The layer-level calls of the C-ABI against the oracle: fixed-point sharing and opening
(mpc_share_fixed / mpc_reconstruct_fixed, Sec. 2 Notation, reading D1), the convolution lowered to
one inner product per output (mpc_conv2d, Sec. 4.1) and the standalone truncation with its
verification (mpc_trunc / mpc_verify_trunc, Fig. trunc, reading T5).  Integer results are
compared bit for bit on every share component, plus transcripts, outcomes and ledgers."""
import numpy as np
import pytest

from oracle import protocols as OP
from oracle import verify as OV
from oracle.shares import Session, Shared
from paper_2411_09287_gb300 import workloads
from test_gpu_parity import assert_ledger, assert_shared_equal, check_trace, gpu_shared, seed_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


EDGES = np.array([0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 2.0 ** -13, -(2.0 ** -13), -1e-300, 1e-300,
                  3.999999, -4.0, 2.0 ** 50, -(2.0 ** 50), 2.0 ** 50 - 2.0 ** -13, 1e30, -1e30,
                  np.inf, -np.inf, np.nan, 12345.678, -98765.4321])


@pytest.mark.parametrize("owner", [0, 1, 2])
@pytest.mark.parametrize("on_host", [True, False])
def test_share_fixed_matches_oracle(mpc, owner, on_host):
    k = 13
    seed = seed_of(f"sfix-{owner}-{on_host}")
    x = np.concatenate([EDGES, workloads.rng("sfix").uniform(-8, 8, 3001)])
    ctx, sess = mpc.Context(seed), Session(seed)
    xin = x if on_host else ctx.torch.from_numpy(x).to(ctx.device)
    gx = ctx.share_fixed(7, xin, k, owner=owner)
    ox = OP.share_input(sess, OP.encode_fixed(x, k), 7, owner=owner)
    assert_shared_equal(gpu_shared(mpc, gx, (x.size,)), ox, "share_fixed")
    assert_ledger(mpc, ctx, sess)
    got = ctx.reconstruct_fixed(gx, x.size, k)
    want = OP.decode_fixed(OP.reconstruct(sess, ox), k)
    assert np.array_equal(got, want)
    finite = np.abs(x) < 2.0 ** 49
    assert np.all(np.abs(got[finite] - x[finite]) <= 2.0 ** -k)


CONV = [(2, 3, 9, 8, 3, 3, 1, 0, 3, 13), (1, 2, 7, 7, 3, 2, 2, 1, 4, 13), (2, 1, 8, 8, 5, 5, 1, 2, 3, 13),
        (2, 4, 6, 6, 1, 1, 1, 0, 3, -1), (1, 3, 11, 9, 4, 3, 3, 2, 2, -1)]


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("case", CONV)
def test_conv2d_matches_oracle(mpc, case, path):
    B, C, H, W, kh, kw, stride, pad, O, t = case
    geom = (B, C, H, W, kh, kw, stride, pad)
    seed = seed_of(f"conv-{case}")
    g = workloads.rng(f"conv-{case}")
    x = OP.encode_fixed(g.uniform(-2, 2, (B, C, H, W)), 13)
    wm = OP.encode_fixed(g.uniform(-1, 1, (C * kh * kw, O)), 13)
    ctx, sess = mpc.Context(seed, gemm_path=path), Session(seed)
    gx, gw = ctx.share_input(1, x.reshape(-1)), ctx.share_input(2, wm.reshape(-1))
    cols, zpre, zout, pq, (Mr, N, K) = ctx.conv2d(3, gx, gw, geom, O, t)
    ox, ow = OP.share_input(sess, x, 1), OP.share_input(sess, wm, 2)
    ocols, res = OP.conv2d(sess, ox, ow, 3, geom, t if t >= 0 else None)
    assert_shared_equal(gpu_shared(mpc, cols, (Mr, K)), ocols, "cols")
    assert_shared_equal(gpu_shared(mpc, zpre, (Mr, N)), res.z_pre, "zpre")
    if t >= 0:
        assert_shared_equal(gpu_shared(mpc, zout, (Mr, N)), res.out, "zout")
    rc, tr = ctx.verify_matmul(4, cols, gw, zpre, pq, Mr, N, K, t, 3, trace=True)
    otr = []
    ok = OV.matmul_verify(sess, ocols, ow, res, 4, t if t >= 0 else None, trace=otr)
    assert ok and rc == mpc.MPC_OK
    Rs = [mpc.default_R(K)] + ([mpc.default_R(64 * Mr * N)] if t >= 0 else [])
    check_trace(mpc, tr, otr, Rs)
    assert_ledger(mpc, ctx, sess)
    out = ctx.reconstruct(zout, Mr * N)
    assert np.array_equal(out, OP.reconstruct(sess, res.out).reshape(-1))


def test_conv2d_rejects_bad_geometry(mpc):
    ctx = mpc.Context(seed_of("conv-bad"))
    gx = ctx.shares(2 * 3 * 4 * 4)
    gw = ctx.shares(27 * 2)
    for geom in [(2, 3, 4, 4, 5, 5, 1, 0), (2, 3, 4, 4, 3, 3, 0, 0), (0, 3, 4, 4, 3, 3, 1, 0),
                 (2, 3, 4, 4, 3, 3, 1, -1)]:
        with pytest.raises(mpc.MpcError):
            ctx.conv2d(3, gx, gw, geom, 2, 13)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n,chunk", [(300, None), (400, 128)])
def test_trunc_matches_oracle(mpc, n, chunk, path):
    t = 13
    seed = seed_of(f"trunc-{n}-{chunk}")
    x = OP.encode_fixed(workloads.rng(f"trunc-{n}").uniform(-1000, 1000, n), 26)
    tune = dict(trunc_chunk=chunk, trunc_block=128) if chunk else None
    ctx, sess = mpc.Context(seed, gemm_path=path, tuning=tune), Session(seed)
    gx = ctx.share_input(1, x)
    ox = OP.share_input(sess, x, 1)
    gz, pq = ctx.trunc(2, gx, n, t)
    oz, tp = OP.trunc(sess, ox, 2, t)
    assert_shared_equal(gpu_shared(mpc, gz, (n,)), oz, "trunc out")
    pqh = mpc.to_u64(pq)[: 12 * n].reshape(2, 6, n)
    for c, f in enumerate(Shared.FIELDS):
        assert np.array_equal(pqh[0, c], getattr(tp.p, f).reshape(-1)), f"p.{f}"
        assert np.array_equal(pqh[1, c], getattr(tp.q, f).reshape(-1)), f"q.{f}"
    with pytest.raises(mpc.MpcError):     # the pairs are pending until verified
        ctx.reconstruct(gz, n)
    rc, tr = ctx.verify_trunc(3, pq, n, t, 2, trace=True)
    otr = []
    oks = OV.trunc_verify(sess, tp, 3, t, chunk=chunk, trace=otr)
    assert all(oks) and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [mpc.default_R(64 * (e1 - e0)) for e0, e1 in OV.trunc_chunks(n, chunk)])
    assert_ledger(mpc, ctx, sess)
    got = ctx.reconstruct(gz, n).astype(np.int64)
    d = got - (x.astype(np.int64) >> t)
    assert np.all((d == 0) | (d == 1))


def test_trunc_aborts_on_a_corrupted_mask_switch(mpc):
    seed = seed_of("trunc-fault")
    x = OP.encode_fixed(np.linspace(-3, 3, 500), 26)
    ctx = mpc.Context(seed)
    gx = ctx.share_input(1, x)
    ctx.inject_fault("TRUNC_D1", 123, 1 << 30)
    with pytest.raises(mpc.MpcError) as ei:
        ctx.trunc(2, gx, 500, 13)
    assert ei.value.code == mpc.MPC_ERR_ABORT
    assert ctx.status() == mpc.MPC_ERR_ABORT


@pytest.mark.parametrize("path", [0, 1])
def test_verify_trunc_rejects_a_faulty_pair(mpc, path):
    """P1 -> P2 [m]_1 of the first pair inner product corrupted: only P2's record of <p> is wrong
    (the pairs' masks, hence the mask switch, are not), so the verification must reject."""
    seed = seed_of(f"trunc-pairfault-{path}")
    n = 200
    x = OP.encode_fixed(np.linspace(-3, 3, n), 26)
    ctx, sess = mpc.Context(seed, gemm_path=path), Session(seed)
    gx, ox = ctx.share_input(1, x), OP.share_input(sess, x, 1)
    ctx.inject_fault("MZ1", 77, 1 << 5)
    sess.arm_fault("MZ1", 77, 1 << 5)
    gz, pq = ctx.trunc(2, gx, n, 13)
    oz, tp = OP.trunc(sess, ox, 2, 13)
    rc, tr = ctx.verify_trunc(3, pq, n, 13, 2, trace=True)
    otr = []
    assert not all(OV.trunc_verify(sess, tp, 3, 13, trace=otr))
    assert rc == mpc.MPC_ERR_VERIFY
    check_trace(mpc, tr, otr, [mpc.default_R(64 * n)])


def test_a_corrupted_pair_mask_aborts_the_mask_switch(mpc):
    """P0 -> P2 [Gamma]_2 of the first pair inner product corrupted: P1's m_{r_x}, hence its
    [r_x]_1 and d1, disagree with P0's, and P2's hash check aborts (on both sides)."""
    seed = seed_of("trunc-gammafault")
    x = OP.encode_fixed(np.linspace(-3, 3, 100), 26)
    ctx, sess = mpc.Context(seed), Session(seed)
    gx, ox = ctx.share_input(1, x), OP.share_input(sess, x, 1)
    ctx.inject_fault("GAMMA2", 5, 1 << 9)
    sess.arm_fault("GAMMA2", 5, 1 << 9)
    with pytest.raises(mpc.MpcError) as ei:
        ctx.trunc(2, gx, 100, 13)
    assert ei.value.code == mpc.MPC_ERR_ABORT
    with pytest.raises(OP.Abort):
        OP.trunc(sess, ox, 2, 13)


def _row_keys(req, layer, rows):
    from oracle.shares import obj_id
    return np.array([obj_id(req * 64 + layer, (r >> 16) & 15, r & 0xFFFF) for r in range(rows)],
                    dtype=np.uint64)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("M,N,K,chunk", [(13, 10, 30, None), (20, 7, 16, 64)])
def test_row_keyed_matmul_matches_oracle(mpc, M, N, K, chunk, path):
    """mpc_matmul_keyed / mpc_verify_matmul_keyed: shares, pairs, transcript (chunked too), ledger
    and opened output equal the oracle's with the same row keys (N not a multiple of 8, so a
    ChaCha block of the call's layout would straddle rows)."""
    t = 13
    seed = seed_of(f"keyed-{M}-{N}-{K}-{chunk}")
    g = workloads.rng(f"keyed-{M}-{N}-{K}")
    X = OP.encode_fixed(g.uniform(-2, 2, (M, K)), 13)
    W = OP.encode_fixed(g.uniform(-2, 2, (K, N)), 13)
    keys = _row_keys(5, 2, M)
    tune = dict(trunc_chunk=chunk, trunc_block=128) if chunk else None
    ctx, sess = mpc.Context(seed, gemm_path=path, tuning=tune), Session(seed)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, t, row_keys=keys)
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=t, row_keys=[int(k) for k in keys])
    assert_shared_equal(gpu_shared(mpc, zpre, (M, N)), res.z_pre, "zpre")
    assert_shared_equal(gpu_shared(mpc, zout, (M, N)), res.out, "zout")
    rc, tr = ctx.verify_matmul(4, gx, gw, zpre, pq, M, N, K, t, 3, trace=True, row_keys=keys)
    otr = []
    ok = OV.matmul_verify(sess, ox, ow, res, 4, t, trace=otr, trunc_chunk=chunk)
    assert ok and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [mpc.default_R(K)] + [mpc.default_R(64 * (e1 - e0))
                                                    for e0, e1 in OV.trunc_chunks(M * N, chunk)])
    assert_ledger(mpc, ctx, sess)
    assert np.array_equal(ctx.reconstruct(zout, M * N), OP.reconstruct(sess, res.out).reshape(-1))


def test_keyed_rows_open_the_same_alone_and_packed(mpc):
    K, N, t = 64, 10, 13
    g = workloads.rng("keyed-pack")
    W = OP.encode_fixed(g.uniform(-1, 1, (K, N)), 13)
    XA = OP.encode_fixed(g.uniform(-1, 1, (3, K)), 13)
    XB = OP.encode_fixed(g.uniform(-1, 1, (5, K)), 13)

    def run(X, keys, call):
        ctx = mpc.Context(seed_of("keyed-pack"))
        M = X.shape[0]
        gx, gw = ctx.share_input(call, X), ctx.share_input(call + 1, W)
        zpre, zout, pq = ctx.matmul(call + 2, gx, gw, M, N, K, t, row_keys=keys)
        rc, _ = ctx.verify_matmul(call + 3, gx, gw, zpre, pq, M, N, K, t, call + 2, row_keys=keys)
        assert rc == mpc.MPC_OK
        return ctx.reconstruct(zout, M * N).reshape(M, N)

    alone = run(XA, _row_keys(1, 0, 3), 10)
    packed = run(np.concatenate([XB, XA]), np.concatenate([_row_keys(2, 0, 5), _row_keys(1, 0, 3)]), 50)
    assert np.array_equal(packed[5:], alone)
