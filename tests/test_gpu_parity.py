"""CUDA path vs oracle, element by element, through the C-ABI (libmpc3).

Each test runs a protocol on the GPU and the same protocol in the oracle with the same seed and
inputs, and compares every share component of every output (bit-exact, integer work), the
verification transcripts (revealed challenges, the shares of h(0) and h(p2) of every Pi_Reduce
round, the opened Delta), accept/reject outcomes, and the ledger.
"""
import hashlib

import numpy as np
import pytest

from oracle import protocols as OP
from oracle import verify as OV
from oracle.shares import Session, Shared
from paper_2411_09287_gb300 import workloads

pytestmark = pytest.mark.gpu

U64 = np.uint64


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


def seed_of(name):
    return hashlib.sha256(name.encode()).digest()


def gpu_shared(M, t, shape):
    a = M.to_u64(t)
    n = int(np.prod(shape))
    a = a[: 6 * n].reshape(6, *shape)
    return Shared(*(a[i].copy() for i in range(6)))


def assert_shared_equal(g: Shared, o: Shared, what=""):
    for f in Shared.FIELDS:
        a, b = getattr(g, f), getattr(o, f)
        assert a.shape == b.shape, (what, f, a.shape, b.shape)
        bad = np.flatnonzero(a.reshape(-1) != b.reshape(-1))
        assert bad.size == 0, f"{what}.{f}: {bad.size} mismatches, first at {bad[:5]}"


def trace_rounds(trace_list):
    rounds = [t for t in trace_list if "round" in t]
    deltas = [t["delta"] for t in trace_list if "delta" in t]
    return rounds, deltas


def check_trace(M, gtrace, otrace, R_list):
    """GPU trace (flat) against the oracle's trace list; R_list = rounds of each batch."""
    g = M.to_u64(gtrace)
    rounds, deltas = trace_rounds(otrace)
    off = 0
    ri = 0
    for bi, R in enumerate(R_list):
        for k in range(R):
            o = rounds[ri]
            ri += 1
            base = off + k * M.TRACE_ROUND
            assert np.array_equal(g[base:base + 64], o["zeta_prime"]), f"batch {bi} round {k+1} zeta'"
            h0 = g[base + 64: base + 448].reshape(6, 64)
            h2 = g[base + 448: base + 832].reshape(6, 64)
            for c, f in enumerate(Shared.FIELDS):
                assert np.array_equal(h0[c], getattr(o["h0"], f)), f"batch {bi} round {k+1} h0.{f}"
                assert np.array_equal(h2[c], getattr(o["h2"], f)), f"batch {bi} round {k+1} h2.{f}"
        d = g[off + R * M.TRACE_ROUND: off + R * M.TRACE_ROUND + 64]
        assert np.array_equal(d, deltas[bi]), f"batch {bi} Delta"
        off += (R + 1) * M.TRACE_ROUND


def ledger_of(sess: Session):
    out = {}
    for e in sess.ledger:
        out[(e.phase, e.proto)] = out.get((e.phase, e.proto), 0) + e.nbytes
    return out


def assert_ledger(M, ctx, sess):
    g, _ = ctx.ledger()
    o = ledger_of(sess)
    for key in set(g) | set(o):
        assert g.get(key, 0) == o.get(key, 0), (key, g.get(key, 0), o.get(key, 0))


# ---------------------------------------------------------------------------------------------
def test_share_input_matches_oracle(mpc):
    seed = seed_of("share")
    x = workloads.uniform_words(1000 + 3, "share-test")
    ctx = mpc.Context(seed)
    sess = Session(seed)
    g = ctx.share_input(7, x)
    o = OP.share_input(sess, x, 7)
    assert_shared_equal(gpu_shared(mpc, g, x.shape), o, "share")
    # device input gives the same sharing
    g2 = ctx.share_input(7, mpc.from_u64(ctx, x))
    assert np.array_equal(mpc.to_u64(g2), mpc.to_u64(g))


@pytest.mark.parametrize("mode", [0, 1])
def test_plain_small_mult_and_verify(mpc, mode):
    """Config 'plain protocol, small': Pi_Mult of two 4096-vectors, Pi_MultVerify, Pi_Rec."""
    seed = workloads.master_seed("C1")
    _, _, a, b = workloads.plain_small()
    xa, xb = OP.encode_fixed(a, 13), OP.encode_fixed(b, 13)
    ctx = mpc.Context(seed, reduce_mode=mode)
    sess = Session(seed, reduce_mode="x" if mode == 0 else "zeta2")
    n = a.size
    ga, gb = ctx.share_input(1, xa), ctx.share_input(2, xb)
    gz = ctx.mult(3, ga, gb, n)
    oa, ob = OP.share_input(sess, xa, 1), OP.share_input(sess, xb, 2)
    oz = OP.mult(sess, oa, ob, 3)
    assert_shared_equal(gpu_shared(mpc, gz, (n,)), oz, "mult")
    rc, tr = ctx.verify_mult(4, ga, gb, gz, n, 3, trace=True)
    otr = []
    ok = OV.mult_verify(sess, oa, ob, oz, 4, trace=otr)
    assert ok and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [mpc.default_R(n)])
    assert_ledger(mpc, ctx, sess)
    z = ctx.reconstruct(gz, n)
    assert np.array_equal(z, OP.reconstruct(sess, oz))
    assert np.array_equal(z, xa * xb)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("M,N,K,t", [(64, 64, 128, 13), (37, 53, 29, 13), (129, 7, 300, 16),
                                     (5, 130, 9, -1), (300, 200, 333, 13)])
def test_matmul_matches_oracle(mpc, M, N, K, t, path):
    seed = seed_of(f"matmul-{M}-{N}-{K}")
    X, W = workloads.gemm_shape(M, N, K)
    if t >= 0:
        g = workloads.rng(f"fx-{M}-{N}-{K}")
        X = OP.encode_fixed(g.uniform(-4, 4, (M, K)), 13)
        W = OP.encode_fixed(g.uniform(-4, 4, (K, N)), 13)
    ctx = mpc.Context(seed, gemm_path=path)
    sess = Session(seed)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, t)
    ctx.sync()
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=t if t >= 0 else None)
    assert_shared_equal(gpu_shared(mpc, zpre, (M, N)), res.z_pre, "zpre")
    if t >= 0:
        assert_shared_equal(gpu_shared(mpc, zout, (M, N)), res.out, "zout")
        pqh = mpc.to_u64(pq)[: 12 * M * N].reshape(2, 6, M * N)
        for c, f in enumerate(Shared.FIELDS):
            assert np.array_equal(pqh[0, c], getattr(res.tp.p, f).reshape(-1)), f"p.{f}"
            assert np.array_equal(pqh[1, c], getattr(res.tp.q, f).reshape(-1)), f"q.{f}"
    assert_ledger(mpc, ctx, sess)


@pytest.mark.parametrize("M,N,K,t,mode,path", [(8, 8, 16, 13, 0, 0), (12, 10, 37, 13, 0, 0),
                                               (3, 5, 70, 13, 1, 0), (16, 16, 64, -1, 0, 0),
                                               (12, 10, 37, 13, 0, 1), (70, 9, 130, 13, 0, 1)])
def test_matmul_verify_transcript_matches_oracle(mpc, M, N, K, t, mode, path):
    seed = seed_of(f"vmat-{M}-{N}-{K}-{t}-{mode}")
    g = workloads.rng(f"vmat-{M}-{N}-{K}")
    X = OP.encode_fixed(g.uniform(-4, 4, (M, K)), 13)
    W = OP.encode_fixed(g.uniform(-4, 4, (K, N)), 13)
    ctx = mpc.Context(seed, reduce_mode=mode, gemm_path=path)
    sess = Session(seed, reduce_mode="x" if mode == 0 else "zeta2")
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, t)
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=t if t >= 0 else None)
    rc, tr = ctx.verify_matmul(4, gx, gw, zpre, pq, M, N, K, t, 3, trace=True)
    otr = []
    ok = OV.matmul_verify(sess, ox, ow, res, 4, t if t >= 0 else None, trace=otr)
    assert ok and rc == mpc.MPC_OK
    Rs = [mpc.default_R(K)] + ([mpc.default_R(64 * M * N)] if t >= 0 else [])
    check_trace(mpc, tr, otr, Rs)
    assert_ledger(mpc, ctx, sess)
    out = ctx.reconstruct(zout, M * N)
    assert np.array_equal(out, OP.reconstruct(sess, res.out).reshape(-1))


@pytest.mark.parametrize("M,N,K", [(256, 192, 1000), (1, 1, 1), (130, 65, 64)])
def test_tc_gemm_full_range_words(mpc, M, N, K):
    """Limb-split tensor-core products on shares of full 64-bit range (every digit plane busy,
    carries through all eight balanced digits) agree with the u64 path and with the oracle."""
    seed = seed_of(f"tcw-{M}-{N}-{K}")
    X = workloads.uniform_words((M, K), f"tcw-x-{M}-{N}-{K}")
    W = workloads.uniform_words((K, N), f"tcw-w-{M}-{N}-{K}")
    outs = []
    for path in (0, 1):
        ctx = mpc.Context(seed, gemm_path=path)
        gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
        zpre, _, _ = ctx.matmul(3, gx, gw, M, N, K, -1)
        ctx.sync()
        outs.append(mpc.to_u64(zpre).copy())
    assert np.array_equal(outs[0], outs[1])
    sess = Session(seed)
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=None)
    assert_shared_equal(gpu_shared(mpc, zpre, (M, N)), res.z_pre, "zpre")


@pytest.mark.parametrize("M,N,K", [(300, 300, 16), (64, 1100, 8), (2048, 1024, 16)])
def test_tc_and_u64_paths_give_identical_verification(mpc, M, N, K):
    """At sizes whose trunc batch spans several e_hi blocks (E > 65536) and many row tiles, the
    tensor-core path (limb GEMMs, tensor-core folds and table products, the grouped products of
    the r^(2e) factor; at E = 2^21 also the tensor-core S_hi combination and split-K batch-0
    products) and the u64 CUDA-core path give the same products, the same verification
    transcript and the same opened output; both paths are pinned to the oracle on the smaller
    shapes above."""
    seed = seed_of(f"paths-{M}-{N}-{K}")
    g = workloads.rng(f"paths-{M}-{N}-{K}")
    X = OP.encode_fixed(g.uniform(-4, 4, (M, K)), 13)
    W = OP.encode_fixed(g.uniform(-4, 4, (K, N)), 13)
    res = []
    for path in (0, 1):
        ctx = mpc.Context(seed, gemm_path=path)
        gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
        zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, 13)
        rc, tr = ctx.verify_matmul(4, gx, gw, zpre, pq, M, N, K, 13, 3, trace=True)
        assert rc == mpc.MPC_OK
        out = ctx.reconstruct(zout, M * N)
        res.append((mpc.to_u64(zpre).copy(), mpc.to_u64(tr).copy(), out))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2])
    # the opened product is the plaintext product, truncated (one-LSB carry allowed)
    # |entries| < 2^15 and K <= 16, so the int64 product is exact
    sref = (X.view(np.int64) @ W.view(np.int64)) >> 13
    got = res[1][2].reshape(M, N).view(np.int64)
    assert np.all(np.abs(got - sref) <= 1)


@pytest.mark.parametrize("R_main,R_trunc", [(0, 0), (2, 3), (7, 9)])
def test_matmul_verify_explicit_R(mpc, R_main, R_trunc):
    M, N, K, t = 6, 4, 20, 13
    seed = seed_of(f"vR-{R_main}-{R_trunc}")
    X, W = workloads.gemm_shape(M, N, K, "vR")
    ctx = mpc.Context(seed)
    sess = Session(seed)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, t)
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=t)
    rc, tr = ctx.verify_matmul(4, gx, gw, zpre, pq, M, N, K, t, 3, R_main, R_trunc, trace=True)
    otr = []
    ok = OV.matmul_verify(sess, ox, ow, res, 4, t, R_main, R_trunc, trace=otr)
    assert ok and rc == mpc.MPC_OK
    check_trace(mpc, tr, otr, [R_main, R_trunc])


@pytest.mark.parametrize("site,mask", [("GAMMA2", 1), ("MZ1", 1), ("MZ2", 1 << 40),
                                       ("HIGH_BIT", 0), ("MX_COPY_P1", 3), ("REC_MSG", 1)])
def test_faults_rejected_like_oracle(mpc, site, mask):
    M, N, K, t = 8, 6, 24, 13
    seed = seed_of(f"fault-{site}")
    X, W = workloads.gemm_shape(M, N, K, "fault")
    ctx = mpc.Context(seed)
    sess = Session(seed)
    ctx.inject_fault(site, 5, mask)
    sess.arm_fault(site, 5, mask)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, t)
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=t)
    rc, _ = ctx.verify_matmul(4, gx, gw, zpre, pq, M, N, K, t, 3)
    try:
        ook = OV.matmul_verify(sess, ox, ow, res, 4, t)
        oabort = False
    except OP.Abort:
        ook, oabort = False, True
    if site == "REC_MSG":
        # the armed Pi_Rec fault fires at the first reveal inside the verification
        assert rc == mpc.MPC_ERR_ABORT and oabort
    else:
        assert rc in (mpc.MPC_ERR_VERIFY, mpc.MPC_ERR_ABORT)
        assert not ook
        assert (rc == mpc.MPC_ERR_ABORT) == oabort
    assert ctx.status() == mpc.MPC_ERR_ABORT          # security with abort: sticky


def test_reconstruct_refused_before_verify_and_abort_on_bad_message(mpc):
    seed = seed_of("rec")
    x = workloads.uniform_words(300, "rec")
    ctx = mpc.Context(seed)
    gx = ctx.share_input(1, x)
    gz = ctx.mult(2, gx, gx, 300)
    with pytest.raises(mpc.MpcError) as ei:
        ctx.reconstruct(gz, 300)
    assert ei.value.code == mpc.MPC_ERR_PENDING
    rc, _ = ctx.verify_mult(3, gx, gx, gz, 300, 2)
    assert rc == mpc.MPC_OK
    assert np.array_equal(ctx.reconstruct(gz, 300), x * x)
    ctx.inject_fault("REC_MSG", 17, 1 << 5)
    with pytest.raises(mpc.MpcError) as ei:
        ctx.reconstruct(gx, 300)
    assert ei.value.code == mpc.MPC_ERR_ABORT


def test_large_reconstruct_multileaf_hash(mpc):
    """Pi_Rec over several 64 KiB hash leaves plus a ragged tail; device output."""
    seed = seed_of("rec-big")
    n = 3 * 8192 + 123
    x = workloads.uniform_words(n, "rec-big")
    ctx = mpc.Context(seed)
    gx = ctx.share_input(1, x)
    out = ctx.reconstruct(gx, n, to_host=False)
    assert np.array_equal(mpc.to_u64(out)[:n], x)
