"""Non-linear layers on the GPU vs the oracle (Sec. 4.3), through the C-ABI: ReLU and 2x2
max-pool outputs bit-exact in every share component, the three verification transcripts of the
layer (daBit and final products, edaBit inner products and edaBit bit products over GR(2^64, 64),
AND gates over GF(2^64)),
the ledger (the arithmetic and the Boolean oracle sessions together), rejection of corrupted
messages, and plaintext correctness at a size the oracle does not reach."""
import hashlib

import numpy as np
import pytest

from oracle import nonlinear as NL
from oracle import protocols as OP
from oracle.boolean import BoolSession, gf_to_words
from oracle.shares import Session, Shared

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


def gpu_shared(M, t, n):
    a = M.to_u64(t)[: 6 * n].reshape(6, n)
    return Shared(*(a[i].copy() for i in range(6)))


def assert_shared_equal(g: Shared, o: Shared, what=""):
    for f in Shared.FIELDS:
        a, b = getattr(g, f).reshape(-1), getattr(o, f).reshape(-1)
        bad = np.flatnonzero(a != b)
        assert bad.size == 0, f"{what}.{f}: {bad.size} mismatches, first at {bad[:5]}"


def ledger_sum(*sessions):
    out = {}
    for s in sessions:
        for e in s.ledger:
            out[(e.phase, e.proto)] = out.get((e.phase, e.proto), 0) + e.nbytes
    return out


def check_gr_batch(M, g, off, otr, R):
    rounds = [t for t in otr if "round" in t]
    delta = [t["delta"] for t in otr if "delta" in t][0]
    assert len(rounds) == R
    for k, o in enumerate(rounds):
        base = off + k * M.TRACE_ROUND
        assert np.array_equal(g[base:base + 64], o["zeta_prime"]), f"round {k + 1} zeta'"
        h0 = g[base + 64: base + 448].reshape(6, 64)
        h2 = g[base + 448: base + 832].reshape(6, 64)
        for c, f in enumerate(Shared.FIELDS):
            assert np.array_equal(h0[c], getattr(o["h0"], f)), f"round {k + 1} h0.{f}"
            assert np.array_equal(h2[c], getattr(o["h2"], f)), f"round {k + 1} h2.{f}"
    assert np.array_equal(g[off + R * M.TRACE_ROUND: off + R * M.TRACE_ROUND + 64], delta)
    return off + (R + 1) * M.TRACE_ROUND


def check_gf_batch(M, g, off, otr, R):
    rounds = [t for t in otr if "round" in t]
    delta = [t["delta"] for t in otr if "delta" in t][0]
    assert len(rounds) == R
    for k, o in enumerate(rounds):
        base = off + k * M.TRACE_GF_ROUND
        assert g[base] == gf_to_words(o["zeta_prime"]), f"GF round {k + 1} zeta'"
        for c, f in enumerate(Shared.FIELDS):
            assert g[base + 1 + c] == gf_to_words(getattr(o["h0"], f)), f"GF round {k + 1} h0.{f}"
            assert g[base + 7 + c] == gf_to_words(getattr(o["h2"], f)), f"GF round {k + 1} h2.{f}"
    assert g[off + R * M.TRACE_GF_ROUND] == gf_to_words(delta)


def check_layer_trace(M, gtrace, otrace, nps):
    g = M.to_u64(gtrace)
    R0, R1, R2, R3 = M.Context.nonlinear_R(nps)
    off = check_gr_batch(M, g, 0, otrace["mult"], R0)
    off = check_gr_batch(M, g, off, otrace["inner"], R1)
    check_gf_batch(M, g, off, otrace["and"], R2)
    off += (R2 + 1) * M.TRACE_GF_ROUND
    check_gr_batch(M, g, off, otrace["eda"], R3)


def signed(a):
    return np.asarray(a, dtype=U64).view(np.int64)


def test_relu_matches_oracle(mpc):
    seed = seed_of("relu")
    g = np.random.default_rng(61)
    n = 100
    vals = np.concatenate([np.array([0, 1, -1, 2 ** 62, -2 ** 62, 2 ** 63 - 1, -2 ** 63],
                                    dtype=np.int64), g.integers(-2 ** 40, 2 ** 40, n - 7)]).view(U64)
    ctx = mpc.Context(seed)
    s, bs = Session(seed), BoolSession(seed)
    gx = ctx.share_input(1, vals)
    ox = OP.share_input(s, vals, 1)
    ctx.ledger_reset()
    s.ledger.clear()
    rc, out, tr = ctx.relu(2, 3, gx, n, trace=True)
    assert rc == mpc.MPC_OK
    oout, triples = NL.relu(s, bs, ox, 2)
    otr = {"mult": [], "inner": [], "and": [], "eda": []}
    assert NL.verify_layer(s, bs, triples, 3, trace=otr)
    assert_shared_equal(gpu_shared(mpc, out, n), oout, "relu out")
    check_layer_trace(mpc, tr, otr, [64 * ((n + 63) // 64)])
    gl, _ = ctx.ledger()
    ol = ledger_sum(s, bs)
    for key in set(gl) | set(ol):
        assert gl.get(key, 0) == ol.get(key, 0), (key, gl.get(key, 0), ol.get(key, 0))
    res = ctx.reconstruct(out, n)
    assert np.array_equal(signed(res), np.maximum(signed(vals), 0))


def test_maxpool2_matches_oracle(mpc):
    seed = seed_of("maxpool")
    shape = (1, 2, 4, 6)
    g = np.random.default_rng(62)
    vals = g.integers(-2 ** 30, 2 ** 30, int(np.prod(shape))).view(U64)
    ctx = mpc.Context(seed)
    s, bs = Session(seed), BoolSession(seed)
    gx = ctx.share_input(1, vals)
    ox = OP.share_input(s, vals, 1)
    rc, out, tr = ctx.maxpool2(2, 3, gx, shape, trace=True)
    assert rc == mpc.MPC_OK
    oout, triples = NL.maxpool2(s, bs, ox, shape, 2)
    otr = {"mult": [], "inner": [], "and": [], "eda": []}
    assert NL.verify_layer(s, bs, triples, 3, trace=otr)
    nw = int(np.prod(shape)) // 4
    assert_shared_equal(gpu_shared(mpc, out, nw), oout, "maxpool out")
    check_layer_trace(mpc, tr, otr, [64 * ((2 * nw + 63) // 64), 64 * ((nw + 63) // 64)])
    v = signed(vals).reshape(shape)
    ref = np.maximum(np.maximum(v[:, :, 0::2, 0::2], v[:, :, 0::2, 1::2]),
                     np.maximum(v[:, :, 1::2, 0::2], v[:, :, 1::2, 1::2]))
    assert np.array_equal(signed(ctx.reconstruct(out, nw)), ref.reshape(-1))


@pytest.mark.parametrize("site", ["AND_GAMMA2", "GAMMA2"])
def test_relu_rejects_corrupted_message(mpc, site):
    seed = seed_of(f"relu-fault-{site}")
    vals = np.random.default_rng(63).integers(-2 ** 40, 2 ** 40, 64).view(U64)
    ctx = mpc.Context(seed)
    gx = ctx.share_input(1, vals)
    ctx.inject_fault(site, 5, 1)
    rc, out, _ = ctx.relu(2, 3, gx, 64)
    assert rc == mpc.MPC_ERR_VERIFY
    # the oracle rejects the same corrupted run
    s, bs = Session(seed), BoolSession(seed)
    ox = OP.share_input(s, vals, 1)
    (bs if site == "AND_GAMMA2" else s).arm_fault("GAMMA2", 5, 1)
    _, triples = NL.relu(s, bs, ox, 2)
    assert not NL.verify_layer(s, bs, triples, 3)


@pytest.mark.parametrize("n", [16384, 1000])
def test_relu_large_plaintext(mpc, n):
    seed = seed_of(f"relu-large-{n}")
    vals = np.random.default_rng(64).integers(-2 ** 45, 2 ** 45, n).view(U64)
    ctx = mpc.Context(seed)
    gx = ctx.share_input(1, vals)
    rc, out, _ = ctx.relu(2, 3, gx, n)
    assert rc == mpc.MPC_OK
    assert np.array_equal(signed(ctx.reconstruct(out, n)), np.maximum(signed(vals), 0))
