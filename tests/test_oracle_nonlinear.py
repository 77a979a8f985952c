"""Pins of the non-linear oracle (Sec. 4.3): Boolean sharings and AND gates over Z_2, daBits,
edaBits, MSB extraction by the carry circuit, B2A, ReLU, 2x2 max-pool and the verification of a
non-linear layer (arithmetic products over GR(2^64, 64), AND gates over GF(2^64)).  Every value
is checked against plain integer arithmetic on the reconstructed plaintexts."""
import numpy as np
import pytest

from oracle import nonlinear as NL
from oracle import protocols as OP
from oracle.boolean import BoolSession, pack_bits, unpack_bits
from oracle.shares import Session

U64 = np.uint64
SEED = bytes(range(32))


def sessions(seed=SEED):
    return Session(seed), BoolSession(seed)


def signed(a):
    return np.asarray(a, dtype=U64).view(np.int64)


def test_pack_roundtrip_and_stream_convention():
    g = np.random.default_rng(1)
    b = g.integers(0, 2, 200).astype(U64)
    assert np.array_equal(unpack_bits(pack_bits(b), 200), b)
    # bit i of a Boolean stream is bit i % 64 of word i // 64
    _, bs = sessions()
    from oracle.chacha import prf_u64
    from oracle.shares import C_R1, P_AND, _COMP_PAIR, tag
    words = prf_u64(bs.keys[_COMP_PAIR[C_R1]], tag(P_AND, C_R1), 5, 0, 3)
    bits = bs.prf(C_R1, P_AND, 5, 150, start=20)
    ref = ((words[(np.arange(20, 170)) // 64] >> (np.arange(20, 170) % 64).astype(U64)) & U64(1))
    assert np.array_equal(bits, ref)


def test_boolean_share_and_gate_and_ledger():
    _, bs = sessions()
    g = np.random.default_rng(2)
    x = g.integers(0, 2, 130).astype(U64)
    y = g.integers(0, 2, 130).astype(U64)
    sx, sy = OP.share_input(bs, x, 1), OP.share_input(bs, y, 2)
    assert np.array_equal(OP.reconstruct(bs, sx), x)
    bs.ledger.clear()
    z = OP.mult(bs, sx, sy, 3)
    assert np.array_equal(OP.reconstruct(bs, z), x & y)
    # Table 1 at l = 1: one bit offline (Gamma), two online (m_z exchange) per AND, in words
    assert bs.ledger_bytes("offline", "mult") == 8 * 3
    assert bs.ledger_bytes("online", "mult") == 2 * 8 * 3


def test_dabits_are_consistent_bits():
    s, bs = sessions()
    ra, rb, triples = NL.dabits(s, bs, 7, 0, 128)
    a = OP.reconstruct(s, ra)
    b = OP.reconstruct(bs, rb)
    assert set(np.unique(a)) <= {0, 1}
    assert np.array_equal(a, b)
    for X, Y, Z in triples:
        assert np.array_equal(OP.reconstruct(s, Z), OP.reconstruct(s, X) * OP.reconstruct(s, Y))


def test_edabits_arithmetic_value_is_the_bit_composition():
    s, bs = sessions()
    ra, rbits, mults, inner = NL.edabits(s, bs, 9, 0, 64)
    r = OP.reconstruct(s, ra)
    bits = OP.reconstruct(bs, rbits)                  # (64, 64): plane i, element e
    comp = np.zeros(64, dtype=object)
    for i in range(64):
        comp += bits[i].astype(object) << i
    assert [int(v) for v in r] == [int(v) % 2 ** 64 for v in comp]


EDGE = [0, 1, 2 ** 63 - 1, 2 ** 63, 2 ** 64 - 1, 2 ** 62, 2 ** 63 + 1, 12345, 2 ** 64 - 12345]


def test_msb_by_carry_circuit_edge_and_random():
    s, bs = sessions()
    g = np.random.default_rng(3)
    vals = np.array(EDGE + [int(v) for v in g.integers(0, 2 ** 63, 64 - len(EDGE), dtype=np.uint64)
                            * np.uint64(2) + g.integers(0, 2, 64 - len(EDGE)).astype(U64)],
                    dtype=U64)
    x = OP.share_input(s, vals, 11)
    ra, rbits, _, _ = NL.edabits(s, bs, 12, 0, 64)
    m, delta, triples = NL.msb(s, bs, x, (ra, rbits), 12, 0)
    assert np.array_equal(OP.reconstruct(bs, m), vals >> U64(63))
    # every AND gate of the circuit is a correct triple, and the circuit has 6 levels
    assert len(triples) == 6
    for X, Y, Z in triples:
        assert np.array_equal(OP.reconstruct(bs, Z), OP.reconstruct(bs, X) & OP.reconstruct(bs, Y))


def test_carry_root_equals_integer_adder_carry():
    """Delta + r computed with integers: the carry into bit 63 is bit 63 of
    (Delta mod 2^63) + (r mod 2^63); the circuit's output is msb = Delta_63 ^ r_63 ^ carry."""
    g = np.random.default_rng(4)
    for _ in range(200):
        d, r = int(g.integers(0, 2 ** 63)) * 2 + int(g.integers(2)), int(g.integers(0, 2 ** 63)) * 2
        carry = (((d % 2 ** 63) + (r % 2 ** 63)) >> 63) & 1
        assert ((d + r) % 2 ** 64) >> 63 == (d >> 63) ^ (r >> 63) ^ carry


def test_b2a_preserves_value():
    s, bs = sessions()
    g = np.random.default_rng(5)
    b = g.integers(0, 2, 64).astype(U64)
    sb = OP.share_input(bs, b, 13)
    ra, rb, _ = NL.dabits(s, bs, 14, 0, 64)
    a = NL.b2a(s, bs, sb, (ra, rb), 14)
    assert np.array_equal(OP.reconstruct(s, a), b)


def test_relu_exact_on_signed_values():
    s, bs = sessions()
    g = np.random.default_rng(6)
    vals = np.concatenate([np.array([0, 1, -1, 2 ** 62, -2 ** 62, 2 ** 63 - 1, -2 ** 63],
                                    dtype=np.int64), g.integers(-2 ** 40, 2 ** 40, 57)]).view(U64)
    x = OP.share_input(s, vals, 21)
    out, triples = NL.relu(s, bs, x, 22)
    got = signed(OP.reconstruct(s, out))
    assert np.array_equal(got, np.maximum(signed(vals), 0))
    assert NL.verify_layer(s, bs, triples, 23)


def test_maxpool2_matches_window_max():
    s, bs = sessions()
    g = np.random.default_rng(7)
    shape = (1, 2, 4, 6)
    vals = g.integers(-2 ** 30, 2 ** 30, int(np.prod(shape))).view(U64)
    x = OP.share_input(s, vals, 31)
    out, triples = NL.maxpool2(s, bs, x, shape, 32)
    v = signed(vals).reshape(shape)
    ref = np.maximum(np.maximum(v[:, :, 0::2, 0::2], v[:, :, 0::2, 1::2]),
                     np.maximum(v[:, :, 1::2, 0::2], v[:, :, 1::2, 1::2]))
    assert np.array_equal(signed(OP.reconstruct(s, out)), ref.reshape(-1))
    assert NL.verify_layer(s, bs, triples, 33)


@pytest.mark.parametrize("where", ["and", "mult"])
def test_layer_verification_rejects_a_corrupted_message(where):
    s, bs = sessions()
    g = np.random.default_rng(8)
    vals = g.integers(-2 ** 40, 2 ** 40, 64).view(U64)
    x = OP.share_input(s, vals, 41)
    (bs if where == "and" else s).arm_fault("GAMMA2", 5, 1)
    out, triples = NL.relu(s, bs, x, 42)
    assert not NL.verify_layer(s, bs, triples, 43)


def test_layer_verification_catches_a_wrong_product_in_each_batch():
    """Reading N9 keeps every product under a check: a product triple made wrong after the fact
    (one share word of z, in the general batch 0 or in the edaBit bit batch 3) is rejected, and
    the untouched layer is accepted by the same call."""
    import copy
    s, bs = sessions(bytes(range(1, 33)))
    vals = np.random.default_rng(9).integers(-2 ** 40, 2 ** 40, 64).view(U64)
    x = OP.share_input(s, vals, 51)
    _, triples = NL.relu(s, bs, x, 52)
    assert len(triples[0]["mults"]) == 3 and len(triples[0]["eda"]) == 1
    assert triples[0]["eda"][0][2].p1_m.shape == (64, 64)
    assert NL.verify_layer(s, bs, triples, 53)
    for batch, comp in (("mults", "p1_m"), ("eda", "p0_r1")):
        bad = copy.deepcopy(triples)
        getattr(bad[0][batch][-1][2], comp).reshape(-1)[7] ^= U64(1 << 20)
        assert not NL.verify_layer(s, bs, bad, 53), (batch, comp)


def test_edabit_bit_batch_has_the_truncation_pairs_form():
    """The x side of batch 3 holds only [r]_1 (components p0_r1, p1_r1), the y side only [r]_2
    (p0_r2, p2_r2): the form whose party sums reduce to P0's single Gram."""
    s, bs = sessions()
    vals = np.random.default_rng(10).integers(-2 ** 40, 2 ** 40, 64).view(U64)
    _, triples = NL.relu(s, bs, OP.share_input(s, vals, 61), 62)
    X, Y, _ = triples[0]["eda"][0]
    for f in ("p0_r2", "p1_m", "p2_m", "p2_r2"):
        assert not getattr(X, f).any(), f
    for f in ("p0_r1", "p1_m", "p1_r1", "p2_m"):
        assert not getattr(Y, f).any(), f
    assert np.array_equal(X.p0_r1, X.p1_r1) and np.array_equal(Y.p0_r2, Y.p2_r2)


def _weighted_error(gr, r, errs):
    """sum_j r^j err_j in GR(2^64, 64) for ring scalars err_j, with r^j by repeated products and
    the scalar products coefficient by coefficient in Python integers."""
    acc = [0] * gr.d
    p = gr.const(1)
    for e in errs:
        e = int(e) % (1 << 64)
        for c in range(gr.d):
            acc[c] = (acc[c] + e * int(p[c])) % (1 << 64)
        p = gr.mul(p, r)
    return np.array(acc, dtype=U64)


def _relation(gr, xs, ys, zs):
    x, y, z = xs.open(gr.mask), ys.open(gr.mask), zs.open(gr.mask)
    return gr.sub(gr.inner(x, y), z)


@pytest.mark.parametrize("bad", [(), (3,), (0, 6)])
def test_multiplication_transform_is_the_weighted_product_error(bad):
    """Fig. MTP as batches 0, 2 and 3 use it: after the transform the claim's relation error
    sum_j x'_j y_j - z' equals sum_j r^j (x_j y_j - z_j), the per-gate errors of the opened
    triples weighted by the powers of r in gate order (zero for honest triples)."""
    from oracle.verify import challenge_r, tran_mult
    s = Session(bytes(range(2, 34)))
    gr = s.gr
    g = np.random.default_rng(12)
    x = g.integers(0, 2 ** 64, 7, dtype=U64)
    y = g.integers(0, 2 ** 64, 7, dtype=U64)
    z = np.array([(int(a) * int(b)) % (1 << 64) for a, b in zip(x, y)], dtype=U64)
    for j in bad:
        z[j] ^= U64(1 << (13 + j))
    X, Y, Z = (OP.share_input(s, v, 70 + k) for k, v in enumerate((x, y, z)))
    r = challenge_r(s, 73, 0)
    errs = [(int(a) * int(b) - int(c)) % (1 << 64) for a, b, c in zip(x, y, z)]
    assert np.array_equal(_relation(gr, *tran_mult(s, X, Y, Z, r)), _weighted_error(gr, r, errs))
    assert _relation(gr, *tran_mult(s, X, Y, Z, r)).any() == bool(bad)


@pytest.mark.parametrize("bad", [(), (1,), (0, 4)])
def test_row_transform_is_the_weighted_inner_product_error(bad):
    """Fig. PBDP as the edaBit inner-product batch (batch 1) uses it: n inner products of
    dimension k, row e weighted by r^e; the relation error equals
    sum_e r^e (sum_i X_ei Y_ei - Z_e) with Python integers."""
    s = Session(bytes(range(3, 35)))
    gr = s.gr
    g = np.random.default_rng(13)
    n, k = 5, 4
    Xv = g.integers(0, 2 ** 64, (n, k), dtype=U64)
    Yv = g.integers(0, 2 ** 64, (n, k), dtype=U64)
    Zv = np.array([sum(int(a) * int(b) for a, b in zip(Xv[e], Yv[e])) % (1 << 64)
                   for e in range(n)], dtype=U64)
    for e in bad:
        Zv[e] += U64(1 << (20 + e))
    X, Y, Z = (OP.share_input(s, v, 80 + q) for q, v in enumerate((Xv, Yv, Zv)))
    from oracle.verify import challenge_r
    r = challenge_r(s, 83, 1)
    errs = [(sum(int(a) * int(b) for a, b in zip(Xv[e], Yv[e])) - int(Zv[e])) % (1 << 64)
            for e in range(n)]
    rel = _relation(gr, *NL.tran_rows(s, X, Y, Z, r))
    assert np.array_equal(rel, _weighted_error(gr, r, errs))
    assert rel.any() == bool(bad)
