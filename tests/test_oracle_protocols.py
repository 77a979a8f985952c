"""Pins for oracle.protocols: reconstruction against plaintext, Table 1 byte counts, truncation
error model (Sec. 4.2) and abort on inconsistent Pi_Rec messages -- no GPU."""
import hashlib

import numpy as np
import pytest

from oracle.protocols import (Abort, asr, decode_fixed, encode_fixed, matmul, mult, reconstruct,
                              share_input, trunc_coeffs)
from oracle.shares import OFFLINE, ONLINE, Session

U64 = np.uint64
SEED = hashlib.sha256(b"mpc3-oracle-tests").digest()


def _rng(i=0):
    return np.random.default_rng(1000 + i)


def test_fixed_point_encoding_sec2():
    # Sec. 2: x >= 0 -> floor(x 2^k); x < 0 -> 2^l + floor(x 2^k)
    assert int(encode_fixed(1.5, 13)) == 3 * (1 << 12)
    assert int(encode_fixed(-1.0, 13)) == (1 << 64) - (1 << 13)
    assert int(encode_fixed(-1e-9, 13)) == (1 << 64) - 1
    v = _rng().uniform(-4, 4, 100)
    assert np.all(np.abs(decode_fixed(encode_fixed(v, 13), 13) - v) <= 2.0 ** -13)


def test_share_and_reconstruct_roundtrip():
    s = Session(SEED)
    x = _rng(1).integers(0, 2**64, 257, dtype=U64)
    X = share_input(s, x, 1)
    assert np.array_equal(reconstruct(s, X), x)
    # the masks are fresh PRG output: m differs from x
    assert not np.array_equal(X.p1_m, x)


def test_mult_reconstructs_product_mod_2_64():
    s = Session(SEED)
    rng = _rng(2)
    x = rng.integers(0, 2**64, 300, dtype=U64)
    y = rng.integers(0, 2**64, 300, dtype=U64)
    Z = mult(s, share_input(s, x, 1), share_input(s, y, 2), 3)
    z = reconstruct(s, Z)
    ref = [(int(a) * int(b)) % (1 << 64) for a, b in zip(x, y)]
    assert [int(v) for v in z] == ref


def test_matmul_reconstructs_product_python_ints():
    s = Session(SEED)
    rng = _rng(3)
    M, K, N = 5, 7, 3
    A = rng.integers(0, 2**64, (M, K), dtype=U64)
    B = rng.integers(0, 2**64, (K, N), dtype=U64)
    res = matmul(s, share_input(s, A, 1), share_input(s, B, 2), 3)
    z = reconstruct(s, res.out)
    for a in range(M):
        for b in range(N):
            ref = sum(int(A[a, k]) * int(B[k, b]) for k in range(K)) % (1 << 64)
            assert int(z[a, b]) == ref


def test_trunc_coefficients_reproduce_arithmetic_shift():
    rng = _rng(4)
    for t in (0, 1, 13, 16, 63):
        c, cp = trunc_coeffs(t)
        b1 = rng.integers(0, 2**64, 50, dtype=U64)
        b2 = rng.integers(0, 2**64, 50, dtype=U64)
        bits = (b1[:, None] >> np.arange(64, dtype=U64)) & (b2[:, None] >> np.arange(64, dtype=U64)) & U64(1)
        rx = b1 + b2 + np.sum(bits * c, axis=1, dtype=U64)
        rz = asr(b1, t) + asr(b2, t) + np.sum(bits * cp, axis=1, dtype=U64)
        assert np.array_equal(rx, b1 ^ b2)
        assert np.array_equal(rz, asr(b1 ^ b2, t))


def test_trunc_error_model_sec4_2():
    """Sec. 4.2: the truncated result is off by at most one in the last bit (carry), and wrong with
    probability about 2^(l_x - l + 1) (wrap)."""
    s = Session(SEED)
    rng = _rng(5)
    M, K, N = 16, 32, 16
    A = encode_fixed(rng.uniform(-4, 4, (M, K)), 13)
    B = encode_fixed(rng.uniform(-4, 4, (K, N)), 13)
    res = matmul(s, share_input(s, A, 1), share_input(s, B, 2), 3, trunc_bits=13)
    zpre = reconstruct(s, res.z_pre)
    assert np.array_equal(zpre, A @ B)
    out = reconstruct(s, res.out)
    diff = out.astype(np.int64) - asr(A @ B, 13).astype(np.int64)
    assert set(np.unique(diff)) <= {0, 1}
    # the pair itself: r_z = r_x >>_arith t
    tp = res.tp
    rx = (tp.rx1_p0 + tp.rx2_p0)
    rz = (tp.rz1_p0 + tp.rz2_p0)
    assert np.array_equal(rx, tp.b1 ^ tp.b2)
    assert np.array_equal(rz, asr(rx, 13))


def test_trunc_wrap_probability():
    """With |x| < 2^(l_x) the wrap of m = x + r_x happens with probability about 2^(l_x - l + 1)."""
    s = Session(SEED)
    rng = _rng(6)
    n = 20000
    lx = 60
    x = rng.integers(-(2**(lx - 1)), 2**(lx - 1), n).astype(np.int64).astype(U64)
    X = share_input(s, x.reshape(n, 1), 1)
    ONE = share_input(s, np.ones((1, 1), dtype=U64), 2)
    res = matmul(s, X, ONE, 3, trunc_bits=13)
    out = reconstruct(s, res.out).reshape(-1).astype(np.int64)
    diff = out - asr(x, 13).astype(np.int64)
    wrong = np.count_nonzero((diff != 0) & (diff != 1))
    # m = x + r wraps (as a signed value) with probability |x| / 2^l for uniform r
    p = np.abs(x.astype(np.int64)).astype(np.float64) / 2.0 ** 64
    mean, sd = p.sum(), np.sqrt((p * (1 - p)).sum())
    assert abs(wrong - mean) <= 5 * sd + 1
    assert wrong <= n * 2.0 ** (lx - 64 + 1)   # Sec. 4.2 bound 2^(l_x - l + 1)


def _per_elem(s, phase, proto, count):
    return s.ledger_bytes(phase, proto) / (8 * count)


def test_ledger_matches_table1(golden):
    import os
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_comm.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            op, off, on = line.split()
            rows[op] = (int(off), int(on))
    rng = _rng(7)
    # mult
    s = Session(SEED)
    x = rng.integers(0, 2**64, 64, dtype=U64)
    X, Y = share_input(s, x, 1), share_input(s, x, 2)
    assert _per_elem(s, ONLINE, "share", 128) == rows["share"][1]
    mult(s, X, Y, 3)
    assert (_per_elem(s, OFFLINE, "mult", 64), _per_elem(s, ONLINE, "mult", 64)) == rows["mult"]
    # inner product (matrix product, n = K independent)
    for K in (1, 9):
        s = Session(SEED)
        A = share_input(s, rng.integers(0, 2**64, (3, K), dtype=U64), 1)
        B = share_input(s, rng.integers(0, 2**64, (K, 4), dtype=U64), 2)
        matmul(s, A, B, 3)
        assert (_per_elem(s, OFFLINE, "inner", 12), _per_elem(s, ONLINE, "inner", 12)) == rows["inner"]
        s.ledger.clear()
        matmul(s, A, B, 4, trunc_bits=13)
        off = _per_elem(s, OFFLINE, "inner", 12) + _per_elem(s, OFFLINE, "trunc", 12)
        on = _per_elem(s, ONLINE, "inner", 12) + _per_elem(s, ONLINE, "trunc", 12)
        assert (off, on) == rows["inner_trunc"]
        assert (_per_elem(s, OFFLINE, "trunc", 12), _per_elem(s, ONLINE, "trunc", 12)) == rows["trunc"]


def test_rec_aborts_on_inconsistent_message():
    s = Session(SEED)
    X = share_input(s, np.arange(10, dtype=U64), 1)
    s.arm_fault("REC_MSG", 3, 1)
    with pytest.raises(Abort):
        reconstruct(s, X)


def test_inconsistent_replica_aborts_at_reconstruction():
    s = Session(SEED)
    s.arm_fault("MX_COPY_P1", 2, 1 << 40)
    X = share_input(s, np.arange(10, dtype=U64), 1)
    with pytest.raises(Abort):
        reconstruct(s, X)


@pytest.mark.parametrize("owner", [0, 1, 2])
def test_input_owner_k_sharing(owner):
    """Pi_<.>^{l,k} (Sec. 2): any party P_k can own an input.  The sharing reconstructs to x and,
    with P_k holding both seeds of the mask, equals P0's sharing of the same call component for
    component; P0 sends m_x twice (to P1 and P2, 2 l bits per element), P1 or P2 once (to the
    other one, l bits), and a product of inputs owned by different parties verifies."""
    from oracle.verify import mult_verify
    rng = _rng(20 + owner)
    x = rng.integers(0, 2**64, 50, dtype=U64)
    y = rng.integers(0, 2**64, 50, dtype=U64)
    s = Session(SEED)
    X = share_input(s, x, 5, owner=owner)
    msgs = [(e.src, e.dst, e.nbytes) for e in s.ledger]
    want = {0: [(0, 1, 400), (0, 2, 400)], 1: [(1, 2, 400)], 2: [(2, 1, 400)]}[owner]
    assert msgs == want
    assert np.array_equal(reconstruct(s, X), x)
    X0 = share_input(Session(SEED), x, 5, owner=0)
    for a, b in zip(X.as_tuple(), X0.as_tuple()):
        assert np.array_equal(a, b)
    Y = share_input(s, y, 6, owner=(owner + 1) % 3)
    Z = mult(s, X, Y, 7)
    assert mult_verify(s, X, Y, Z, 8)
    assert np.array_equal(reconstruct(s, Z), x * y)


def test_owner_two_message_to_p1_inconsistent_aborts():
    s = Session(SEED)
    s.arm_fault("MX_COPY_P1", 4, 1 << 3)
    X = share_input(s, np.arange(10, dtype=U64), 1, owner=2)
    with pytest.raises(Abort):
        reconstruct(s, X)


def test_input_owner_out_of_range_rejected():
    with pytest.raises(ValueError):
        share_input(Session(SEED), np.arange(3, dtype=U64), 1, owner=3)


# ---------------------------------------------------------------------------------------------
# reading D1 (fixed point out of range), standalone Pi_Trunc (reading T5), convolution lowering
# ---------------------------------------------------------------------------------------------
def test_encode_fixed_saturates_and_maps_nan_to_zero():
    k = 13
    big = np.array([2.0 ** 60, -(2.0 ** 60), np.inf, -np.inf, np.nan, 2.0 ** 50 - 1.0])
    v = encode_fixed(big, k).astype(np.int64)
    assert v[0] == np.iinfo(np.int64).max and v[2] == np.iinfo(np.int64).max
    assert v[1] == np.iinfo(np.int64).min and v[3] == np.iinfo(np.int64).min
    assert v[4] == 0
    assert v[5] == (2 ** 50 - 1) * 2 ** 13        # in range: exact
    # the boundary: x 2^k = -2^63 is representable, 2^63 is not
    edge = encode_fixed(np.array([-(2.0 ** 50), 2.0 ** 50]), k).astype(np.int64)
    assert edge[0] == np.iinfo(np.int64).min and edge[1] == np.iinfo(np.int64).max


def test_standalone_trunc_opens_the_shifted_value_and_counts_its_messages():
    from oracle.protocols import trunc
    from oracle.verify import trunc_verify
    s = Session(SEED)
    rng = np.random.default_rng(21)
    x = encode_fixed(rng.uniform(-1000, 1000, 300), 26)      # |x| < 2^36: no wrap expected
    X = share_input(s, x, 1)
    s.ledger.clear()
    Z, tp = trunc(s, X, 2, 13)
    got = reconstruct(s, Z).astype(np.int64)
    want = x.astype(np.int64) >> 13
    assert np.all((got - want == 0) | (got - want == 1))
    assert np.any(got - want == 1) and np.any(got == want)   # both carries occur
    off = s.ledger_bytes(OFFLINE, "trunc")
    on = s.ledger_bytes(ONLINE, "trunc")
    assert off == 6 * 8 * 300                                 # Table 1 / Sec. 4.2: 6 l offline
    assert on == 2 * 8 * 300 + 2 * 32                         # mask switch: 2 l + two hashes
    assert all(trunc_verify(s, tp, 2, 13))


def test_standalone_trunc_rejects_a_corrupted_mask_switch():
    from oracle.protocols import trunc
    s = Session(SEED)
    X = share_input(s, encode_fixed(np.linspace(-3, 3, 40), 26), 1)
    s.arm_fault("TRUNC_D1", 7, 1 << 20)
    with pytest.raises(Abort):
        trunc(s, X, 2, 13)


def _conv_by_definition(x, w, stride, pad):
    """out[b, o, i, j] = sum_{c, di, dj} x[b, c, i s + di - p, j s + dj - p] w[o, c, di, dj]
    mod 2^64, with Python integers, over a zero-padded copy made with numpy.pad."""
    B, C, H, W = x.shape
    O, _, kh, kw = w.shape
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    Ho, Wo = (H + 2 * pad - kh) // stride + 1, (W + 2 * pad - kw) // stride + 1
    out = np.zeros((B, O, Ho, Wo), dtype=np.uint64)
    for b in range(B):
        for o in range(O):
            for i in range(Ho):
                for j in range(Wo):
                    win = xp[b, :, i * stride:i * stride + kh, j * stride:j * stride + kw]
                    acc = sum(int(a) * int(c) for a, c in zip(win.reshape(-1), w[o].reshape(-1)))
                    out[b, o, i, j] = acc % (1 << 64)
    return out


@pytest.mark.parametrize("geom", [(2, 3, 6, 5, 3, 3, 1, 0), (1, 2, 7, 7, 3, 2, 2, 1),
                                  (2, 1, 5, 5, 5, 5, 1, 2)])
def test_conv2d_opens_the_convolution(geom):
    from oracle.protocols import conv2d, conv_out_size
    B, C, H, W, kh, kw, stride, pad = geom
    O = 4
    s = Session(SEED)
    rng = np.random.default_rng(22)
    x = rng.integers(0, 2**64, (B, C, H, W), dtype=np.uint64)
    w = rng.integers(0, 2**64, (O, C, kh, kw), dtype=np.uint64)
    wm = np.ascontiguousarray(w.reshape(O, -1).T)             # rows (c, di, dj)
    X, Wm = share_input(s, x, 1), share_input(s, wm, 2)
    cols, res = conv2d(s, X, Wm, 3, geom)
    Ho, Wo = conv_out_size(H, W, kh, kw, stride, pad)
    got = reconstruct(s, res.z_pre).reshape(B, Ho, Wo, O).transpose(0, 3, 1, 2)
    assert np.array_equal(got, _conv_by_definition(x, w, stride, pad))


# ---------------------------------------------------------------------------------------------
# truncation bits keyed by output row (reading A12): a row opens to the same truncated value in
# any batch
# ---------------------------------------------------------------------------------------------
def _row_key(req: int, layer: int, row: int) -> int:
    from oracle.shares import obj_id
    return obj_id(req * 64 + layer, (row >> 16) & 15, row & 0xFFFF)


def test_keyed_trunc_bits_are_the_rows_streams():
    from oracle.protocols import trunc_bit_words
    from oracle.shares import C_TB1, P_TRUNC_BITS
    s = Session(SEED)
    keys = [_row_key(7, 1, i) for i in range(3)]
    w = trunc_bit_words(s, C_TB1, 99, 3 * 5, keys, 5)
    for i, k in enumerate(keys):
        assert np.array_equal(w[5 * i:5 * i + 5], s.prf(C_TB1, P_TRUNC_BITS, k, 5))


def test_a_request_opens_the_same_truncated_rows_alone_and_packed():
    """Request A (2 rows) alone and packed behind request B (3 rows): with row-keyed truncation
    bits, A's opened truncated outputs are bit-identical; with call-keyed bits they differ in
    some carry."""
    rng = np.random.default_rng(31)
    K, N = 40, 6
    W = encode_fixed(rng.uniform(-1, 1, (K, N)), 13)
    XA = encode_fixed(rng.uniform(-1, 1, (2, K)), 13)
    XB = encode_fixed(rng.uniform(-1, 1, (3, K)), 13)
    keysA = [_row_key(1, 0, i) for i in range(2)]
    keysB = [_row_key(2, 0, i) for i in range(3)]

    def run(X, keys, call):
        s = Session(SEED)
        SX, SW = share_input(s, X, call), share_input(s, W, call + 1)
        res = matmul(s, SX, SW, call + 2, trunc_bits=13, row_keys=keys)
        return reconstruct(s, res.out)

    alone = run(XA, keysA, 10)
    packed = run(np.concatenate([XB, XA]), keysB + keysA, 20)
    assert np.array_equal(packed[3:], alone)
    unkeyed_alone = run(XA, None, 10)
    unkeyed_packed = run(np.concatenate([XB, XA]), None, 20)
    exact = (XA.astype(np.int64) @ W.astype(np.int64)) >> 13
    for out in (alone, unkeyed_alone, unkeyed_packed[3:]):
        assert np.all(np.abs(out.astype(np.int64) - exact) <= 1)
    assert not np.array_equal(unkeyed_packed[3:], unkeyed_alone)
