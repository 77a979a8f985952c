"""Pins for oracle.verify: completeness, rejection of injected errors, brute-force soundness over
every challenge on tiny Galois rings (Lemma transl / polyred / polyvv), Lagrange identities,
literal-vs-consolidated agreement, and the weakness of the 2*zeta' reading -- no GPU."""
import hashlib
import itertools

import numpy as np
import pytest

from oracle.galois import GR, gr64
from oracle.protocols import Abort, encode_fixed, matmul, mult, share_input
from oracle.shares import P_VER_ALPHA, P_VER_ZETA, Session, obj_id
from oracle.verify import (bi_verify, challenge_r, inner_verify, lagrange, matmul_verify,
                           mult_verify, reduce_round, third_point, tran_matmul_literal,
                           tran_matmul_rank1, tran_trunc, tran_trunc_literal)

U64 = np.uint64
SEED = hashlib.sha256(b"mpc3-oracle-verify").digest()


def _all_elements(gr):
    q = 1 << gr.ell
    return np.array([[(v >> (gr.ell * c)) % q for c in range(gr.d)] for v in range(q ** gr.d)],
                    dtype=U64)


# ---------------------------------------------------------------------------------------------
# completeness and rejection at l = d = 64
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["x", "zeta2"])
def test_mult_verify_complete(mode):
    s = Session(SEED, reduce_mode=mode)
    rng = np.random.default_rng(1)
    x, y = (rng.integers(0, 2**64, 200, dtype=U64) for _ in range(2))
    X, Y = share_input(s, x, 1), share_input(s, y, 2)
    Z = mult(s, X, Y, 3)
    trace = []
    assert mult_verify(s, X, Y, Z, 4, trace=trace)
    assert not np.any(trace[-1]["delta"])
    assert len([t for t in trace if "round" in t]) == 2   # R = ceil(log2 200) - 6


@pytest.mark.parametrize("mode", ["x", "zeta2"])
def test_matmul_verify_complete_rank1_and_literal(mode):
    s = Session(SEED, reduce_mode=mode)
    rng = np.random.default_rng(2)
    A = encode_fixed(rng.uniform(-4, 4, (3, 4)), 13)
    B = encode_fixed(rng.uniform(-4, 4, (4, 2)), 13)
    SA, SB = share_input(s, A, 1), share_input(s, B, 2)
    res = matmul(s, SA, SB, 3, trunc_bits=13)
    assert matmul_verify(s, SA, SB, res, 4, 13)
    assert matmul_verify(s, SA, SB, res, 5, 13, literal=True)


@pytest.mark.parametrize("site,mask", [("GAMMA2", 1), ("MZ1", 1), ("MZ2", 1 << 17),
                                       ("HIGH_BIT", 0)])
def test_mult_verify_rejects_faults(site, mask):
    s = Session(SEED)
    rng = np.random.default_rng(3)
    x, y = (rng.integers(0, 2**64, 256, dtype=U64) for _ in range(2))
    X, Y = share_input(s, x, 1), share_input(s, y, 2)
    s.arm_fault(site, 77, mask)
    Z = mult(s, X, Y, 3)
    try:
        assert not mult_verify(s, X, Y, Z, 4, R=2)
    except Abort:
        pass


def _concat(parts):
    from oracle.shares import Shared
    return Shared(*(np.concatenate([getattr(p, f) for p in parts]) for f in Shared.FIELDS))


@pytest.mark.parametrize("fault_layer", [None, 0, 3, 5])
def test_deferred_mult_verify_over_a_chain(fault_layer):
    """A depth-6 chain z_(l+1) = z_l y_l of Pi_Mult gates checked once over all of its triples
    (every gate of the circuit in one batch, before any output is opened): an honest run accepts
    and opens the plaintext chain mod 2^64; an error in any one gate's message is rejected."""
    from oracle.protocols import reconstruct
    s = Session(SEED)
    rng = np.random.default_rng(11)
    n, D = 40, 6
    x = rng.integers(0, 2**64, n, dtype=U64)
    ys = [rng.integers(0, 2**64, n, dtype=U64) for _ in range(D)]
    Z = share_input(s, x, 1)
    trip = []
    for layer in range(D):
        Y = share_input(s, ys[layer], 10 + layer)
        if layer == fault_layer:
            s.arm_fault("MZ1", 7, 1 << 9)
        Zn = mult(s, Z, Y, 100 + layer)
        trip.append((Z, Y, Zn))
        Z = Zn
    batch = [_concat([t[i] for t in trip]) for i in range(3)]
    try:
        ok = mult_verify(s, *batch, 500)
    except Abort:
        ok = False
    if fault_layer is None:
        assert ok
        want = x.copy()
        for y in ys:
            want = want * y
        assert np.array_equal(reconstruct(s, Z), want)
    else:
        assert not ok


@pytest.mark.parametrize("site,mask", [("GAMMA2", 1), ("MZ1", 1), ("MZ2", 5), ("HIGH_BIT", 0)])
def test_matmul_verify_rejects_faults(site, mask):
    s = Session(SEED)
    rng = np.random.default_rng(4)
    A = rng.integers(0, 2**64, (4, 8), dtype=U64)
    B = rng.integers(0, 2**64, (8, 4), dtype=U64)
    SA, SB = share_input(s, A, 1), share_input(s, B, 2)
    s.arm_fault(site, 5, mask)
    res = matmul(s, SA, SB, 3, trunc_bits=13)
    try:
        assert not matmul_verify(s, SA, SB, res, 4, 13, R_main=2, R_trunc=4)
    except Abort:
        pass


def test_trunc_pair_fault_rejected_by_trunc_batch():
    """An error in P0's Gamma of a trunc-pair inner product is caught by batch 1."""
    s = Session(SEED)
    rng = np.random.default_rng(5)
    A = rng.integers(0, 2**64, (2, 3), dtype=U64)
    B = rng.integers(0, 2**64, (3, 2), dtype=U64)
    SA, SB = share_input(s, A, 1), share_input(s, B, 2)
    res = matmul(s, SA, SB, 3, trunc_bits=13)
    res.tp.q.p2_m[1] ^= U64(1 << 9)
    res.tp.q.p1_m[1] ^= U64(1 << 9)
    assert not matmul_verify(s, SA, SB, res, 4, 13)


def test_ring_attack_high_bit_many_seeds_mode_x():
    """e = 2^63 added to one product (Sec. 3 'Ring-Specific Challenges') is rejected every time."""
    for i in range(6):
        s = Session(hashlib.sha256(bytes([i])).digest())
        x = np.arange(1, 129, dtype=U64)
        X, Y = share_input(s, x, 1), share_input(s, x, 2)
        s.arm_fault("HIGH_BIT", i * 11, 0)
        Z = mult(s, X, Y, 3)
        assert not mult_verify(s, X, Y, Z, 4, R=1)


# ---------------------------------------------------------------------------------------------
# Lagrange weights
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["x", "zeta2"])
def test_lagrange_identities(mode):
    gr = gr64()
    rng = np.random.default_rng(6)
    zp = rng.integers(0, 2**64, 64, dtype=U64)
    zeta, L0, L1, L2 = lagrange(gr, zp, mode)
    assert np.array_equal(gr.add(gr.add(L0, L1), L2), gr.const(1))
    # h(zeta) for a random degree-2 polynomial over GR equals the interpolation
    a, b, c = (rng.integers(0, 2**64, 64, dtype=U64) for _ in range(3))
    h = lambda t: gr.add(gr.add(gr.mul(a, gr.mul(t, t)), gr.mul(b, t)), c)
    p2 = third_point(gr, mode)
    interp = gr.add(gr.add(gr.mul(L0, h(gr.const(0))), gr.mul(L1, h(gr.const(1)))), gr.mul(L2, h(p2)))
    assert np.array_equal(interp, h(zeta))


def test_lagrange_basis_at_nodes_mode_x():
    gr = gr64()
    nodes = [gr.const(0), gr.const(1), gr.x()]
    for j, node in enumerate(nodes):
        _, *Ls = lagrange(gr, node, "x")
        for i, L in enumerate(Ls):
            assert np.array_equal(L, gr.const(1 if i == j else 0))


# ---------------------------------------------------------------------------------------------
# brute force over every challenge on tiny Galois rings
# ---------------------------------------------------------------------------------------------
TINY = [(2, 2, (0, 1)), (3, 2, (0, 1)), (2, 3, (0, 1)), (1, 4, (0, 1))]


@pytest.mark.parametrize("ell,d,taps", TINY)
def test_bruteforce_lemma_polyred_mode_x(ell, d, taps):
    """Lemma polyred: for every z-error e != 0 and adversarial e1, e2 the error after one
    reduction, L0 e1 + L1 (e - e1) + L2 e2, vanishes for at most 2 / 2^d of all zeta."""
    gr = GR(ell, d, taps)
    el = _all_elements(gr)
    n = len(el)
    Ls = [lagrange(gr, z, "x")[1:] for z in el]
    L0 = np.stack([L[0] for L in Ls]); L1 = np.stack([L[1] for L in Ls]); L2 = np.stack([L[2] for L in Ls])
    rng = np.random.default_rng(7)
    errs = el[1:] if n <= 64 else el[rng.choice(np.arange(1, n), 40, replace=False)]
    adv = el if n <= 16 else el[rng.choice(n, 16, replace=False)]
    worst = 0.0
    for e in errs:
        for e1 in adv:
            base = gr.add(gr.mul(L0, e1), gr.mul(L1, gr.sub(e, e1)))       # (n, d)
            for e2 in adv:
                psi = gr.add(base, gr.mul(L2, e2))
                worst = max(worst, np.mean(~np.any(psi, axis=1)))
    assert worst <= 2.0 / 2 ** d + 1e-12


@pytest.mark.parametrize("ell,d,taps", [(2, 2, (0, 1)), (3, 2, (0, 1)), (3, 1, (0,))])
def test_zeta2_reading_accepts_errors_multiple_of_2_pow_l_minus_2(ell, d, taps):
    """Under the 2*zeta' reading L1 = 4 z'(1 - z') is always a multiple of 4, so an error
    e = 2^(l-2) in z survives one honest reduction for every zeta'.  The default reading (third
    point x) does not have this weakness (previous test)."""
    gr = GR(ell, d, taps)
    e = gr.const(1 << (ell - 2))
    survive = [not np.any(gr.mul(lagrange(gr, z, "zeta2")[2], e)) for z in _all_elements(gr)]
    assert all(survive)


@pytest.mark.parametrize("ell,d,taps", TINY)
def test_bruteforce_lemma_polyvv(ell, d, taps):
    """Lemma polyvv: for e != 0 and any e', alpha e + e' = 0 for at most 1/2^d of all alpha."""
    gr = GR(ell, d, taps)
    el = _all_elements(gr)
    worst = 0.0
    for e in el[1:]:
        prod = gr.mul(el, e)                                                 # alpha * e
        # the e' that is hit most often is the most frequent value of -alpha e
        _, counts = np.unique(prod, axis=0, return_counts=True)
        worst = max(worst, counts.max() / len(el))
    assert worst <= 1.0 / 2 ** d + 1e-12


@pytest.mark.parametrize("ell,d,taps", TINY)
def test_bruteforce_lemma_transl(ell, d, taps):
    """Lemma transl: a non-zero error vector (e_0..e_{G-1}) gives sum_i r^i e_i = 0 for at most
    (G - 1) / 2^d of all r."""
    gr = GR(ell, d, taps)
    el = _all_elements(gr)
    rng = np.random.default_rng(8)
    G = 3
    pw = np.stack([gr.powers(r, G) for r in el])                             # (n, G, d)
    worst = 0.0
    cands = [np.stack([gr.const(1 << (ell - 1)), gr.zeros(), gr.zeros()]),
             np.stack([gr.zeros(), gr.const(1 << (ell - 1)), gr.const(1 << (ell - 1))])]
    cands += [el[rng.integers(0, len(el), G)] for _ in range(30)]
    for ev in cands:
        if not np.any(ev):
            continue
        tot = gr.sum(gr.mul(pw, ev[None]), axis=1)
        worst = max(worst, np.mean(~np.any(tot, axis=1)))
    assert worst <= (G - 1) / 2 ** d + 1e-12


def test_plain_ring_check_passes_high_bit_error_half_the_time():
    """Sec. 3: with d = 1 (the plain ring Z_2^l) the error e = 2^(l-1) survives r^i e for every
    even r, i.e. with probability 1/2."""
    gr = GR(8, 1, (0,))
    el = _all_elements(gr)
    e = gr.const(1 << 7)
    passes = np.mean(~np.any(gr.mul(el, e), axis=1))
    assert passes == 0.5


@pytest.mark.parametrize("mode,ell,d,taps", [("x", 2, 2, (0, 1)), ("x", 3, 2, (0, 1))])
def test_protocol_level_reduce_then_verify_bruteforce(mode, ell, d, taps):
    """The full share-level Pi_Reduce + Pi_InnerVerify on a tiny ring, with zeta' forced to every
    ring element and alpha = 1: a claim with error e in z is accepted for at most 2/2^d of zeta'."""
    gr = GR(ell, d, taps)
    el = _all_elements(gr)
    rng = np.random.default_rng(9)
    x = el[rng.integers(0, len(el), 4)]
    y = el[rng.integers(0, len(el), 4)]
    for e in (gr.const(1), gr.const(1 << (ell - 1)), el[-1]):
        z = gr.add(gr.inner(x, y), e)
        accepted = 0
        for zp in el:
            s = Session(SEED, gr=gr, reduce_mode=mode)
            X = share_input(s, x, 1)
            Y = share_input(s, y, 2)
            Zs = share_input(s, z[None], 3)[0]
            s.forced[(P_VER_ZETA, obj_id(10, 0, 1))] = zp
            s.forced[(P_VER_ALPHA, obj_id(10, 0, 0))] = gr.const(1)
            if bi_verify(s, X, Y, Zs, 10, 0, R=1):
                accepted += 1
        assert accepted / len(el) <= 2.0 / 2 ** d + 1e-12


def test_honest_tiny_ring_accepts_every_challenge():
    gr = GR(2, 2, (0, 1))
    el = _all_elements(gr)
    x, y = el[[3, 7, 9]], el[[1, 14, 5]]
    z = gr.inner(x, y)
    for zp in el:
        s = Session(SEED, gr=gr)
        X, Y, Zs = share_input(s, x, 1), share_input(s, y, 2), share_input(s, z[None], 3)[0]
        s.forced[(P_VER_ZETA, obj_id(10, 0, 1))] = zp
        assert bi_verify(s, X, Y, Zs, 10, 0, R=1)


# ---------------------------------------------------------------------------------------------
# consolidations: literal form == rank-1 / merged form
# ---------------------------------------------------------------------------------------------
def _relation_error(gr, xs, ys, zs):
    x, y, z = xs.open(gr.mask), ys.open(gr.mask), zs.open(gr.mask)
    return gr.sub(gr.inner(x, y), z)


@pytest.mark.parametrize("fault", [None, ("MZ2", 1), ("GAMMA2", 1 << 63)])
def test_rank1_equals_literal_consolidation(fault):
    s = Session(SEED)
    gr = s.gr
    rng = np.random.default_rng(10)
    A = rng.integers(0, 2**64, (3, 4), dtype=U64)
    B = rng.integers(0, 2**64, (4, 2), dtype=U64)
    SA, SB = share_input(s, A, 1), share_input(s, B, 2)
    if fault:
        s.arm_fault(*fault[:1], 3, fault[1])
    res = matmul(s, SA, SB, 3)
    r = challenge_r(s, 4, 0)
    e_lit = _relation_error(gr, *tran_matmul_literal(s, SA, SB, res.z_pre, r))
    e_r1 = _relation_error(gr, *tran_matmul_rank1(s, SA, SB, res.z_pre, r))
    assert np.array_equal(e_lit, e_r1)
    assert np.any(e_r1) == (fault is not None)


def test_merged_equals_literal_trunc_consolidation():
    s = Session(SEED)
    gr = s.gr
    rng = np.random.default_rng(11)
    SA = share_input(s, rng.integers(0, 2**64, (2, 3), dtype=U64), 1)
    SB = share_input(s, rng.integers(0, 2**64, (3, 2), dtype=U64), 2)
    res = matmul(s, SA, SB, 3, trunc_bits=13)
    r = challenge_r(s, 4, 1)
    for corrupt in (False, True):
        if corrupt:
            res.tp.p.p1_m[0, ] ^= U64(1 << 63)
        e_lit = _relation_error(gr, *tran_trunc_literal(s, res.tp, r, 13))
        e_mrg = _relation_error(gr, *tran_trunc(s, res.tp, r, 13))
        assert np.array_equal(e_lit, e_mrg)
        assert np.any(e_mrg) == corrupt


# ---------------------------------------------------------------------------------------------
# reading C1: the trunc batch split into independently verified chunks of consecutive outputs
# ---------------------------------------------------------------------------------------------
def test_trunc_chunks_partition_the_outputs():
    from oracle.verify import trunc_chunks
    assert trunc_chunks(10, None) == [(0, 10)]
    assert trunc_chunks(10, 10) == [(0, 10)]
    assert trunc_chunks(10, 64) == [(0, 10)]
    assert trunc_chunks(10, 4) == [(0, 4), (4, 8), (8, 10)]
    assert trunc_chunks(12, 4) == [(0, 4), (4, 8), (8, 12)]
    for E, C in [(1, 1), (7, 3), (100, 7), (2**26, 2**24)]:
        parts = trunc_chunks(E, C)
        assert parts[0][0] == 0 and parts[-1][1] == E
        assert all(a1 == b0 for (_, a1), (b0, _) in zip(parts, parts[1:]))
        assert all(0 < e1 - e0 <= C for e0, e1 in parts)


def _chunk_relation_by_definition(s, tp, e0, e1, r, t):
    """The relation error a chunk's batch certifies, straight from Fig. trunc's two inner
    products: sum over the chunk's outputs of r^(2e') (sum_j c_j b1_j b2_j - p_e) +
    r^(2e'+1) (sum_j c'_j b1_j b2_j - q_e), e' = e - e0 (scalars in Python integers mod 2^64)."""
    from oracle.protocols import trunc_coeffs
    gr = s.gr
    c, cp = trunc_coeffs(t, gr.ell)
    p = tp.p.open(gr.mask).reshape(-1)
    q = tp.q.open(gr.mask).reshape(-1)
    pw = gr.powers(r, 2 * (e1 - e0))
    acc = gr.zeros()
    for e in range(e0, e1):
        b1, b2 = int(tp.b1.reshape(-1)[e]), int(tp.b2.reshape(-1)[e])
        bb = [((b1 >> j) & 1) * ((b2 >> j) & 1) for j in range(gr.ell)]
        dp = (sum(int(c[j]) * bb[j] for j in range(gr.ell)) - int(p[e])) % (1 << 64)
        dq = (sum(int(cp[j]) * bb[j] for j in range(gr.ell)) - int(q[e])) % (1 << 64)
        k = 2 * (e - e0)
        acc = gr.add(acc, gr.add(gr.scale(pw[k], np.uint64(dp)), gr.scale(pw[k + 1], np.uint64(dq))))
    return acc


@pytest.mark.parametrize("corrupt", [None, 2, 9])
def test_chunked_trunc_relation_equals_literal_and_definition(corrupt):
    """Per chunk, the merged consolidation (what the verification runs) carries exactly the
    relation error of the unmerged one and of Fig. trunc's definition over that chunk's outputs;
    an error in output e shows up in e's chunk only."""
    from oracle.verify import trunc_chunk_pairs, trunc_chunks
    s = Session(SEED)
    gr = s.gr
    rng = np.random.default_rng(12)
    SA = share_input(s, rng.integers(0, 2**64, (3, 4), dtype=U64), 1)
    SB = share_input(s, rng.integers(0, 2**64, (4, 5), dtype=U64), 2)
    res = matmul(s, SA, SB, 3, trunc_bits=13)
    if corrupt is not None:
        res.tp.q.p1_m.reshape(-1)[corrupt] ^= U64(1 << 40)
    for i, (e0, e1) in enumerate(trunc_chunks(15, 4)):
        part = trunc_chunk_pairs(res.tp, e0, e1)
        r = challenge_r(s, 4, 1 + i)
        e_mrg = _relation_error(gr, *tran_trunc(s, part, r, 13))
        e_lit = _relation_error(gr, *tran_trunc_literal(s, part, r, 13))
        e_def = _chunk_relation_by_definition(s, res.tp, e0, e1, r, 13)
        assert np.array_equal(e_mrg, e_lit)
        assert np.array_equal(e_mrg, e_def)
        assert np.any(e_mrg) == (corrupt is not None and e0 <= corrupt < e1)


@pytest.mark.parametrize("fault_out", [None, 0, 6, 14])
def test_chunked_trunc_verify_accepts_honest_and_rejects_in_the_faulty_chunk(fault_out):
    from oracle.verify import trunc_verify
    s = Session(SEED)
    rng = np.random.default_rng(13)
    SA = share_input(s, rng.integers(0, 2**64, (3, 4), dtype=U64), 1)
    SB = share_input(s, rng.integers(0, 2**64, (4, 5), dtype=U64), 2)
    res = matmul(s, SA, SB, 3, trunc_bits=13)
    if fault_out is not None:   # P0's Gamma of output fault_out's p inner product, as P2 sees it
        res.tp.p.p2_m.reshape(-1)[fault_out] ^= U64(1)
        res.tp.p.p1_m.reshape(-1)[fault_out] ^= U64(1)
    oks = trunc_verify(s, res.tp, 4, 13, chunk=4)
    want = [fault_out is None or not (4 * i <= fault_out < 4 * i + 4) for i in range(4)]
    assert oks == want


def test_one_chunk_is_the_unchunked_batch():
    """With the chunk at least the batch, the chunked verification is the batch's own: the same
    challenges, rounds and opened Delta."""
    rng = np.random.default_rng(14)
    A = rng.integers(0, 2**64, (2, 6), dtype=U64)
    B = rng.integers(0, 2**64, (6, 3), dtype=U64)
    traces = []
    for chunk in (None, 6, 1000):
        s = Session(SEED)
        SA, SB = share_input(s, A, 1), share_input(s, B, 2)
        res = matmul(s, SA, SB, 3, trunc_bits=13)
        tr = []
        assert matmul_verify(s, SA, SB, res, 4, 13, trace=tr, trunc_chunk=chunk)
        traces.append(tr)
    for other in traces[1:]:
        assert len(other) == len(traces[0])
        for a, b in zip(traces[0], other):
            assert a.keys() == b.keys()
            for k in a:
                va, vb = a[k], b[k]
                if hasattr(va, "as_tuple"):
                    assert all(np.array_equal(x, y) for x, y in zip(va.as_tuple(), vb.as_tuple()))
                else:
                    assert np.array_equal(np.asarray(va), np.asarray(vb))
