"""Non-linear layers (Sec. 4.3): daBits, edaBits, MSB extraction by a carry circuit, B2A, ReLU,
2x2 max-pool, and the verification of every product they create (oracle; test infrastructure
only).

Conventions (readings, also in the design notes):
  - An arithmetic sharing of a bit known to a pair follows reading A1 ([r] = -b): a bit from
    eta01 is (0, b, 0) with [r]_1 = -b, one from eta02 has [r]_2 = -b, one from eta12 has m = b.
  - Boolean sharings are <.>^1 over Z_2 in a BoolSession; + and - are XOR.
  - Every per-element batch is padded to n_pad = 64 * ceil(n / 64) elements (zeros), and Boolean
    values of several bit positions are stored plane-major, shape (planes, n_pad): the bit of
    plane p and element e is stream / wire position p * n_pad + e.
  - Streams of one layer call use obj_id(call_id, stage, sub): stage 0 for ReLU and the first
    max-pool comparison, 1 for the second; sub = circuit level for the AND gates.
  - The Boolean AND gates are verified in GF(2^64) with verify batch 2, so that their challenges
    never share a stream with the arithmetic batches 0 (products) and 1 (edaBit inner products).
  - Reading N9: the edaBit bit products b_{i,1} b_{i,2} (64 per element) are verified in a batch
    of their own (verify batch 3) and batch 0 keeps the daBit and final products (3 per element).
    Every product is still checked with a fresh challenge; splitting one Pi_MultVerify batch into
    two adds their soundness errors (union bound).  The bit batch has the truncation pairs' form:
    x carries only [r]_1 (P0, P1 copies) and y only [r]_2 (P0, P2 copies).
"""
from __future__ import annotations

import numpy as np

from .protocols import inner_rows, mult, reconstruct
from .shares import (C_G1, C_M12, C_R1, C_R2, OFFLINE, P_AND, P_DA_MULT1, P_DA_MULT2, P_DABIT,
                     P_EDA_INNER, P_EDA_MULT, P_EDABIT, P_NL_MULT, Session, Shared, obj_id)
from .verify import BATCH_MAIN, bi_verify, challenge_r, lift_shared, tran_mult, _gr_sum

U64 = np.uint64
BATCH_EDA_INNER = 1
BATCH_BOOL = 2
BATCH_EDA_MULT = 3


def n_padded(n: int) -> int:
    return 64 * ((n + 63) // 64)


# ---- sharings of pair-known bits and public constants ------------------------------------------
def arith_from_r1_bits(b) -> Shared:
    """<b> := (0, b, 0) (Fig. edabits), i.e. [r]_1 = -b under reading A1."""
    z = np.zeros_like(b, dtype=U64)
    nb = (U64(0) - b.astype(U64))
    return Shared(nb, z.copy(), z.copy(), nb.copy(), z.copy(), z.copy())


def arith_from_r2_bits(b) -> Shared:
    z = np.zeros_like(b, dtype=U64)
    nb = (U64(0) - b.astype(U64))
    return Shared(z, nb, z.copy(), z.copy(), z.copy(), nb.copy())


def arith_from_m_bits(m) -> Shared:
    z = np.zeros_like(m, dtype=U64)
    return Shared(z, z.copy(), m.astype(U64), z.copy(), m.astype(U64).copy(), z.copy())


def s_add(a: Shared, b: Shared) -> Shared:
    return a.zip(b, lambda u, v: u + v)


def s_sub(a: Shared, b: Shared) -> Shared:
    return a.zip(b, lambda u, v: u - v)


def s_scale(a: Shared, c) -> Shared:
    c = np.asarray(c, dtype=U64)
    return a.map(lambda u: u * c)


def s_add_public(a: Shared, c) -> Shared:
    """<a + c> for public c: only the m components change."""
    c = np.asarray(c, dtype=U64)
    return Shared(a.p0_r1.copy(), a.p0_r2.copy(), a.p1_m + c, a.p1_r1.copy(), a.p2_m + c,
                  a.p2_r2.copy())


def b_xor(a: Shared, b: Shared) -> Shared:
    return a.zip(b, lambda u, v: u ^ v)


def b_and_public(a: Shared, c) -> Shared:
    c = np.asarray(c, dtype=U64) & U64(1)
    return a.map(lambda u: u & c)


def b_xor_public(a: Shared, c) -> Shared:
    c = np.asarray(c, dtype=U64) & U64(1)
    return Shared(a.p0_r1.copy(), a.p0_r2.copy(), a.p1_m ^ c, a.p1_r1.copy(), a.p2_m ^ c,
                  a.p2_r2.copy())


def b_public(c, shape) -> Shared:
    v = np.broadcast_to(np.asarray(c, dtype=U64) & U64(1), shape).copy()
    z = np.zeros(shape, dtype=U64)
    return Shared(z, z.copy(), v, z.copy(), v.copy(), z.copy())


def stack(parts) -> Shared:
    return Shared(*(np.stack([getattr(p, f) for p in parts]) for f in Shared.FIELDS))


def row(s: Shared, i) -> Shared:
    return Shared(*(getattr(s, f)[i] for f in Shared.FIELDS))


# ---- daBits and edaBits (Sec. 4.3, Fig. edabits) ----------------------------------------------------
def dabits(sess: Session, bsess: Session, call_id: int, stage: int, n_pad: int):
    """n_pad daBits (<r>^l, <r>^1): P0,P1 pick r1, P0,P2 pick r2, P1,P2 pick r3; <r>^1 = (r3, r1, r2);
    <r'> = <r1> + <r2> - 2 <r1><r2>, <r> = <r'> + <r3> - 2 <r'><r3> (two Pi_Mult rounds)."""
    obj = obj_id(call_id, stage, 0)
    r1 = bsess.prf(C_R1, P_DABIT, obj, n_pad)
    r2 = bsess.prf(C_R2, P_DABIT, obj, n_pad)
    r3 = bsess.prf(C_M12, P_DABIT, obj, n_pad)
    rb = Shared(r1, r2, r3, r1.copy(), r3.copy(), r2.copy())
    A1, A2, A3 = arith_from_r1_bits(r1), arith_from_r2_bits(r2), arith_from_m_bits(r3)
    t = mult(sess, A1, A2, call_id, P_DA_MULT1, stage)
    rp = s_sub(s_add(A1, A2), s_scale(t, 2))
    u = mult(sess, rp, A3, call_id, P_DA_MULT2, stage)
    ra = s_sub(s_add(rp, A3), s_scale(u, 2))
    return ra, rb, [(A1, A2, t), (rp, A3, u)]


def edabits(sess: Session, bsess: Session, call_id: int, stage: int, n_pad: int):
    """n_pad edaBits (<r>^l, {<r[i]>^1}) by Fig. edabits: P0,P1 pick b_{i,1}; P0,P2 pick b_{i,2};
    P1,P2 pick m_i; <r[i]>^1 := (m_i, b_{i,1}, b_{i,2}); <r'[i]> = <b_{i,1}> + <b_{i,2}> - 2 <b_{i,1}><b_{i,2}>
    (64 Pi_Mult per element) and <r> = sum_i 2^i (<m_i> + <r'[i]>) - <sum_i 2^(i+1) m_i r'[i]>, the
    last sum being one Pi_Inner of dimension 64 per element (the paper merges the second product
    round into an inner product).  Bits are plane-major: plane i, element e."""
    obj = obj_id(call_id, stage, 0)
    b1 = bsess.prf(C_R1, P_EDABIT, obj, 64 * n_pad).reshape(64, n_pad)
    b2 = bsess.prf(C_R2, P_EDABIT, obj, 64 * n_pad).reshape(64, n_pad)
    mb = bsess.prf(C_M12, P_EDABIT, obj, 64 * n_pad).reshape(64, n_pad)
    rbits = Shared(b1, b2, mb, b1.copy(), mb.copy(), b2.copy())
    B1, B2, Mv = arith_from_r1_bits(b1), arith_from_r2_bits(b2), arith_from_m_bits(mb)
    prod = mult(sess, B1, B2, call_id, P_EDA_MULT, stage)
    rp = s_sub(s_add(B1, B2), s_scale(prod, 2))
    coef = (U64(2) << np.arange(64, dtype=U64))[:, None]          # 2^(i+1), plane i (wraps at 64)
    X = Mv.map(lambda a: np.ascontiguousarray(a.T))                  # (n_pad, 64): element, bit
    Y = s_scale(rp, coef).map(lambda a: np.ascontiguousarray(a.T))
    rz1 = sess.prf(C_R1, P_EDA_INNER, obj, n_pad)
    rz2 = sess.prf(C_R2, P_EDA_INNER, obj, n_pad)
    g1 = sess.prf(C_G1, P_EDA_INNER, obj, n_pad)
    z, _ = inner_rows(sess, X, Y, rz1, rz2, g1, "inner", OFFLINE, OFFLINE)
    pw = (U64(1) << np.arange(64, dtype=U64))[:, None]
    lin = s_scale(s_add(Mv, rp), pw).map(lambda a: np.sum(a, axis=0, dtype=U64))
    ra = s_sub(lin, z)
    return ra, rbits, [(B1, B2, prod)], [(X, Y, z)]


# ---- MSB by a parallel-prefix carry circuit ------------------------------------------------------
def msb(sess: Session, bsess: Session, x: Shared, eda, call_id: int, stage: int):
    """<msb(x)>^1 (Sec. 4.3 bit extraction): open Delta = x - r, then x = Delta + r, so
    msb(x) = Delta_63 xor r[63] xor c_63 with c_63 the carry into bit 63 of Delta + r.  The carry
    is the root of a 6-level tree over the (generate, propagate) pairs of bits 0..62
    (g_i = Delta_i r[i], p_i = Delta_i xor r[i], both local because Delta is public; leaf 63 is the
    identity (0, 1)); a node combines (G_hi, P_hi) o (G_lo, P_lo) = (G_hi xor P_hi G_lo, P_hi P_lo).
    The ANDs of one level are one Boolean Pi_Mult: planes 0..C-1 are P_hi G_lo of the C nodes,
    planes C..2C-1 (not at the root) P_hi P_lo."""
    ra, rbits = eda[0], eda[1]
    n_pad = x.p1_m.shape[0]
    delta = reconstruct(sess, s_sub(x, ra))
    db = (delta[None, :] >> np.arange(64, dtype=U64)[:, None]) & U64(1)   # (64, n_pad)
    G = [b_and_public(row(rbits, i), db[i]) for i in range(63)] + [b_public(0, (n_pad,))]
    P = [b_xor_public(row(rbits, i), db[i]) for i in range(63)] + [b_public(1, (n_pad,))]
    triples = []
    level = 0
    while len(G) > 1:
        level += 1
        C = len(G) // 2
        root = C == 1
        xs = [P[2 * k + 1] for k in range(C)] + ([] if root else [P[2 * k + 1] for k in range(C)])
        ys = [G[2 * k] for k in range(C)] + ([] if root else [P[2 * k] for k in range(C)])
        X, Y = stack(xs), stack(ys)
        Z = mult(bsess, X, Y, call_id, P_AND, stage, level)
        triples.append((X, Y, Z))
        G = [b_xor(G[2 * k + 1], row(Z, k)) for k in range(C)]
        P = [] if root else [row(Z, C + k) for k in range(C)]
    out = b_xor_public(b_xor(row(rbits, 63), G[0]), db[63])
    return out, delta, triples


def b2a(sess: Session, bsess: Session, b: Shared, dab, call_id: int):
    """<b>^1 -> <b>^l with a daBit (Sec. 4.3): open Delta = b xor r over Z_2, then
    <b>^l = Delta + <r>^l - 2 Delta <r>^l (local, Delta public)."""
    ra, rb = dab[0], dab[1]
    delta = reconstruct(bsess, b_xor(b, rb))
    sign = (U64(1) - U64(2) * delta.astype(U64))
    return s_add_public(s_scale(ra, sign), delta)


# ---- layers ---------------------------------------------------------------------------------------
def compare_select(sess: Session, bsess: Session, a: Shared, b: Shared, call_id: int, stage: int):
    """<max(a, b)> (signed, |a - b| < 2^63) = b + (a - b) [a >= b], [a >= b] = 1 - msb(a - b)
    (reading A16).  Returns the output and every product made, for the layer's verification."""
    n_pad = a.p1_m.shape[0]
    d = s_sub(a, b)
    ra, rbits, eda_mults, eda_inner = edabits(sess, bsess, call_id, stage, n_pad)
    m, _, and_triples = msb(sess, bsess, d, (ra, rbits), call_id, stage)
    ge = b_xor_public(m, 1)
    da_ra, da_rb, da_mults = dabits(sess, bsess, call_id, stage, n_pad)
    ge_a = b2a(sess, bsess, ge, (da_ra, da_rb), call_id)
    prod = mult(sess, d, ge_a, call_id, P_NL_MULT, stage)
    out = s_add(b, prod)
    return out, {"mults": da_mults + [(d, ge_a, prod)], "eda": eda_mults, "inner": eda_inner,
                 "and": and_triples}


def pad_shared(x: Shared, n_pad: int) -> Shared:
    def f(a):
        out = np.zeros(n_pad, dtype=U64)
        out[: a.size] = a.reshape(-1)
        return out
    return x.map(f)


def relu(sess: Session, bsess: Session, x: Shared, call_id: int):
    """ReLU(x) = x [x >= 0] = max(x, 0), ReLU(0) = 0; x is padded to n_pad elements."""
    n = x.p1_m.size
    xp = pad_shared(x, n_padded(n))
    zero = xp.map(np.zeros_like)
    out, tr = compare_select(sess, bsess, xp, zero, call_id, 0)
    return out.map(lambda a: a[:n].copy()), [tr]


def maxpool2(sess: Session, bsess: Session, x: Shared, shape, call_id: int):
    """2x2 / stride-2 max-pool of a (B, C, H, W) tensor (H, W even): stage 0 compares the pairs
    (a, b) and (c, d) of every window (a = [2i][2j], b = [2i][2j+1], c = [2i+1][2j], d = [2i+1][2j+1])
    in one batch [a; c] vs [b; d]; stage 1 compares the two winners."""
    B, Cc, H, W = shape
    v = x.map(lambda a: a.reshape(B, Cc, H, W))
    q = [v.map(lambda a, s=s: np.ascontiguousarray(a[:, :, s[0]::2, s[1]::2]).reshape(-1))
         for s in ((0, 0), (0, 1), (1, 0), (1, 1))]
    nw = B * Cc * (H // 2) * (W // 2)
    n0 = n_padded(2 * nw)
    left = pad_shared(q[0].zip(q[2], lambda u, w: np.concatenate([u, w])), n0)
    right = pad_shared(q[1].zip(q[3], lambda u, w: np.concatenate([u, w])), n0)
    m, tr0 = compare_select(sess, bsess, left, right, call_id, 0)
    n1 = n_padded(nw)
    m1 = pad_shared(m.map(lambda a: a[:nw]), n1)
    m2 = pad_shared(m.map(lambda a: a[nw:2 * nw]), n1)
    out, tr1 = compare_select(sess, bsess, m1, m2, call_id, 1)
    return out.map(lambda a: a[:nw].copy()), [tr0, tr1]


# ---- verification of a non-linear layer ---------------------------------------------------------
def _flat_concat(triples, k):
    return Shared(*(np.concatenate([getattr(t[k], f).reshape(-1) for t in triples])
                    for f in Shared.FIELDS))


def tran_rows(sess: Session, X: Shared, Y: Shared, Z: Shared, r) -> tuple:
    """Fig. PBDP for n inner products of dimension k (rows of X, Y): weight r^e on row e,
    x'_{e,i} = r^e X_{e,i}, y lifted, z = sum_e r^e Z_e; flattened e-major."""
    gr = sess.gr
    n, k = X.p1_m.shape
    pw = gr.powers(r, n)
    xs = X.map(lambda a: gr.scale(np.repeat(pw, k, axis=0), a.reshape(-1)))
    ys = lift_shared(gr, Y.map(lambda a: a.reshape(-1)))
    zs = Z.map(lambda a: _gr_sum(gr, gr.scale(pw, a.reshape(-1))))
    return xs, ys, zs


def verify_layer(sess: Session, bsess: Session, triples, verify_id: int, R_mult=None,
                 R_inner=None, R_and=None, trace=None, R_eda=None) -> bool:
    """Pi_MultVerify of the daBit and final products (batch 0), Pi_BIVerify of the edaBit inner
    products (batch 1), both over GR(2^64, 64), Pi_MultVerify of every AND gate over GF(2^64)
    (batch 2) (Sec. 4.3: products over Z_2^l and Z_2 verified in their rings), and Pi_MultVerify
    of the edaBit bit products over GR(2^64, 64) (batch 3, reading N9).  `trace`, if given, is a
    dict of four lists."""
    mults = [t for tr in triples for t in tr["mults"]]
    edas = [t for tr in triples for t in tr["eda"]]
    inner = [t for tr in triples for t in tr["inner"]]
    ands = [t for tr in triples for t in tr["and"]]
    tr = trace if trace is not None else {"mult": None, "inner": None, "and": None, "eda": None}
    X, Y, Z = (_flat_concat(mults, k) for k in range(3))
    r = challenge_r(sess, verify_id, BATCH_MAIN)
    ok0 = bi_verify(sess, *tran_mult(sess, X, Y, Z, r), verify_id, BATCH_MAIN, R_mult, tr["mult"])
    Xi = Shared(*(np.concatenate([getattr(t[0], f) for t in inner]) for f in Shared.FIELDS))
    Yi = Shared(*(np.concatenate([getattr(t[1], f) for t in inner]) for f in Shared.FIELDS))
    Zi = Shared(*(np.concatenate([getattr(t[2], f).reshape(-1) for t in inner]) for f in Shared.FIELDS))
    r1 = challenge_r(sess, verify_id, BATCH_EDA_INNER)
    ok1 = bi_verify(sess, *tran_rows(sess, Xi, Yi, Zi, r1), verify_id, BATCH_EDA_INNER, R_inner,
                    tr["inner"])
    Xa, Ya, Za = (_flat_concat(ands, k) for k in range(3))
    r2 = challenge_r(bsess, verify_id, BATCH_BOOL)
    ok2 = bi_verify(bsess, *tran_mult(bsess, Xa, Ya, Za, r2), verify_id, BATCH_BOOL, R_and,
                    tr["and"])
    Xe, Ye, Ze = (_flat_concat(edas, k) for k in range(3))
    r3 = challenge_r(sess, verify_id, BATCH_EDA_MULT)
    ok3 = bi_verify(sess, *tran_mult(sess, Xe, Ye, Ze, r3), verify_id, BATCH_EDA_MULT, R_eda,
                    tr["eda"])
    return bool(ok0 and ok1 and ok2 and ok3)
