"""Sharing, reconstruction, multiplication, inner product and truncation (oracle; test infra only).

Each function restates one of the paper's protocols, in the paper's order and notation, on all
three parties' views.  Every random value comes from the pairwise PRG streams of ``Session``.

* ``share_input``   Pi_<.>^{l,k}(x) with owner P0 (Sec. 2 "Secret sharing").
* ``reconstruct``   Pi_Rec (Sec. 2 "Verifiability of share reconstruction").
* ``mult``          Pi_Mult offline + online (Fig. MultP; Sec. 2 "Multiplication gate").
* ``inner_rows``    Pi_Inner offline + online for a batch of inner products (Fig. DPP).
* ``matmul``        Pi_Inner for every output of X.W (Sec. 4.1: a matrix product is m inner
                    products), optionally with Pi_Trunc^t (Fig. trunc).
* ``trunc_pair``    Pi_Trunc^t preprocessing (Fig. trunc); its bits keyed by the call or, for
                    packed serving batches, by output row (``trunc_bit_words``, reading A12).
* ``trunc``         Pi_Trunc^t of an existing sharing (Fig. trunc, reading T5).
* ``conv2d``        a convolution as one Pi_Inner per output (Sec. 4.1), on the im2col rows of the
                    input written out from the definition of a convolution.

Readings of the paper (where it is silent, ambiguous or garbled):
  A1  m = x + r everywhere (Sec. 2 Notation); a bit sharing <b> := (0, b, 0) therefore carries
      [r] = -b so that its value is b.
  A2  Gamma = r_x r_y + r_z (Fig. MultP, Fig. DPP); "m_{y_i}" there means m_y.
  T1  r_z's second sum runs over j = l-t .. l-1, so r_z = r_x >>_arith t.
  T2  m_z = m_x >>_arith t ("rshift", Fig. trunc).
  T3  [r_x]_1 := m_{r_x} - [r_{r_x}]_1 (P1) and [r_x]_2 := -[r_{r_x}]_2 (P2); P0 computes both
      from m_{r_x} = Gamma (it knows every r).  Same for r_z.
  T5  Fig. trunc assigns the pair's r_x to the input wire before the gate that produces it runs
      ("executed preferentially"), as ``matmul`` does.  For a sharing <x> whose mask r is not a
      pair's r_x, the mask is switched to r_x first: P1 sends d1 = [r_x]_1 - [r]_1 to P2 and P2
      sends d2 = [r_x]_2 - [r]_2 to P1 (l bits each), both set m' = m + d1 + d2 = x + r_x, and
      P0, who knows d1 and d2, sends H(d1) to P2 and H(d2) to P1 (a party whose received d
      disagrees with the hash aborts, as in Pi_Rec); then m_z = m' >>_arith t.  This is the
      standalone truncation with 2 l bits online that the paper attributes to SWIFT.
  D1  Fixed point: floor(x 2^k) mod 2^l (Sec. 2 Notation); a value whose x 2^k lies outside
      [-2^63, 2^63) saturates to the nearest end, and NaN encodes 0 (the paper assumes values in
      range and says nothing about the others).
Parity: pinned (tests/test_oracle_protocols.py) by reconstruction against plaintext products mod
2^l, the truncation error model of Sec. 4.2, and the communication counts of Table 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .merkle import hash_u64
from .shares import (C_G1, C_R1, C_R2, C_TB1, C_TB2, OFFLINE, ONLINE, P_INNER, P_MULT,
                     P_SHARE, P_TRUNC_BITS, P_TRUNC_P, P_TRUNC_Q, Session, Shared, obj_id)

U64 = np.uint64


class Abort(Exception):
    """A party received inconsistent messages in Pi_Rec and aborts (security with abort)."""


# ---------------------------------------------------------------------------------------------
# fixed point (Sec. 2 Notation): x >= 0 -> floor(x 2^k); x < 0 -> 2^l + floor(x 2^k)
# ---------------------------------------------------------------------------------------------
def encode_fixed(x, k: int) -> np.ndarray:
    """floor(x 2^k) as a two's-complement word (reading D1 for values out of range and NaN)."""
    v = np.floor(np.asarray(x, dtype=np.float64) * float(1 << k))
    lo, hi = -9223372036854775808.0, 9223372036854775808.0    # -2^63, 2^63
    out = np.zeros(v.shape, dtype=np.int64)
    ok = (v >= lo) & (v < hi)
    out[ok] = v[ok].astype(np.int64)
    out[v >= hi] = np.iinfo(np.int64).max
    out[v < lo] = np.iinfo(np.int64).min
    return out.astype(np.uint64)


def decode_fixed(v, k: int) -> np.ndarray:
    return np.asarray(v, dtype=np.uint64).astype(np.int64).astype(np.float64) / float(1 << k)


def asr(v, t: int) -> np.ndarray:
    """Arithmetic right shift of two's-complement u64 values by t bits."""
    return (np.asarray(v, dtype=np.uint64).astype(np.int64) >> np.int64(t)).astype(np.uint64)


# ---------------------------------------------------------------------------------------------
# Pi_<.>^{l,k}(x): P_k owns x
# ---------------------------------------------------------------------------------------------
def share_input(sess: Session, x, call_id: int, phase: str = ONLINE, owner: int = 0) -> Shared:
    """Pi_<.>^{l,k} (Sec. 2, Secret sharing).  Offline: [r_x] <- Pi_[.] (r1 from eta01, r2 from
    eta02); the owner P_k holds both seeds of this mask and sends m_x = x + [r_x]_1 + [r_x]_2 to
    P1 and P2: P0 sends two messages, P1 (P2) keeps its own copy and sends one to P2 (P1).
    Reading: "P_i send" there is the owner P_k, and the owner's seeds give the same r1, r2 as
    P0's, so the sharing does not depend on k; only the messages do."""
    if owner not in (0, 1, 2):
        raise ValueError("owner must be 0, 1 or 2")
    x = np.asarray(x, dtype=U64) & sess.mask
    obj = obj_id(call_id)
    r1 = sess.prf(C_R1, P_SHARE, obj, x.size).reshape(x.shape)
    r2 = sess.prf(C_R2, P_SHARE, obj, x.size).reshape(x.shape)
    m = (x + r1 + r2) & sess.mask
    if owner == 0:
        m_p1 = sess.send(0, 1, phase, "share", m, site="MX_COPY_P1")
        m_p2 = sess.send(0, 2, phase, "share", m)
    elif owner == 1:
        m_p1 = m.copy()
        m_p2 = sess.send(1, 2, phase, "share", m)
    else:
        m_p1 = sess.send(2, 1, phase, "share", m, site="MX_COPY_P1")
        m_p2 = m.copy()
    return Shared(r1.copy(), r2.copy(), m_p1, r1.copy(), m_p2, r2.copy())


# ---------------------------------------------------------------------------------------------
# Pi_Rec
# ---------------------------------------------------------------------------------------------
def reconstruct(sess: Session, x: Shared, phase: str = ONLINE, proto: str = "rec") -> np.ndarray:
    """P0 sends [r]_1 to P2 and [r]_2 to P1; P1 sends m to P0 and H([r]_1) to P2; P2 sends H(m)
    to P0 and H([r]_2) to P1.  Any party seeing a value disagree with its hash aborts; otherwise
    each outputs x = m - [r]_1 - [r]_2."""
    r1_at_p2 = sess.send(0, 2, phase, proto, x.p0_r1)
    r2_at_p1 = sess.send(0, 1, phase, proto, x.p0_r2, site="REC_MSG")
    m_at_p0 = sess.send(1, 0, phase, proto, x.p1_m)
    w = sess.wire
    h_r1_at_p2 = sess.send_hash(1, 2, phase, proto, hash_u64(w(x.p1_r1)))
    h_m_at_p0 = sess.send_hash(2, 0, phase, proto, hash_u64(w(x.p2_m)))
    h_r2_at_p1 = sess.send_hash(2, 1, phase, proto, hash_u64(w(x.p2_r2)))
    if hash_u64(w(m_at_p0)) != h_m_at_p0:
        raise Abort("P0: m from P1 disagrees with H(m) from P2")
    if hash_u64(w(r2_at_p1)) != h_r2_at_p1:
        raise Abort("P1: [r]_2 from P0 disagrees with H([r]_2) from P2")
    if hash_u64(w(r1_at_p2)) != h_r1_at_p2:
        raise Abort("P2: [r]_1 from P0 disagrees with H([r]_1) from P1")
    mask = sess.mask
    out0 = (m_at_p0 - x.p0_r1 - x.p0_r2) & mask
    out1 = (x.p1_m - x.p1_r1 - r2_at_p1) & mask
    out2 = (x.p2_m - r1_at_p2 - x.p2_r2) & mask
    assert np.array_equal(out0, out1) and np.array_equal(out1, out2)
    return out1


# ---------------------------------------------------------------------------------------------
# Pi_Mult (elementwise)
# ---------------------------------------------------------------------------------------------
def _gamma_message(sess: Session, gamma_p0, g1, proto: str, phase: str):
    """Pi_[.](Gamma) by P0: [Gamma]_1 = PRG(eta01) (computed by P0 and P1), P0 sends
    [Gamma]_2 = Gamma - [Gamma]_1 to P2.  The HIGH_BIT site models the ring attack e = 2^(l-1)."""
    g2 = (gamma_p0 - g1) & sess.mask
    if "HIGH_BIT" in sess.faults:
        idx, _ = sess.faults.pop("HIGH_BIT")
        sess.faults["GAMMA2"] = (idx, 1 << (sess.gr.ell - 1))
    return sess.send(0, 2, phase, proto, g2, site="GAMMA2")


def _exchange_mz(sess: Session, mz1, mz2, proto: str, phase: str):
    mz1_at_p2 = sess.send(1, 2, phase, proto, mz1, site="MZ1")
    mz2_at_p1 = sess.send(2, 1, phase, proto, mz2, site="MZ2")
    mask = sess.mask
    return (mz1 + mz2_at_p1) & mask, (mz1_at_p2 + mz2) & mask


def mult(sess: Session, x: Shared, y: Shared, call_id: int, purpose: int = P_MULT,
         batch: int = 0, sub: int = 0) -> Shared:
    """Fig. MultP.  Offline: [r_z] <- Pi_[.]; P0 computes Gamma = r_x r_y + r_z and shares it with
    Pi_[.](Gamma).  Online: P_j computes [m_z]_j = (j-1) m_x m_y - m_x [r_y]_j - m_y [r_x]_j +
    [Gamma]_j, and P1, P2 exchange their shares to reconstruct m_z.  Element i's mask and [Gamma]_1
    are words i of the (purpose, obj_id(call_id, batch, sub)) streams; over Z_2 (a Boolean
    session) the same formulas are the AND gate, with + and - both XOR."""
    mask = sess.mask
    obj = obj_id(call_id, batch, sub)
    n = x.p1_m.size
    shape = x.p1_m.shape
    rz1 = sess.prf(C_R1, purpose, obj, n).reshape(shape)
    rz2 = sess.prf(C_R2, purpose, obj, n).reshape(shape)
    # offline, P0
    rx = (x.p0_r1 + x.p0_r2) & mask
    ry = (y.p0_r1 + y.p0_r2) & mask
    gamma = (rx * ry + rz1 + rz2) & mask
    g1 = sess.prf(C_G1, purpose, obj, n).reshape(shape)
    g2_at_p2 = _gamma_message(sess, gamma, g1, "mult", OFFLINE)
    # online, P1 (j = 1) and P2 (j = 2)
    mz1 = (U64(0) - x.p1_m * y.p1_r1 - y.p1_m * x.p1_r1 + g1) & mask
    mz2 = (x.p2_m * y.p2_m - x.p2_m * y.p2_r2 - y.p2_m * x.p2_r2 + g2_at_p2) & mask
    mz_p1, mz_p2 = _exchange_mz(sess, mz1, mz2, "mult", ONLINE)
    return Shared(rz1.copy(), rz2.copy(), mz_p1, rz1.copy(), mz_p2, rz2.copy())


# ---------------------------------------------------------------------------------------------
# Pi_Inner for a batch of inner products over the last axis
# ---------------------------------------------------------------------------------------------
def inner_rows(sess: Session, x: Shared, y: Shared, mask_r1, mask_r2, g1, proto: str,
               phase_gamma: str, phase_mz: str) -> tuple:
    """Fig. DPP for z_e = sum_i x_{e,i} y_{e,i} (one inner product per leading index e), with the
    output mask [r_z] = (mask_r1, mask_r2) and [Gamma]_1 = g1 supplied by the caller's streams.
    Returns (<z>, Gamma as computed by P0)."""
    mask = sess.mask
    rx = (x.p0_r1 + x.p0_r2) & mask
    ry = (y.p0_r1 + y.p0_r2) & mask
    gamma = (np.sum(rx * ry, axis=-1, dtype=U64) + mask_r1 + mask_r2) & mask
    g2_at_p2 = _gamma_message(sess, gamma, g1, proto, phase_gamma)
    mz1 = (np.sum(U64(0) - x.p1_m * y.p1_r1 - y.p1_m * x.p1_r1, axis=-1, dtype=U64) + g1) & mask
    mz2 = (np.sum(x.p2_m * y.p2_m - x.p2_m * y.p2_r2 - y.p2_m * x.p2_r2, axis=-1, dtype=U64)
           + g2_at_p2) & mask
    mz_p1, mz_p2 = _exchange_mz(sess, mz1, mz2, proto, phase_mz)
    z = Shared(mask_r1.copy(), mask_r2.copy(), mz_p1, mask_r1.copy(), mz_p2, mask_r2.copy())
    return z, gamma


# ---------------------------------------------------------------------------------------------
# Pi_Trunc^t preprocessing
# ---------------------------------------------------------------------------------------------
def trunc_coeffs(t: int, ell: int = 64):
    """Coefficients of the two dimension-l inner products of Fig. trunc, written as
    r_x = b1 + b2 + sum_j c_j b1_j b2_j and r_z = asr(b1,t) + asr(b2,t) + sum_j c'_j b1_j b2_j
    (b1 + b2 - 2 b1 b2 = b1 xor b2 bitwise).  c_j = -2^(j+1); c'_j = -2 w_j where w_j is the
    weight of bit j in an arithmetic shift by t: 2^(j-t) for t <= j < l-1, and for the sign bit
    2^(l-1-t) + sum_{i=l-t}^{l-1} 2^i (reading T1)."""
    M = 1 << ell
    c = np.array([(-(1 << (j + 1))) % M for j in range(ell)], dtype=np.uint64)
    w = [0] * ell
    for j in range(t, ell - 1):
        w[j] = 1 << (j - t)
    w[ell - 1] = ((1 << (ell - 1 - t)) + sum(1 << i for i in range(ell - t, ell))) % M
    cp = np.array([(-2 * wj) % M for wj in w], dtype=np.uint64)
    return c, cp


def bit_matrix(words, ell: int = 64) -> np.ndarray:
    """(E,) u64 words -> (E, l) array of their bits (bit j in column j)."""
    words = np.asarray(words, dtype=U64)
    return (words[:, None] >> np.arange(ell, dtype=U64)[None, :]) & U64(1)


@dataclass
class TruncPair:
    b1: np.ndarray            # (E,) words of bits b_{1,j}: P0 and P1
    b2: np.ndarray            # (E,) words of bits b_{2,j}: P0 and P2
    p: Shared                 # <sum_j c_j b1_j b2_j>   (Pi_Inner #1)
    q: Shared                 # <sum_j c'_j b1_j b2_j>  (Pi_Inner #2)
    rx1_p0: np.ndarray        # [r_x]_1 at P0
    rx2_p0: np.ndarray
    rx1_p1: np.ndarray        # [r_x]_1 at P1
    rx2_p2: np.ndarray        # [r_x]_2 at P2
    rz1_p0: np.ndarray
    rz2_p0: np.ndarray
    rz1_p1: np.ndarray
    rz2_p2: np.ndarray


def bit_sharings(sess: Session, b1, b2):
    """<b1_j> := (m = 0, [r]_1 = -b1_j, [r]_2 = 0) and <b2_j> := (0, 0, -b2_j) (Fig. trunc with
    reading A1), as (E, l) Shared arrays."""
    mask = sess.mask
    B1 = bit_matrix(b1, sess.gr.ell)
    B2 = bit_matrix(b2, sess.gr.ell)
    z = np.zeros_like(B1)
    nb1 = (U64(0) - B1) & mask
    nb2 = (U64(0) - B2) & mask
    sb1 = Shared(nb1, z, z, nb1, z, z)
    sb2 = Shared(z, nb2, z, z, z, nb2)
    return sb1, sb2


def trunc_bit_words(sess: Session, comp: int, call_id: int, E: int, row_keys=None, N: int = None):
    """The E words of a truncation-bit stream: word e of the call's stream, or, keyed by rows
    (reading A12: randomness keyed by request, layer and row, never by batch slot), word e mod N
    of the stream of object row_keys[e // N]."""
    if row_keys is None:
        return sess.prf(comp, P_TRUNC_BITS, obj_id(call_id), E)
    rows = [sess.prf(comp, P_TRUNC_BITS, int(k), N) for k in row_keys]
    return np.concatenate(rows)[:E] if rows else np.zeros(0, dtype=U64)


def trunc_pair(sess: Session, call_id: int, E: int, t: int, row_keys=None, N: int = None
               ) -> TruncPair:
    """Fig. trunc, preprocessing: P0,P1 pick bits b1 (eta01); P0,P2 pick bits b2 (eta02);
    <r_x> and <r_z> are obtained with two Pi_Inner of dimension l over the bit sharings; then the
    additive shares [r_x], [r_z] are formed as in reading T3.  row_keys: see ``trunc_bit_words``."""
    mask = sess.mask
    ell = sess.gr.ell
    obj = obj_id(call_id)
    b1 = trunc_bit_words(sess, C_TB1, call_id, E, row_keys, N)
    b2 = trunc_bit_words(sess, C_TB2, call_id, E, row_keys, N)
    c, cp = trunc_coeffs(t, ell)
    sb1, sb2 = bit_sharings(sess, b1, b2)
    xs_p = sb1.map(lambda a: (a * c[None, :]) & mask)
    xs_q = sb1.map(lambda a: (a * cp[None, :]) & mask)
    rp1 = sess.prf(C_R1, P_TRUNC_P, obj, E)
    rp2 = sess.prf(C_R2, P_TRUNC_P, obj, E)
    gp1 = sess.prf(C_G1, P_TRUNC_P, obj, E)
    p, gamma_p = inner_rows(sess, xs_p, sb2, rp1, rp2, gp1, "trunc", OFFLINE, OFFLINE)
    rq1 = sess.prf(C_R1, P_TRUNC_Q, obj, E)
    rq2 = sess.prf(C_R2, P_TRUNC_Q, obj, E)
    gq1 = sess.prf(C_G1, P_TRUNC_Q, obj, E)
    q, gamma_q = inner_rows(sess, xs_q, sb2, rq1, rq2, gq1, "trunc", OFFLINE, OFFLINE)
    # <r_x> = sum_j 2^j (<b1_j> + <b2_j>) + <p>: components [r]_1 = -b1 + rp1, [r]_2 = -b2 + rp2
    a1, a2 = asr(b1, t), asr(b2, t)
    rx1_p1 = (p.p1_m + b1 - rp1) & mask        # m_{r_x} - [r_{r_x}]_1 at P1
    rx2_p2 = (b2 - rp2) & mask                 # -[r_{r_x}]_2 at P2
    rx1_p0 = (gamma_p + b1 - rp1) & mask       # P0 knows m_{r_x} = Gamma_p
    rx2_p0 = rx2_p2.copy()
    rz1_p1 = (q.p1_m + a1 - rq1) & mask
    rz2_p2 = (a2 - rq2) & mask
    rz1_p0 = (gamma_q + a1 - rq1) & mask
    rz2_p0 = rz2_p2.copy()
    return TruncPair(b1, b2, p, q, rx1_p0, rx2_p0, rx1_p1, rx2_p2, rz1_p0, rz2_p0, rz1_p1, rz2_p2)


# ---------------------------------------------------------------------------------------------
# Pi_Inner matrix product (+ Pi_Trunc^t)
# ---------------------------------------------------------------------------------------------
@dataclass
class MatmulResult:
    z_pre: Shared             # <X.W> with mask r_x of the trunc pair (or fresh [r_z])
    out: Shared               # truncated output (== z_pre when no truncation)
    tp: TruncPair | None


def matmul(sess: Session, X: Shared, W: Shared, call_id: int, trunc_bits: int | None = None,
           row_keys=None) -> MatmulResult:
    """Sec. 4.1 views the M x N product as M*N inner products of dimension K, each by Fig. DPP:
    offline P0 computes Gamma = R_X R_W + R_Z and shares it; online P1 computes
    [m_Z]_1 = -M_X [R_W]_1 - [R_X]_1 M_W + [Gamma]_1, P2 computes
    [m_Z]_2 = M_X M_W - M_X [R_W]_2 - [R_X]_2 M_W + [Gamma]_2, and they exchange.
    With truncation the output wire's mask R_Z is the trunc pair's r_x (Fig. trunc: "executed
    preferentially"), and the online truncation is m_out = m_Z >>_arith t."""
    mask = sess.mask
    M, K = X.p1_m.shape
    K2, N = W.p1_m.shape
    assert K == K2
    E = M * N
    obj = obj_id(call_id)
    tp = None
    if trunc_bits is None:
        r1 = sess.prf(C_R1, P_INNER, obj, E).reshape(M, N)
        r2 = sess.prf(C_R2, P_INNER, obj, E).reshape(M, N)
        m1_p0, m2_p0, m1_p1, m2_p2 = r1, r2, r1, r2
    else:
        tp = trunc_pair(sess, call_id, E, trunc_bits, row_keys, N)
        m1_p0, m2_p0 = tp.rx1_p0.reshape(M, N), tp.rx2_p0.reshape(M, N)
        m1_p1, m2_p2 = tp.rx1_p1.reshape(M, N), tp.rx2_p2.reshape(M, N)
    # offline, P0
    RX = (X.p0_r1 + X.p0_r2) & mask
    RW = (W.p0_r1 + W.p0_r2) & mask
    gamma = (np.matmul(RX, RW) + m1_p0 + m2_p0) & mask
    g1 = sess.prf(C_G1, P_INNER, obj, E).reshape(M, N)
    g2_at_p2 = _gamma_message(sess, gamma, g1, "inner", OFFLINE)
    # online
    mz1 = (U64(0) - np.matmul(X.p1_m, W.p1_r1) - np.matmul(X.p1_r1, W.p1_m) + g1) & mask
    mz2 = (np.matmul(X.p2_m, W.p2_m) - np.matmul(X.p2_m, W.p2_r2) - np.matmul(X.p2_r2, W.p2_m)
           + g2_at_p2) & mask
    mz_p1, mz_p2 = _exchange_mz(sess, mz1, mz2, "inner", ONLINE)
    z_pre = Shared(m1_p0.copy(), m2_p0.copy(), mz_p1, m1_p1.copy(), mz_p2, m2_p2.copy())
    if tp is None:
        return MatmulResult(z_pre, z_pre, None)
    t = trunc_bits
    out = Shared(tp.rz1_p0.reshape(M, N).copy(), tp.rz2_p0.reshape(M, N).copy(),
                 asr(mz_p1, t) & mask, tp.rz1_p1.reshape(M, N).copy(),
                 asr(mz_p2, t) & mask, tp.rz2_p2.reshape(M, N).copy())
    return MatmulResult(z_pre, out, tp)


# ---------------------------------------------------------------------------------------------
# Pi_Trunc^t of an existing sharing (reading T5)
# ---------------------------------------------------------------------------------------------
def trunc(sess: Session, x: Shared, call_id: int, t: int):
    """Fig. trunc on <x> of any mask: the pairs' preprocessing (6 l bits offline), the switch of
    the wire's mask to r_x (2 l bits online and two hashes), then m_z = m' >>_arith t.
    Returns (<z>, TruncPair)."""
    mask = sess.mask
    shape = x.p1_m.shape
    E = x.p1_m.size
    tp = trunc_pair(sess, call_id, E, t)
    f = lambda a: a.reshape(-1)
    d1 = (tp.rx1_p1 - f(x.p1_r1)) & mask              # P1
    d2 = (tp.rx2_p2 - f(x.p2_r2)) & mask              # P2
    d1_p0 = (tp.rx1_p0 - f(x.p0_r1)) & mask           # P0 knows both
    d2_p0 = (tp.rx2_p0 - f(x.p0_r2)) & mask
    d1_at_p2 = sess.send(1, 2, ONLINE, "trunc", d1, site="TRUNC_D1")
    d2_at_p1 = sess.send(2, 1, ONLINE, "trunc", d2)
    w = sess.wire
    h1_at_p2 = sess.send_hash(0, 2, ONLINE, "trunc", hash_u64(w(d1_p0)))
    h2_at_p1 = sess.send_hash(0, 1, ONLINE, "trunc", hash_u64(w(d2_p0)))
    if hash_u64(w(d2_at_p1)) != h2_at_p1:
        raise Abort("P1: d2 from P2 disagrees with H(d2) from P0")
    if hash_u64(w(d1_at_p2)) != h1_at_p2:
        raise Abort("P2: d1 from P1 disagrees with H(d1) from P0")
    m1 = (f(x.p1_m) + d1 + d2_at_p1) & mask           # m' = x + r_x at P1
    m2 = (f(x.p2_m) + d1_at_p2 + d2) & mask           # and at P2
    out = Shared(tp.rz1_p0.copy(), tp.rz2_p0.copy(), asr(m1, t) & mask, tp.rz1_p1.copy(),
                 asr(m2, t) & mask, tp.rz2_p2.copy())
    return out.map(lambda a: a.reshape(shape)), tp


# ---------------------------------------------------------------------------------------------
# convolution: one inner product per output (Sec. 4.1)
# ---------------------------------------------------------------------------------------------
def conv_out_size(H: int, W: int, kh: int, kw: int, stride: int, pad: int):
    return (H + 2 * pad - kh) // stride + 1, (W + 2 * pad - kw) // stride + 1


def im2col_rows(x, B: int, C: int, H: int, W: int, kh: int, kw: int, stride: int, pad: int):
    """The input of every output's inner product, from the definition of a convolution:
    row (b, i, j), column (c, di, dj) holds x[b, c, i stride + di - pad, j stride + dj - pad],
    0 outside the image.  x: (B, C, H, W) words (one share component)."""
    Ho, Wo = conv_out_size(H, W, kh, kw, stride, pad)
    out = np.zeros((B * Ho * Wo, C * kh * kw), dtype=np.uint64)
    for b in range(B):
        for i in range(Ho):
            for j in range(Wo):
                row = (b * Ho + i) * Wo + j
                for c in range(C):
                    for di in range(kh):
                        for dj in range(kw):
                            y, z = i * stride + di - pad, j * stride + dj - pad
                            if 0 <= y < H and 0 <= z < W:
                                out[row, (c * kh + di) * kw + dj] = x[b, c, y, z]
    return out


def conv2d(sess: Session, X: Shared, Wm: Shared, call_id: int, geom, trunc_bits: int | None = None):
    """Convolution of the NCHW sharing X (geom = (B, C, H, W, kh, kw, stride, pad)) with the
    weight sharing Wm of the (C kh kw) x C_out matrix (rows (c, di, dj)): every component is
    lowered to its im2col rows (a local, public rearrangement), then one Pi_Inner per output
    (``matmul``).  Output rows (b, i, j), columns c_out.  Returns (cols, MatmulResult)."""
    B, C, H, W, kh, kw, stride, pad = geom
    cols = X.map(lambda a: im2col_rows(a.reshape(B, C, H, W), B, C, H, W, kh, kw, stride, pad))
    return cols, matmul(sess, cols, Wm, call_id, trunc_bits)
