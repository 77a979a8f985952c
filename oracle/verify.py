"""Batched verification over GR(2^l, d) (oracle; test infrastructure only).

* ``reveal_random_gr``  <r>^{l[x]} <- Pi_<.>^{l[x]} (random) followed by Pi_Rec (Fig. MTP, Fig.
                        Reduce).
* ``secure_inner_gr``   Pi_Inner over GR: the semi-honest inner product of Sec. 2 run on
                        <.>^{l[x]} sharings (used for h(0), h(2) in Fig. Reduce and for Delta in
                        Fig. DPV).
* ``secure_mult_gr``    Pi_Mult over GR (x'_i = x_i * alpha in Fig. DPV).
* ``reduce_round``      Pi_Reduce (Fig. Reduce).
* ``inner_verify``      Pi_InnerVerify (Fig. DPV).
* ``bi_verify``         Pi_Reduce applied R times, then Pi_InnerVerify (Fig. PPEV / Fig. PBDP).
* ``tran_mult``         Pi_Tran for Pi_Mult triples (Fig. MTP).
* ``tran_matmul_rank1`` consolidation of a matrix product's M*N inner products (Fig. PBDP) in the
                        rank-1 form sum_k Xt_k Wt_k (reading V1); ``tran_matmul_literal`` is the
                        literal M*N*K-dimensional consolidation, for tiny shapes.
* ``tran_trunc``        consolidation of the trunc pairs' 2E inner products of dimension l; the two
                        inner products of one output share their y vector and are merged
                        (reading V1t); ``tran_trunc_literal`` is the unmerged 2*l*E form.
* ``trunc_chunks``      the split of a layer's trunc batch into independently verified chunks of
                        consecutive outputs (reading C1); ``trunc_verify`` runs them.

Readings of the paper (where it is silent, ambiguous or garbled):
  A4  lifting pads with zero coefficients (Fig. MTP text).
  A5  r, zeta', alpha are <.>^{l[x]}-random from the pairwise streams; r and zeta' are revealed
      with Pi_Rec, alpha is not.
  A6/X The interpolation of Fig. Reduce divides by 2, which is not invertible in GR(2^l, d).
      mode "zeta2": points 0, 1, 2 and evaluation point zeta = 2 zeta', whose Lagrange weights
      L0 = (2z'-1)(z'-1), L1 = 4z'(1-z'), L2 = z'(2z'-1) are integral.
      mode "x" (default): points 0, 1, x (x the ring's generator; x and 1-x are units), any
      zeta, L0 = (z-1)(z-x)/x, L1 = z(z-x)/(1-x), L2 = z(z-1)/(x(x-1)).  Mode "zeta2" accepts every
      error that is a multiple of 2^(l-2) in z (L1 is always a multiple of 4); the tests show it.
  A7  the consolidation weight of triple i is r^i, with row-major (a, b) -> a N + b.
  A8  R = max(0, ceil(log2 D) - 6) unless given.
  C1  A layer's trunc batch may be split into chunks of at most C consecutive outputs (row-major
      e = a N + b).  Chunk i is a Pi_BIVerify batch of its own (Fig. PBDP): its own challenge r
      from the streams of batch 1 + i, weights r^(2e') and r^(2e'+1) over the chunk-local index
      e' = e - e0, its own R (default from its dimension 64 E_i).  The paper verifies a batch of
      |G| inner products with error at most |G| / 2^(d-R-2) (Thm. multvv); split batches each
      keep that bound for their own |G_i|, and a union bound over the chunks gives the layer's.
  Odd length in Pi_Reduce: one (0, 0) pair is appended.
Parity: pinned by completeness (honest runs give Delta = 0), rejection of injected errors, brute
force over every challenge on tiny rings against the bounds of Lemma transl / polyred / polyvv,
Lagrange identities, and literal-vs-consolidated agreement (tests/test_oracle_verify.py).
"""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np

from .galois import GR
from .protocols import Abort, bit_sharings, reconstruct, trunc_coeffs
from .shares import (C_G1, C_M12, C_R1, C_R2, P_VER_ALPHA, P_VER_DELTA, P_VER_H0, P_VER_H2,
                     P_VER_R, P_VER_XA, P_VER_ZETA, VERIFY, Session, Shared, obj_id,
                     shared_concat)

U64 = np.uint64


def default_R(D: int) -> int:
    return max(0, math.ceil(math.log2(D)) - 6) if D > 1 else 0


# ---------------------------------------------------------------------------------------------
# share-level helpers (public GR constants act on every component)
# ---------------------------------------------------------------------------------------------
def cmul(gr: GR, c, s: Shared) -> Shared:
    return s.map(lambda a: gr.mul(c, a))


def sadd(gr: GR, a: Shared, b: Shared) -> Shared:
    return a.zip(b, gr.add)


def ssub(gr: GR, a: Shared, b: Shared) -> Shared:
    return a.zip(b, gr.sub)


def lift_shared(gr: GR, s: Shared) -> Shared:
    return s.map(gr.lift)


def random_gr_shared(sess: Session, purpose: int, obj: int, n: int = None) -> Shared:
    """Pi_<.>^{l[x]} of a random value: [.]_1 from eta01, [.]_2 from eta02, m from eta12.
    Tests may fix the shared value through ``sess.forced[(purpose, obj)]`` (brute force over all
    challenges); m is then chosen so that m - [.]_1 - [.]_2 equals the forced value."""
    r1 = sess.prf_gr(C_R1, purpose, obj, n)
    r2 = sess.prf_gr(C_R2, purpose, obj, n)
    m = sess.prf_gr(C_M12, purpose, obj, n)
    if (purpose, obj) in sess.forced:
        m = sess.gr.add(sess.gr.add(np.asarray(sess.forced[(purpose, obj)], dtype=U64), r1), r2)
    return Shared(r1, r2.copy(), m, r1.copy(), m.copy(), r2)


def reveal_random_gr(sess: Session, purpose: int, obj: int) -> np.ndarray:
    s = random_gr_shared(sess, purpose, obj)
    return reconstruct(sess, s, VERIFY, "verify")


# ---------------------------------------------------------------------------------------------
# Pi_Inner / Pi_Mult over GR
# ---------------------------------------------------------------------------------------------
def _gr_sum(gr: GR, a):
    return gr.sum(a, axis=0) if a.shape[0] else gr.zeros()


def secure_inner_gr(sess: Session, x: Shared, y: Shared, purpose: int, obj: int) -> Shared:
    """<h> = <sum_i x_i y_i> over GR: output mask [r_h] from the (purpose, obj) streams,
    Gamma = sum_i r_{x_i} r_{y_i} + r_h shared by P0 with Pi_[.], cross terms by P1 and P2, one
    exchange of m shares (Fig. DPP over GR(2^l, d))."""
    gr = sess.gr
    rh1 = sess.prf_gr(C_R1, purpose, obj)
    rh2 = sess.prf_gr(C_R2, purpose, obj)
    g1 = sess.prf_gr(C_G1, purpose, obj)
    rx = gr.add(x.p0_r1, x.p0_r2)
    ry = gr.add(y.p0_r1, y.p0_r2)
    gamma = gr.add(gr.add(_gr_sum(gr, gr.mul(rx, ry)), rh1), rh2)
    g2_at_p2 = sess.send(0, 2, VERIFY, "verify", gr.sub(gamma, g1))
    mz1 = gr.add(gr.neg(_gr_sum(gr, gr.add(gr.mul(x.p1_m, y.p1_r1), gr.mul(y.p1_m, x.p1_r1)))), g1)
    t2 = gr.sub(gr.sub(gr.mul(x.p2_m, y.p2_m), gr.mul(x.p2_m, y.p2_r2)), gr.mul(y.p2_m, x.p2_r2))
    mz2 = gr.add(_gr_sum(gr, t2), g2_at_p2)
    mz1_at_p2 = sess.send(1, 2, VERIFY, "verify", mz1)
    mz2_at_p1 = sess.send(2, 1, VERIFY, "verify", mz2)
    return Shared(rh1, rh2, gr.add(mz1, mz2_at_p1), rh1.copy(), gr.add(mz1_at_p2, mz2), rh2.copy())


def secure_mult_gr(sess: Session, x: Shared, a: Shared, purpose: int, obj: int) -> Shared:
    """<x_i * a> for every i over GR (Fig. MultP over GR(2^l, d)); element i's mask and
    [Gamma]_1 are words i*d + c of the (purpose, obj) streams."""
    gr = sess.gr
    n = x.p1_m.shape[0]
    rz1 = sess.prf_gr(C_R1, purpose, obj, n)
    rz2 = sess.prf_gr(C_R2, purpose, obj, n)
    g1 = sess.prf_gr(C_G1, purpose, obj, n)
    rx = gr.add(x.p0_r1, x.p0_r2)
    ra = gr.add(a.p0_r1, a.p0_r2)
    gamma = gr.add(gr.add(gr.mul(rx, ra), rz1), rz2)
    g2_at_p2 = sess.send(0, 2, VERIFY, "verify", gr.sub(gamma, g1))
    mz1 = gr.add(gr.neg(gr.add(gr.mul(x.p1_m, a.p1_r1), gr.mul(a.p1_m, x.p1_r1))), g1)
    t2 = gr.sub(gr.sub(gr.mul(x.p2_m, a.p2_m), gr.mul(x.p2_m, a.p2_r2)), gr.mul(a.p2_m, x.p2_r2))
    mz2 = gr.add(t2, g2_at_p2)
    mz1_at_p2 = sess.send(1, 2, VERIFY, "verify", mz1)
    mz2_at_p1 = sess.send(2, 1, VERIFY, "verify", mz2)
    return Shared(rz1, rz2, gr.add(mz1, mz2_at_p1), rz1.copy(), gr.add(mz1_at_p2, mz2), rz2.copy())


# ---------------------------------------------------------------------------------------------
# Lagrange weights of Fig. Reduce (readings A6 / X)
# ---------------------------------------------------------------------------------------------
def third_point(gr: GR, mode: str):
    return gr.const(2) if mode == "zeta2" else gr.x()


def lagrange(gr: GR, zeta_prime, mode: str):
    """Returns (evaluation point zeta, L0, L1, L2) with h(zeta) = L0 h(0) + L1 h(1) + L2 h(p2)."""
    one = gr.const(1)
    if mode == "zeta2":
        z = zeta_prime
        zeta = gr.add(z, z)
        two_z = zeta
        L0 = gr.mul(gr.sub(two_z, one), gr.sub(z, one))
        L1 = gr.mul(gr.const(4), gr.mul(z, gr.sub(one, z)))
        L2 = gr.mul(z, gr.sub(two_z, one))
        return zeta, L0, L1, L2
    x = gr.x()
    zeta = zeta_prime
    L0 = gr.mul(gr.mul(gr.sub(zeta, one), gr.sub(zeta, x)), gr.inv(x))
    L1 = gr.mul(gr.mul(zeta, gr.sub(zeta, x)), gr.inv(gr.sub(one, x)))
    L2 = gr.mul(gr.mul(zeta, gr.sub(zeta, one)), gr.inv(gr.mul(x, gr.sub(x, one))))
    return zeta, L0, L1, L2


def fold(gr: GR, zeta, v0: Shared, v1: Shared) -> Shared:
    """f_i(zeta) = zeta f_i(1) - (zeta - 1) f_i(0) = (1 - zeta) f_i(0) + zeta f_i(1)."""
    one_minus = gr.sub(gr.const(1), zeta)
    return sadd(gr, cmul(gr, one_minus, v0), cmul(gr, zeta, v1))


# ---------------------------------------------------------------------------------------------
# Pi_Reduce, Pi_InnerVerify, batch driver
# ---------------------------------------------------------------------------------------------
def reduce_round(sess: Session, x: Shared, y: Shared, z: Shared, call_id: int, batch: int,
                 k: int, trace: list | None = None):
    """Fig. Reduce, round k (1-based): from a D-dimensional claim (x, y, z) to a
    ceil(D/2)-dimensional one."""
    gr = sess.gr
    D = x.p1_m.shape[0]
    if D % 2:
        zero = Shared(*(gr.zeros((1,)) for _ in range(6)))
        x = shared_concat([x, zero])
        y = shared_concat([y, zero])
    f0, f1 = x[0::2], x[1::2]
    g0, g1 = y[0::2], y[1::2]
    p2 = third_point(gr, sess.reduce_mode)
    fp = fold(gr, p2, f0, f1)   # f_i(p2) = (1 - p2) f_i(0) + p2 f_i(1)
    gp = fold(gr, p2, g0, g1)
    obj = obj_id(call_id, batch, k)
    h0 = secure_inner_gr(sess, f0, g0, P_VER_H0, obj)
    h2 = secure_inner_gr(sess, fp, gp, P_VER_H2, obj)
    h1 = ssub(gr, z, h0)
    zeta_prime = reveal_random_gr(sess, P_VER_ZETA, obj)
    zeta, L0, L1, L2 = lagrange(gr, zeta_prime, sess.reduce_mode)
    z_new = sadd(gr, sadd(gr, cmul(gr, L0, h0), cmul(gr, L1, h1)), cmul(gr, L2, h2))
    if trace is not None:
        trace.append(dict(round=k, h0=h0, h2=h2, zeta_prime=zeta_prime))
    return fold(gr, zeta, f0, f1), fold(gr, zeta, g0, g1), z_new


def inner_verify(sess: Session, x: Shared, y: Shared, z: Shared, call_id: int, batch: int,
                 trace: list | None = None) -> bool:
    """Fig. DPV: alpha random (not revealed); x'_i = x_i alpha (secure mult);
    Delta = sum_i x'_i y_i - alpha z as one secure inner product of dimension D + 1;
    Delta = Pi_Rec(<Delta>); output 1 iff Delta = 0."""
    gr = sess.gr
    obj = obj_id(call_id, batch, 0)
    alpha = random_gr_shared(sess, P_VER_ALPHA, obj)
    xa = secure_mult_gr(sess, x, alpha, P_VER_XA, obj)
    lhs = shared_concat([xa, alpha.map(lambda a: a[None, :])])
    rhs = shared_concat([y, z.map(lambda a: gr.neg(a)[None, :])])
    delta_sh = secure_inner_gr(sess, lhs, rhs, P_VER_DELTA, obj)
    delta = reconstruct(sess, delta_sh, VERIFY, "verify")
    if trace is not None:
        trace.append(dict(delta=delta))
    return not np.any(delta)


def bi_verify(sess: Session, x: Shared, y: Shared, z: Shared, call_id: int, batch: int,
              R: int | None = None, trace: list | None = None) -> bool:
    """Fig. PPEV / Fig. PBDP after consolidation: R rounds of Pi_Reduce, then Pi_InnerVerify."""
    D = x.p1_m.shape[0]
    if R is None:
        R = default_R(D)
    for k in range(1, R + 1):
        x, y, z = reduce_round(sess, x, y, z, call_id, batch, k, trace)
    return inner_verify(sess, x, y, z, call_id, batch, trace)


def challenge_r(sess: Session, call_id: int, batch: int) -> np.ndarray:
    """<r>^{l[x]} random, revealed with Pi_Rec (Fig. MTP preprocessing + first online step)."""
    return reveal_random_gr(sess, P_VER_R, obj_id(call_id, batch, 0))


# ---------------------------------------------------------------------------------------------
# consolidations (Pi_Tran and Pi_BIVerify's first steps)
# ---------------------------------------------------------------------------------------------
def tran_mult(sess: Session, X: Shared, Y: Shared, Z: Shared, r) -> tuple:
    """Fig. MTP: lift; x'_i = r^i x_i; z = sum_i r^i z_i; y unchanged."""
    gr = sess.gr
    n = X.p1_m.size
    pw = gr.powers(r, n)
    xs = X.map(lambda a: gr.scale(pw, a.reshape(-1)))
    ys = lift_shared(gr, Y.map(lambda a: a.reshape(-1)))
    zs = Z.map(lambda a: _gr_sum(gr, gr.scale(pw, a.reshape(-1))))
    return xs, ys, zs


def tran_matmul_rank1(sess: Session, X: Shared, W: Shared, Z: Shared, r) -> tuple:
    """Fig. PBDP for the M*N inner products of Z = X W, with triple (a, b) weighted by r^(aN+b).
    Because r^(aN+b) = rho^a r^b with rho = r^N, the consolidated relation
    sum_{a,b,k} r^(aN+b) X_ak W_kb = sum_{a,b} r^(aN+b) Z_ab equals
    sum_k Xt_k Wt_k = zt with Xt_k = sum_a rho^a X_ak, Wt_k = sum_b r^b W_kb (reading V1)."""
    gr = sess.gr
    M, K = X.p1_m.shape
    N = W.p1_m.shape[1]
    Q = gr.powers(r, N)                   # r^b
    rho = gr.pow(r, N)
    P = gr.powers(rho, M)                 # rho^a
    mask = gr.mask
    xt = X.map(lambda a: np.matmul(a.T, P) & mask)          # (K, d)
    wt = W.map(lambda a: np.matmul(a, Q) & mask)            # (K, d)
    zt = Z.map(lambda a: _gr_sum(gr, gr.mul(P, np.matmul(a, Q) & mask)))
    return xt, wt, zt


def tran_matmul_literal(sess: Session, X: Shared, W: Shared, Z: Shared, r) -> tuple:
    """Fig. PBDP literally: one vector of dimension M*N*K, entry ((aN+b)K + k) being
    (r^(aN+b) X_ak, W_kb), and z = sum r^(aN+b) Z_ab."""
    gr = sess.gr
    M, K = X.p1_m.shape
    N = W.p1_m.shape[1]
    pw = gr.powers(r, M * N).reshape(M, N, gr.d)
    xs = X.map(lambda a: gr.scale(pw[:, :, None, :], np.broadcast_to(a[:, None, :], (M, N, K)))
               .reshape(M * N * K, gr.d))
    ys = W.map(lambda a: gr.lift(np.broadcast_to(a.T[None, :, :], (M, N, K))).reshape(-1, gr.d))
    zs = Z.map(lambda a: _gr_sum(gr, gr.scale(pw.reshape(-1, gr.d), a.reshape(-1))))
    return xs, ys, zs


def trunc_u(sess: Session, r, t: int):
    """u_j = c_j + r c'_j: the merged weight of bit product j of one output (reading V1t)."""
    gr = sess.gr
    c, cp = trunc_coeffs(t, gr.ell)
    return gr.add(gr.lift(c), gr.scale(r[None, :], cp))


def tran_trunc(sess: Session, tp, r, t: int) -> tuple:
    """Consolidation of the trunc pairs.  Output e contributes two inner products of dimension l,
    (c_j <b1_j>, <b2_j>) -> <p_e> weighted by r^(2e) and (c'_j <b1_j>, <b2_j>) -> <q_e> weighted
    by r^(2e+1).  They share y, so sum_j (r^(2e) c_j + r^(2e+1) c'_j) b1_j b2_j
    = r^(2e) (p_e + r q_e): one entry per (e, j) at index l*e + j with x = r^(2e) u_j <b1_j>."""
    gr = sess.gr
    E = tp.b1.shape[0]
    u = trunc_u(sess, r, t)                                   # (l, d)
    r2 = gr.mul(r, r)
    pw = gr.powers(r2, E)                                     # r^(2e)
    kappa = gr.mul(pw[:, None, :], u[None, :, :])             # (E, l, d)
    sb1, sb2 = bit_sharings(sess, tp.b1, tp.b2)
    xs = sb1.map(lambda a: gr.scale(kappa, a).reshape(E * gr.ell, gr.d))
    ys = sb2.map(lambda a: gr.lift(a).reshape(E * gr.ell, gr.d))
    zp = tp.p.map(lambda a: gr.scale(pw, a.reshape(-1)))
    zq = tp.q.map(lambda a: gr.scale(pw, a.reshape(-1)))
    zs = zp.zip(zq, lambda a, b: _gr_sum(gr, gr.add(a, gr.mul(r, b))))
    return xs, ys, zs


def tran_trunc_literal(sess: Session, tp, r, t: int) -> tuple:
    """Unmerged: index (2e) l + j holds (r^(2e) c_j <b1_j>, <b2_j>); index (2e+1) l + j holds
    (r^(2e+1) c'_j <b1_j>, <b2_j>); z = sum_e r^(2e) p_e + r^(2e+1) q_e."""
    gr = sess.gr
    E = tp.b1.shape[0]
    c, cp = trunc_coeffs(t, gr.ell)
    pw = gr.powers(r, 2 * E)
    sb1, sb2 = bit_sharings(sess, tp.b1, tp.b2)
    cc = np.stack([np.broadcast_to(c, (E, gr.ell)), np.broadcast_to(cp, (E, gr.ell))], axis=1)
    w = gr.scale(pw.reshape(E, 2, 1, gr.d), cc)               # (E, 2, l, d)
    xs = sb1.map(lambda a: gr.mul(w, gr.lift(a)[:, None, :, :]).reshape(2 * E * gr.ell, gr.d))
    ys = sb2.map(lambda a: np.broadcast_to(gr.lift(a)[:, None], (E, 2, gr.ell, gr.d))
                 .reshape(2 * E * gr.ell, gr.d).copy())
    zs = tp.p.zip(tp.q, lambda a, b: _gr_sum(gr, gr.add(
        gr.scale(pw[0::2], a.reshape(-1)), gr.scale(pw[1::2], b.reshape(-1)))))
    return xs, ys, zs


def trunc_chunks(E: int, chunk: int | None) -> list:
    """Reading C1: the output ranges [e0, e1) of the chunks of a trunc batch of E outputs (one
    range when chunk is None or at least E)."""
    C = E if chunk is None else min(E, int(chunk))
    return [(e0, min(E, e0 + C)) for e0 in range(0, E, C)]


def trunc_chunk_pairs(tp, e0: int, e1: int) -> SimpleNamespace:
    """The bits and <p>, <q> of outputs e0 .. e1-1 of a layer's trunc pairs."""
    return SimpleNamespace(b1=tp.b1.reshape(-1)[e0:e1], b2=tp.b2.reshape(-1)[e0:e1],
                           p=tp.p.map(lambda a: a.reshape(-1)[e0:e1]),
                           q=tp.q.map(lambda a: a.reshape(-1)[e0:e1]))


# ---------------------------------------------------------------------------------------------
# protocol-level entry points
# ---------------------------------------------------------------------------------------------
BATCH_MAIN, BATCH_TRUNC = 0, 1
MAX_TRUNC_CHUNKS = 15   # batch ids 1 .. 15 of the object-id layout


def trunc_verify(sess: Session, tp, call_id: int, t: int, R: int | None = None,
                 chunk: int | None = None, literal: bool = False, trace=None) -> list:
    """Pi_BIVerify of a layer's trunc pairs, chunk by chunk (reading C1); one bool per chunk."""
    E = tp.b1.size
    parts = trunc_chunks(E, chunk)
    assert len(parts) <= MAX_TRUNC_CHUNKS
    oks = []
    for i, (e0, e1) in enumerate(parts):
        batch = BATCH_TRUNC + i
        part = trunc_chunk_pairs(tp, e0, e1)
        r_t = challenge_r(sess, call_id, batch)
        if literal:
            xs, ys, zs = tran_trunc_literal(sess, part, r_t, t)
        else:
            xs, ys, zs = tran_trunc(sess, part, r_t, t)
        oks.append(bi_verify(sess, xs, ys, zs, call_id, batch, R, trace))
    return oks


def mult_verify(sess: Session, X: Shared, Y: Shared, Z: Shared, call_id: int,
                R: int | None = None, trace=None) -> bool:
    """Pi_MultVerify^R (Fig. PPEV) of the Pi_Mult triples (X_i, Y_i, Z_i)."""
    r = challenge_r(sess, call_id, BATCH_MAIN)
    xs, ys, zs = tran_mult(sess, X, Y, Z, r)
    return bi_verify(sess, xs, ys, zs, call_id, BATCH_MAIN, R, trace)


def matmul_verify(sess: Session, X: Shared, W: Shared, res, call_id: int, t: int | None,
                  R_main: int | None = None, R_trunc: int | None = None,
                  literal: bool = False, trace=None, trunc_chunk: int | None = None) -> bool:
    """Pi_BIVerify (Fig. PBDP) of one matrix-product layer: the M*N inner products of the
    product (batch 0) and, with truncation, the 2*M*N inner products of its trunc pairs
    (batch 1, or batches 1, 2, ... of at most trunc_chunk outputs each, reading C1).  Returns
    True iff every batch verifies."""
    r = challenge_r(sess, call_id, BATCH_MAIN)
    if literal:
        xs, ys, zs = tran_matmul_literal(sess, X, W, res.z_pre, r)
    else:
        xs, ys, zs = tran_matmul_rank1(sess, X, W, res.z_pre, r)
    ok = bi_verify(sess, xs, ys, zs, call_id, BATCH_MAIN, R_main, trace)
    if res.tp is not None:
        ok = all(trunc_verify(sess, res.tp, call_id, t, R_trunc, trunc_chunk, literal,
                              trace)) and ok
    return ok


__all__ = ["Abort", "bi_verify", "challenge_r", "default_R", "inner_verify", "lagrange",
           "matmul_verify", "mult_verify", "reduce_round", "secure_inner_gr", "secure_mult_gr",
           "tran_matmul_literal", "tran_matmul_rank1", "tran_mult", "tran_trunc",
           "tran_trunc_literal", "trunc_chunk_pairs", "trunc_chunks", "trunc_u", "trunc_verify"]
