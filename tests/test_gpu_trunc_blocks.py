"""The blocked, compact, row-split and chunked evaluations of the truncation batch against the
oracle, through the C-ABI.

By default those code paths only run on layers of 65536 outputs and more, far beyond what the
oracle can check.  The context's tuning (mpc_set_tuning) moves their thresholds without changing
any protocol value, so small layers take them here:
  - trunc_block L = 128 or 256: the r^(2e) table in e_hi blocks (several blocks: the grouped
    table product; E a multiple of L on the tensor-core path: the compact table, its first-block
    limb GEMM and 12 nhi GR products);
  - row_split L': the folded-vector product of x_e = r^(2 L' e_hi) sum_j b_(e,j) r^(2 e_lo) V_j
    with its transposed bit rows, output row map and padded rows (out_lim), and, in compact mode,
    the rows r^(2 L' e_hi) gathered as T_hi[e / L] r^(2 (e mod L)) with e mod L != 0 (L = 384,
    L' = 256: e = 0, 256, 512); L' above L (the whole table of powers is kept);
  - tc_combine_min: sum_(e_hi) r^(2 L e_hi) S_hi on the tensor cores;
  - trunc_chunk: the batch split into independently verified chunks (reading C1), ragged last
    chunk included.
Each case compares the whole transcript of both batches (every revealed zeta', the six
components of <h(0)> and <h(p2)> of every round, the opened Delta of every chunk), the outcome,
the ledger and the opened output with the oracle, on both GEMM paths, and once with a faulted
truncation pair.
"""
import functools

import numpy as np
import pytest

from oracle import protocols as OP
from oracle import verify as OV
from oracle.shares import Session
from paper_2411_09287_gb300 import workloads
from test_gpu_parity import check_trace, ledger_of, seed_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


CASES = {
    # name: (M, N, K, tuning)
    "compact-2blocks-tccombine": (16, 16, 16, dict(trunc_block=128, tc_combine_min=2)),
    "ragged-2blocks": (10, 20, 8, dict(trunc_block=128)),
    "compact-rowsplit-offset": (24, 32, 8, dict(trunc_block=384, row_split=256, tc_combine_min=2)),
    "rowsplit-above-block": (16, 16, 8, dict(trunc_block=128, row_split=384)),
    "chunks-ragged": (15, 20, 8, dict(trunc_block=128, trunc_chunk=128)),
}


def _inputs(name):
    M, N, K, _ = CASES[name]
    g = workloads.rng(f"tblk-{name}")
    X = OP.encode_fixed(g.uniform(-4, 4, (M, K)), 13)
    W = OP.encode_fixed(g.uniform(-4, 4, (K, N)), 13)
    return X, W


@functools.lru_cache(maxsize=None)
def _oracle(name, fault_out):
    """The oracle's run of a case (independent of the GEMM path): transcript, outcome, ledger and
    opened output."""
    M, N, K, tune = CASES[name]
    X, W = _inputs(name)
    sess = Session(seed_of(f"tblk-{name}"))
    ox, ow = OP.share_input(sess, X, 1), OP.share_input(sess, W, 2)
    if fault_out is not None:
        sess.arm_fault("GAMMA2", fault_out, 1 << 7)
    res = OP.matmul(sess, ox, ow, 3, trunc_bits=13)
    otr = []
    ok = OV.matmul_verify(sess, ox, ow, res, 4, 13, trace=otr, trunc_chunk=tune.get("trunc_chunk"))
    ledger = ledger_of(sess)   # before the output's Pi_Rec, like the GPU side's
    out = OP.reconstruct(sess, res.out).reshape(-1) if ok else None
    return otr, ok, ledger, out


def _run(mpc, name, path, fault_out=None):
    M, N, K, tune = CASES[name]
    t = 13
    X, W = _inputs(name)
    ctx = mpc.Context(seed_of(f"tblk-{name}"), gemm_path=path, tuning=tune)
    gx, gw = ctx.share_input(1, X), ctx.share_input(2, W)
    if fault_out is not None:   # P0 -> P2 [Gamma]_2 of the first trunc-pair inner product
        ctx.inject_fault("GAMMA2", fault_out, 1 << 7)
    zpre, zout, pq = ctx.matmul(3, gx, gw, M, N, K, t)
    rc, tr = ctx.verify_matmul(4, gx, gw, zpre, pq, M, N, K, t, 3, trace=True)
    otr, ok, oledger, oout = _oracle(name, fault_out)
    chunk = tune.get("trunc_chunk")
    Rs = [mpc.default_R(K)] + [mpc.default_R(64 * (e1 - e0))
                               for e0, e1 in OV.trunc_chunks(M * N, chunk)]
    assert tr.numel() == sum(R + 1 for R in Rs) * mpc.TRACE_ROUND
    check_trace(mpc, tr, otr, Rs)
    g, _ = ctx.ledger()
    for key in set(g) | set(oledger):
        assert g.get(key, 0) == oledger.get(key, 0), (key, g.get(key, 0), oledger.get(key, 0))
    return ctx, rc, ok, zout, oout


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_blocked_trunc_batch_transcript_matches_oracle(mpc, name, path):
    ctx, rc, ok, zout, oout = _run(mpc, name, path)
    assert ok and rc == mpc.MPC_OK
    M, N = CASES[name][:2]
    out = ctx.reconstruct(zout, M * N)
    assert np.array_equal(out, oout)


@pytest.mark.parametrize("path", [0, 1])
def test_blocked_trunc_batch_rejects_a_faulty_pair(mpc, path):
    """A corrupted [Gamma]_2 of output 150's trunc pair: the chunk holding it (outputs 128..255)
    opens Delta != 0, exactly as the oracle's does, and the layer is rejected."""
    ctx, rc, ok, _, _ = _run(mpc, "chunks-ragged", path, fault_out=150)
    assert not ok
    assert rc == mpc.MPC_ERR_VERIFY
    assert ctx.status() == mpc.MPC_ERR_ABORT


def test_tuning_round_trip_and_range(mpc):
    ctx = mpc.Context(seed_of("tune"))
    d = ctx.tuning()
    assert d["trunc_block"] == 65536 and d["trunc_chunk"] == 1 << 24 and d["row_split"] == 0
    ctx.set_tuning(trunc_block=256, row_split=384)
    d2 = ctx.tuning()
    assert d2["trunc_block"] == 256 and d2["row_split"] == 384 and d2["tc_combine_min"] == 32
    for bad in (dict(trunc_block=100), dict(trunc_block=131072), dict(row_split=64 + 1),
                dict(trunc_chunk=-1)):
        with pytest.raises(mpc.MpcError):
            ctx.set_tuning(**bad)
    # more than 15 chunks cannot be planned
    ctx.set_tuning(trunc_chunk=10)
    with pytest.raises(mpc.MpcError):
        ctx.ws_size(mpc.OP_VERIFY_MATMUL, 16, 16, 8, 13)


# every variant of the GR-matrix product kernel (the autotuner's candidates) on a blocked, compact
# and a chunked batch: register producers (8 and 16 drain warps), TMA producers with 16 drain
# warps, A in tensor memory
GR_VARIANTS = [dict(gr_producers=1), dict(gr_producers=1, gr_drain_warps=16),
               dict(gr_producers=2, gr_drain_warps=16), dict(gr_producers=3),
               # the autotuner's other knobs, away from their defaults
               dict(gemm_split_min=2, gram_split=19, fold_batch_max=1 << 20)]


@pytest.mark.parametrize("variant", range(len(GR_VARIANTS)))
@pytest.mark.parametrize("name", ["compact-2blocks-tccombine", "chunks-ragged"])
def test_gr_product_variants_match_oracle(mpc, name, variant):
    M, N, K, tune = CASES[name]
    saved = dict(tune)
    try:
        tune.update(GR_VARIANTS[variant])
        ctx, rc, ok, zout, oout = _run(mpc, name, 1)
    finally:
        tune.clear()
        tune.update(saved)
    assert ok and rc == mpc.MPC_OK
    assert np.array_equal(ctx.reconstruct(zout, M * N), oout)
