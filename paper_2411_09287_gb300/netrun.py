"""Pi_MultVerify^R under the paper's LAN / MAN / WAN settings: GPU computation measured, network
time from the protocol's message schedule (``netmodel``).

The paper picks R per network from runs that include both computation and communication.  One
GPU has no network, so a run here times the verification's work on the GPU (CUDA events around
mpc_verify_mult, every round's kernels and Pi_Rec reveals included) for each R, checks that the
messages it sent (the library's ledger) are exactly those ``netmodel`` prices, and adds the
network time of that message schedule: per dependent step one one-way delay plus its busiest
link's bytes over the bandwidth.  The computation of a round and its messages are sequential in
the protocol (each round's challenge depends on the previous round's messages), so the two times
add.

  python -m paper_2411_09287_gb300.netrun [--log2-D 18 20] [--R-max 16]
"""
from __future__ import annotations

import argparse
import hashlib
import json

import numpy as np

from . import netmodel as NM


def best_by_total(gpu_s: dict, D: int, net) -> tuple:
    """(R, seconds) minimising measured GPU seconds + network seconds (ties: smaller R)."""
    tot = {R: gpu_s[R] + NM.verify_time(D, R, net) for R in gpu_s}
    R = min(tot, key=lambda r: (tot[r], r))
    return R, tot[R]


def measure(mpc, D: int, Rs, reps: int = 3, seed: bytes = None):
    """GPU seconds of mpc_verify_mult on D triples for each R (median of reps); raises if a run's
    ledger differs from netmodel.verify_bytes / verify_messages."""
    import torch
    seed = seed or hashlib.sha256(f"netrun-{D}".encode()).digest()
    ctx = mpc.Context(seed)
    g = np.random.default_rng(D)
    x = g.integers(0, 2**64, D, dtype=np.uint64)
    y = g.integers(0, 2**64, D, dtype=np.uint64)
    xs, ys = ctx.share_input(1, x), ctx.share_input(2, y)
    zs = ctx.mult(3, xs, ys, D)
    vid = 100
    ctx.verify_mult(vid, xs, ys, zs, D, 3, R=Rs[0])   # warm-up
    out = {}
    for R in Rs:
        ts = []
        for _ in range(reps):
            vid += 1
            b0, m0 = ctx.ledger()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            rc, _ = ctx.verify_mult(vid, xs, ys, zs, D, 3, R=R)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            assert rc == mpc.MPC_OK
            b1, m1 = ctx.ledger()
            sent = sum(b1.values()) - sum(b0.values())
            if sent != NM.verify_bytes(D, R) or m1 - m0 != NM.verify_messages(R):
                raise AssertionError(f"D={D} R={R}: ledger {sent} B / {m1 - m0} messages, model "
                                     f"{NM.verify_bytes(D, R)} B / {NM.verify_messages(R)}")
            ts.append(e0.elapsed_time(e1) / 1e3)
        out[R] = float(np.median(ts))
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2-D", type=int, nargs="+", default=[18, 20])
    ap.add_argument("--R-max", type=int, default=16)
    a = ap.parse_args()
    from . import mpc
    res = {}
    for k in a.log2_D:
        D = 1 << k
        gpu = measure(mpc, D, list(range(0, a.R_max + 1)))
        rec = {"gpu_ms": {R: round(t * 1e3, 3) for R, t in gpu.items()}}
        for name, net in NM.NETWORKS.items():
            R, tot = best_by_total(gpu, D, net)
            rec[name] = {"best_R_measured": R, "total_ms": round(tot * 1e3, 2),
                         "best_R_comm_only": NM.best_R(D, net, a.R_max)}
        res[f"2^{k}"] = rec
    print(json.dumps(res))


if __name__ == "__main__":
    main()
