"""Secure inference of a fully connected ReLU network through libmpc3 (config C2 shape:
784-128-128-10 at 13 fractional bits).

P0 owns the inputs and the weights (reading A13) and shares them (Pi_<.>).  Each layer is one
Pi_Inner matrix product with Pi_Trunc^13 (Sec. 4.1-4.2) followed, except after the last layer, by
a ReLU (Sec. 4.3); every layer is verified before the next one uses its output (reading A14), and
only the logits are opened (Pi_Rec).  All protocol work runs in libmpc3's kernels; this module
only sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import mpc as M


def mlp_weights(sizes, seed_name: str, std: float = 0.05):
    """Synthetic weights N(0, std^2) (numpy PCG64 from the named seed), one matrix per layer."""
    from .workloads import rng
    g = rng(seed_name)
    return [g.normal(0.0, std, (sizes[i], sizes[i + 1])) for i in range(len(sizes) - 1)]


def fp64_forward(x, weights):
    """The plaintext model in float64 (ReLU after every layer but the last)."""
    h = np.asarray(x, dtype=np.float64)
    for i, w in enumerate(weights):
        h = h @ w
        if i + 1 < len(weights):
            h = np.maximum(h, 0.0)
    return h


def quantized(x, k: int):
    """The values the fixed-point encoding of Sec. 2 represents (floor(x 2^k) / 2^k), for the
    float64 reference model."""
    return np.floor(np.asarray(x, dtype=np.float64) * float(1 << k)) / float(1 << k)


def share_weights(ctx: "M.Context", weights, k: int = 13, call_base: int = 900):
    """P0 shares the weight matrices once (mpc_share_fixed); the sharings serve any number of
    forward passes."""
    return [ctx.share_fixed(call_base + i, np.ascontiguousarray(w, dtype=np.float64).reshape(-1), k)
            for i, w in enumerate(weights)]


def secure_forward(ctx: "M.Context", x, weights, k: int = 13, call_base: int = 1000,
                   shared_weights=None, segments=None):
    """Secure forward pass.  x: (B, n0) float inputs; weights: list of (n_i, n_{i+1}) float
    matrices, shared by P0 (mpc_share_fixed) unless shared_weights already holds their sharings.
    segments: [(request id, images), ...] of a packed batch; the truncation bits of every layer
    are then keyed by (request, layer, row) so that each request opens to the logits it would
    get alone.  Returns the opened logits (B, n_last) as float64 (mpc_reconstruct_fixed)."""
    B = x.shape[0]
    cid = call_base
    h = ctx.share_fixed(cid, np.ascontiguousarray(x, dtype=np.float64).reshape(-1), k)
    cid += 1
    for i, w in enumerate(weights):
        n_in, n_out = w.shape
        gw = (shared_weights[i] if shared_weights is not None
              else ctx.share_fixed(cid, np.ascontiguousarray(w, dtype=np.float64).reshape(-1), k))
        keys = M.segment_row_keys(segments, i, 1) if segments is not None else None
        zpre, zout, pq = ctx.matmul(cid + 1, h, gw, B, n_out, n_in, k, row_keys=keys)
        rc, _ = ctx.verify_matmul(cid + 2, h, gw, zpre, pq, B, n_out, n_in, k, cid + 1,
                                  row_keys=keys)
        if rc != M.MPC_OK:
            raise M.MpcError(rc, f"layer {i}: verification rejected")
        h = zout
        cid += 3
        if i + 1 < len(weights):
            rc, h, _ = ctx.relu(cid, cid + 1, h, B * n_out)
            if rc != M.MPC_OK:
                raise M.MpcError(rc, f"layer {i}: ReLU verification rejected")
            cid += 2
    n_last = weights[-1].shape[1]
    return ctx.reconstruct_fixed(h, B * n_last, k).reshape(B, n_last)
