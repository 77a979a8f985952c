"""Secure CNN inference through libmpc3 (config C4; geometry of reading A17):
  Net A: 28x28x1 input, conv 5x5x16, 2x2 max-pool, conv 5x5x16, 2x2 max-pool, FC 256-100-10;
  Net B: 32x32x3 input, VGG-style: conv 3x3 pad 1 to 64, 64 (pool), 128, 128 (pool), 256 (pool)
  channels, flatten 4096, FC 512, FC 10; ReLU after every conv and FC but the last.  The channel
  widths of Net B are our reading: the pools take 32x32 to 4x4, so 4096 = 256 x 4 x 4.

A convolution is mpc_conv2d (the library lowers the shares to the im2col rows of the outputs'
inner products and runs Pi_Inner with Pi_Trunc^k on them, Sec. 4.1) with its verification, then a
local rearrangement of the output rows (b, i, j) x c_out back to NCHW (mpc_gather).
Max-pool and ReLU are the Sec. 4.3 layers; they commute (max of ReLUs = ReLU of the max), so
every conv block pools first and applies ReLU to the 4x smaller result.  Non-linear layers are
called per chunk of at most `nl_chunk` elements, each chunk with its own verification.  The index
maps are integer plumbing computed here; all share arithmetic runs in libmpc3's kernels.
"""
from __future__ import annotations

import numpy as np

from . import mpc as M


# ---- index maps -------------------------------------------------------------------------------
def net_b_params(seed_name: str):
    from .workloads import rng
    g = rng(seed_name)
    chans = [3, 64, 64, 128, 128, 256]
    p = {f"c{i + 1}": he_normal(g, (chans[i + 1], chans[i], 3, 3), chans[i] * 9) for i in range(5)}
    p["f1"] = he_normal(g, (4096, 512), 4096)
    p["f2"] = he_normal(g, (512, 10), 512)
    return p


NET_B_POOL = {"c1": False, "c2": True, "c3": False, "c4": True, "c5": True}


def im2col_index(B, C, H, W, kh, kw):
    """Rows (b, i, j) of the valid output, columns (c, di, dj): index into the NCHW input."""
    Ho, Wo = H - kh + 1, W - kw + 1
    b, i, j, c, di, dj = np.meshgrid(np.arange(B), np.arange(Ho), np.arange(Wo), np.arange(C),
                                     np.arange(kh), np.arange(kw), indexing="ij")
    return (((b * C + c) * H + i + di) * W + j + dj).reshape(-1).astype(np.int64), Ho, Wo


def rows_to_nchw_index(B, Co, Ho, Wo):
    """Output element (b, oc, i, j) <- product row (b, i, j), column oc."""
    b, oc, i, j = np.meshgrid(np.arange(B), np.arange(Co), np.arange(Ho), np.arange(Wo), indexing="ij")
    return (((b * Ho + i) * Wo + j) * Co + oc).reshape(-1).astype(np.int64)


def conv_weight_matrix(w):
    """(C_out, C, kh, kw) -> (C kh kw, C_out) with rows (c, di, dj)."""
    return np.ascontiguousarray(w.reshape(w.shape[0], -1).T)


# ---- plaintext model ----------------------------------------------------------------------------
def he_normal(g, shape, fan_in):
    return g.normal(0.0, np.sqrt(2.0 / fan_in), shape)


def net_a_params(seed_name: str):
    from .workloads import rng
    g = rng(seed_name)
    return {"c1": he_normal(g, (16, 1, 5, 5), 25), "c2": he_normal(g, (16, 16, 5, 5), 400),
            "f1": he_normal(g, (256, 100), 256), "f2": he_normal(g, (100, 10), 100)}


def _conv_fp64(x, w, pad: int = 0):
    if pad:
        x = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    B, C, H, W = x.shape
    idx, Ho, Wo = im2col_index(B, C, H, W, w.shape[2], w.shape[3])
    cols = x.reshape(-1)[idx].reshape(B * Ho * Wo, -1)
    z = cols @ conv_weight_matrix(w)
    return z.reshape(B, Ho, Wo, -1).transpose(0, 3, 1, 2)


def _pool_fp64(x):
    return np.maximum(np.maximum(x[:, :, 0::2, 0::2], x[:, :, 0::2, 1::2]),
                      np.maximum(x[:, :, 1::2, 0::2], x[:, :, 1::2, 1::2]))


def net_b_fp64(x, p):
    h = x
    for i in range(1, 6):
        h = _conv_fp64(h, p[f"c{i}"], pad=1)
        if NET_B_POOL[f"c{i}"]:
            h = _pool_fp64(h)
        h = np.maximum(h, 0.0)
    h = h.reshape(h.shape[0], -1)
    h = np.maximum(h @ p["f1"], 0.0)
    return h @ p["f2"]


def net_a_fp64(x, p):
    h = np.maximum(_pool_fp64(_conv_fp64(x, p["c1"])), 0.0)
    h = np.maximum(_pool_fp64(_conv_fp64(h, p["c2"])), 0.0)
    h = h.reshape(h.shape[0], -1)
    h = np.maximum(h @ p["f1"], 0.0)
    return h @ p["f2"]


# ---- secure model -------------------------------------------------------------------------------
class _Ids:
    def __init__(self, base):
        self.v = base

    def take(self, k=1):
        v = self.v
        self.v += k
        return v


def _matmul_verified(ctx, ids, h, gw, Mr, N, K, k, keys=None):
    c = ids.take(2)
    zpre, zout, pq = ctx.matmul(c, h, gw, Mr, N, K, k, row_keys=keys)
    rc, _ = ctx.verify_matmul(c + 1, h, gw, zpre, pq, Mr, N, K, k, c, row_keys=keys)
    if rc != M.MPC_OK:
        raise M.MpcError(rc, "matrix-product layer rejected")
    return zout


def _relu_chunked(ctx, ids, h, n, chunk):
    if n <= chunk:
        c = ids.take(2)
        rc, out, _ = ctx.relu(c, c + 1, h, n)
        if rc != M.MPC_OK:
            raise M.MpcError(rc, "ReLU rejected")
        return out
    parts = []
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        part = ctx.gather(h, n, np.arange(s, e, dtype=np.int64))
        parts.append((_relu_chunked(ctx, ids, part, e - s, chunk), e - s))
    return _concat(ctx, parts)


def _concat(ctx, parts):
    n = sum(m for _, m in parts)
    out = ctx.shares(n)
    off = 0
    for t, m in parts:
        for c in range(6):
            out[c * n + off: c * n + off + m].copy_(t[c * m:(c + 1) * m])
        off += m
    return out


# Comparisons per non-linear call: each call (a ReLU chunk, or whole channel planes of a max-pool)
# is verified on its own; 2^16 comparisons take about 37 GB of workspace.
NL_CHUNK = 1 << 16


def pool_planes(nl_budget: int, H: int, W: int, planes: int) -> int:
    """Channel planes per max-pool call: about nl_budget comparisons (3/4 of the elements)."""
    return max(1, min(planes, (4 * nl_budget) // (3 * H * W)))


def _pool_chunked(ctx, ids, h, shape, nl_budget):
    """2x2 max-pool of a (B, C, H, W) sharing in calls of whole channel planes, each call at most
    about nl_budget comparisons (3/4 of its elements), each verified on its own."""
    B, C, H, W = shape
    planes, per = B * C, H * W
    step = pool_planes(nl_budget, H, W, planes)
    parts = []
    for p0 in range(0, planes, step):
        p1 = min(planes, p0 + step)
        part = ctx.gather(h, planes * per, np.arange(p0 * per, p1 * per, dtype=np.int64))
        c = ids.take(2)
        rc, out, _ = ctx.maxpool2(c, c + 1, part, (p1 - p0, 1, H, W))
        if rc != M.MPC_OK:
            raise M.MpcError(rc, "max-pool rejected")
        parts.append((out, (p1 - p0) * (H // 2) * (W // 2)))
    return _concat(ctx, parts)


def _conv_block(ctx, ids, h, shape, gw, wshape, k, nl_budget, relu_chunk, segments=None,
                layer=0, pad=0, pool=True):
    B, C, H, W = shape
    Co, _, kh, kw = wshape
    c = ids.take(2)
    geom = (B, C, H, W, kh, kw, 1, pad)
    Ho, Wo = ctx.conv_out(geom)
    keys = M.segment_row_keys(segments, layer, Ho * Wo) if segments is not None else None
    cols, zpre, zout, pq, (Mr, N, K) = ctx.conv2d(c, h, gw, geom, Co, k, row_keys=keys)
    rc, _ = ctx.verify_matmul(c + 1, cols, gw, zpre, pq, Mr, N, K, k, c, row_keys=keys)
    if rc != M.MPC_OK:
        raise M.MpcError(rc, "convolution rejected")
    z = ctx.gather(zout, Mr * Co, rows_to_nchw_index(B, Co, Ho, Wo))
    if pool:
        z = _pool_chunked(ctx, ids, z, (B, Co, Ho, Wo), nl_budget)
        Ho, Wo = Ho // 2, Wo // 2
    n = B * Co * Ho * Wo
    return _relu_chunked(ctx, ids, z, n, relu_chunk), (B, Co, Ho, Wo)


def share_params(ctx: "M.Context", params, k: int = 13, call_base: int = 4000):
    """P0 shares Net A's weights once (mpc_share_fixed): the conv kernels as (C kh kw) x C_out
    matrices (a public layout of P0's plaintext), the FC matrices as they are.  The sharings can
    serve any number of forward passes."""
    out = {}
    for i, name in enumerate(("c1", "c2", "f1", "f2")):
        w = params[name]
        m = conv_weight_matrix(w) if name.startswith("c") else w
        out[name] = ctx.share_fixed(call_base + i, np.ascontiguousarray(m, dtype=np.float64).reshape(-1), k)
    return out


def net_a_secure(ctx: "M.Context", x, params, k: int = 13, call_base: int = 5000,
                 nl_budget: int = NL_CHUNK, relu_chunk: int = NL_CHUNK, shared=None, segments=None):
    """Secure Net A forward.  x: (B, 1, 28, 28) float inputs; params: the float parameters (shared
    by P0 here unless `shared` holds share_params' sharings); segments: as for
    secure_mlp.secure_forward (truncation bits keyed by request, layer and row).  Returns the
    opened logits (B, 10) as float64."""
    ids = _Ids(call_base)
    if shared is None:
        shared = share_params(ctx, params, k, ids.take(4))
    B = x.shape[0]
    h = ctx.share_fixed(ids.take(), np.ascontiguousarray(x, dtype=np.float64).reshape(-1), k)
    shape = x.shape
    h, shape = _conv_block(ctx, ids, h, shape, shared["c1"], params["c1"].shape, k, nl_budget,
                           relu_chunk, segments, 0)
    h, shape = _conv_block(ctx, ids, h, shape, shared["c2"], params["c2"].shape, k, nl_budget,
                           relu_chunk, segments, 1)
    flat = int(np.prod(shape[1:]))
    for layer, name, last in ((2, "f1", False), (3, "f2", True)):
        w = params[name]
        keys = M.segment_row_keys(segments, layer, 1) if segments is not None else None
        h = _matmul_verified(ctx, ids, h, shared[name], B, w.shape[1], flat, k, keys)
        flat = w.shape[1]
        if not last:
            h = _relu_chunked(ctx, ids, h, B * flat, relu_chunk)
    return ctx.reconstruct_fixed(h, B * flat, k).reshape(B, flat)


def share_params_b(ctx: "M.Context", params, k: int = 13, call_base: int = 4000):
    """P0 shares Net B's weights once (as share_params does for Net A)."""
    out = {}
    for i, name in enumerate(("c1", "c2", "c3", "c4", "c5", "f1", "f2")):
        w = params[name]
        m = conv_weight_matrix(w) if name.startswith("c") else w
        out[name] = ctx.share_fixed(call_base + i, np.ascontiguousarray(m, dtype=np.float64).reshape(-1), k)
    return out


def net_b_secure(ctx: "M.Context", x, params, k: int = 13, call_base: int = 7000,
                 nl_budget: int = NL_CHUNK, relu_chunk: int = NL_CHUNK, shared=None, segments=None):
    """Secure Net B forward.  x: (B, 3, 32, 32) float inputs; params: the float parameters;
    shared / segments as for net_a_secure.  Returns the opened logits (B, 10) as float64."""
    ids = _Ids(call_base)
    if shared is None:
        shared = share_params_b(ctx, params, k, ids.take(7))
    B = x.shape[0]
    h = ctx.share_fixed(ids.take(), np.ascontiguousarray(x, dtype=np.float64).reshape(-1), k)
    shape = x.shape
    for i in range(1, 6):
        name = f"c{i}"
        h, shape = _conv_block(ctx, ids, h, shape, shared[name], params[name].shape, k, nl_budget,
                               relu_chunk, segments, i - 1, pad=1, pool=NET_B_POOL[name])
    flat = int(np.prod(shape[1:]))
    for layer, name, last in ((5, "f1", False), (6, "f2", True)):
        w = params[name]
        keys = M.segment_row_keys(segments, layer, 1) if segments is not None else None
        h = _matmul_verified(ctx, ids, h, shared[name], B, w.shape[1], flat, k, keys)
        flat = w.shape[1]
        if not last:
            h = _relu_chunked(ctx, ids, h, B * flat, relu_chunk)
    return ctx.reconstruct_fixed(h, B * flat, k).reshape(B, flat)


def main():
    """Images/s of one secure forward pass of Net A or Net B at a batch size (synthetic inputs,
    He-normal weights), and its largest deviation from the float64 model of the quantised
    parameters."""
    import argparse
    import json
    import time
    from .workloads import master_seed, rng
    from .secure_mlp import quantized
    ap = argparse.ArgumentParser()
    ap.add_argument("--net", choices=["a", "b"], default="a")
    ap.add_argument("--batch", type=int, default=256)
    a = ap.parse_args()
    import torch
    if a.net == "a":
        p = net_a_params("C4-netA-weights")
        x = rng("C4-netA-inputs").uniform(0.0, 1.0, (a.batch, 1, 28, 28))
        run, ref, share = net_a_secure, net_a_fp64, share_params
    else:
        p = net_b_params("C4-netB-weights")
        x = rng("C4-netB-inputs").uniform(0.0, 1.0, (a.batch, 3, 32, 32))
        run, ref, share = net_b_secure, net_b_fp64, share_params_b
    ctx = M.Context(master_seed(f"C4-net{a.net}"))
    shared = share(ctx, p, 13, 100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = run(ctx, x, p, 13, shared=shared)
    dt = time.perf_counter() - t0
    err = float(np.max(np.abs(got - ref(quantized(x, 13), {n: quantized(w, 13) for n, w in p.items()}))))
    print(json.dumps({"net": a.net, "batch": a.batch, "seconds": round(dt, 2),
                      "images_per_s": round(a.batch / dt, 3), "max_abs_err_vs_fp64": err}))


if __name__ == "__main__":
    main()
