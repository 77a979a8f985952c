"""Thin Python binding of libmpc3 (include/mpc3.h).

Every method marshals arguments and calls the C-ABI of the same name; all protocol work runs in
the library's CUDA kernels.  PyTorch is used only to allocate device memory (sharings, workspace,
traces) and to supply the CUDA stream.  There is no CPU fallback: constructing a ``Context``
without a CUDA device or without the built library raises.

Sharings are int64 CUDA tensors holding u64 bit patterns, 6*n words each, component order
(P0.[r]_1, P0.[r]_2, P1.m, P1.[r]_1, P2.m, P2.[r]_2).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib

MPC_OK, MPC_ERR_ARG, MPC_ERR_SHAPE, MPC_ERR_WORKSPACE, MPC_ERR_CUDA = 0, 1, 2, 3, 4
MPC_ERR_TIMEOUT, MPC_ERR_VERIFY, MPC_ERR_ABORT, MPC_ERR_PENDING = 5, 6, 7, 8
REDUCE_POINT_X, REDUCE_POINT_2 = 0, 1
GEMM_U64, GEMM_LIMB_TC = 0, 1
(OP_SHARE, OP_MULT, OP_MATMUL, OP_VERIFY_MULT, OP_VERIFY_MATMUL, OP_RECONSTRUCT, OP_RELU,
 OP_MAXPOOL2, OP_VERIFY_MULT_CALLS, OP_SHARE_FIXED, OP_RECONSTRUCT_FIXED, OP_TRUNC,
 OP_VERIFY_TRUNC) = range(13)
SITES = {"GAMMA2": 0, "MZ1": 1, "MZ2": 2, "MX_COPY_P1": 3, "REC_MSG": 4, "HIGH_BIT": 5,
         "AND_GAMMA2": 6, "TRUNC_D1": 7}
TRACE_GF_ROUND = 13
PHASES = ("offline", "online", "verify")
PROTOS = ("share", "mult", "inner", "trunc", "rec", "verify")
TRACE_ROUND = 832
NOALLOC_MAX_N = 262144
PROF_PHASES = ("share", "mult", "trunc_pairs", "gemm", "exchange", "verify_gemm", "trunc_setup",
               "trunc_s", "trunc_rounds", "trunc_materialize", "trunc_tail", "rec", "verify_mult",
               "k_limb_gemm", "k_trunc_s", "k_gr_matmul", "k_gram", "k_gr_mul_rows", "nonlinear")
ERR_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_WORKSPACE", 4: "ERR_CUDA",
             5: "ERR_TIMEOUT", 6: "ERR_VERIFY", 7: "ERR_ABORT", 8: "ERR_PENDING"}


class MpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libmpc3 needs a CUDA device (no CPU fallback)")
    return torch


H2D_SLOTS = 4   # MPC_H2D_SLOTS: the upload slots of mpc_h2d_async


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def default_R(D: int) -> int:
    if D <= 1:
        return 0
    return max(0, int(np.ceil(np.log2(D))) - 6)


class Context:
    """One three-party run: keys from `seed`, ledger, abort state; work on the current stream."""

    def __init__(self, seed: bytes, device: int = 0, reduce_mode: int = REDUCE_POINT_X,
                 gemm_path: int = GEMM_LIMB_TC, stream=None, tuning: dict | None = None):
        torch = _torch()
        self.torch = torch
        self.lib = _lib.load()
        assert len(seed) == 32
        self.device = torch.device("cuda", device)
        cfg = _lib.MpcConfig()
        for i, b in enumerate(seed):
            cfg.seed[i] = b
        cfg.device = device
        cfg.reduce_mode = reduce_mode
        cfg.gemm_path = gemm_path
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        cfg.stream = C.c_void_p(stream.cuda_stream)
        h = C.c_void_p()
        rc = self.lib.mpc_create(C.byref(cfg), C.byref(h))
        if rc != MPC_OK:
            raise MpcError(rc, "mpc_create failed")
        self.h = h
        self._ws = None
        if tuning:
            self.set_tuning(**tuning)

    TUNING_FIELDS = tuple(f for f, _ in _lib.MpcTuning._fields_)

    def set_tuning(self, **fields):
        """mpc_set_tuning: fields of mpc_tuning by name; unnamed fields keep their defaults."""
        t = _lib.MpcTuning()
        for k, v in fields.items():
            if k not in self.TUNING_FIELDS:
                raise KeyError(k)
            setattr(t, k, int(v))
        self._check(self.lib.mpc_set_tuning(self.h, C.byref(t)))

    def tuning(self) -> dict:
        t = _lib.MpcTuning()
        self._check(self.lib.mpc_get_tuning(self.h, C.byref(t)))
        return {k: int(getattr(t, k)) for k in self.TUNING_FIELDS}

    def trace_words(self, op: int, a: int, b: int = 0, c: int = 0, trunc_bits: int = -1,
                    R_main: int = -1, R_trunc: int = -1) -> int:
        v = self.lib.mpc_trace_words(self.h, op, a, b, c, trunc_bits, R_main, R_trunc)
        if v < 0:
            raise MpcError(MPC_ERR_ARG, "bad trace query")
        return int(v)

    def set_stream(self, stream):
        """Enqueue subsequent work on `stream` (a torch.cuda.Stream), e.g. a graph-capture stream."""
        self._check(self.lib.mpc_set_stream(self.h, C.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def h2d_async(self, dst, src, slot: int = 0):
        """mpc_h2d_async: copy the host tensor `src` (pinned, for overlap) into the device tensor
        `dst` on the copy stream, after the work enqueued so far; recorded under `slot`."""
        nbytes = src.numel() * src.element_size()
        assert dst.numel() * dst.element_size() >= nbytes
        self._check(self.lib.mpc_h2d_async(self.h, C.c_void_p(_ptr(dst)), C.c_void_p(_ptr(src)),
                                           nbytes, slot))

    def d2h_async(self, dst, src, slot: int = 0):
        """mpc_d2h_async: copy the device tensor `src` into the host tensor `dst` (pinned) on the
        copy stream, after the work enqueued so far; recorded under `slot`."""
        nbytes = src.numel() * src.element_size()
        assert dst.numel() * dst.element_size() >= nbytes
        self._check(self.lib.mpc_d2h_async(self.h, C.c_void_p(_ptr(dst)), C.c_void_p(_ptr(src)),
                                           nbytes, slot))

    def h2d_wait(self, slot: int = 0):
        """mpc_h2d_wait: the context's stream waits (on the device) for the copy of `slot`."""
        self._check(self.lib.mpc_h2d_wait(self.h, slot))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- helpers -------------------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != MPC_OK:
            raise MpcError(rc, self.lib.mpc_last_error(self.h).decode())
        return rc

    def empty(self, nwords: int):
        return self.torch.empty(max(int(nwords), 1), dtype=self.torch.int64, device=self.device)

    def zeros(self, nwords: int):
        return self.torch.zeros(max(int(nwords), 1), dtype=self.torch.int64, device=self.device)

    def shares(self, n: int):
        return self.empty(6 * n)

    def workspace(self, nbytes: int):
        """Grow-only workspace tensor (256-byte aligned by the caching allocator)."""
        nwords = (int(nbytes) + 7) // 8 + 32
        if self._ws is None or self._ws.numel() < nwords:
            self._ws = None
            self._ws = self.torch.empty(nwords, dtype=self.torch.int64, device=self.device)
        return self._ws

    def ws_size(self, op: int, a: int, b: int = 0, c: int = 0, trunc_bits: int = -1,
                R_main: int = -1, R_trunc: int = -1) -> int:
        v = self.lib.mpc_workspace_size(self.h, op, a, b, c, trunc_bits, R_main, R_trunc)
        if v < 0:
            raise MpcError(MPC_ERR_ARG, "bad workspace query")
        return int(v)

    # ---- protocols -------------------------------------------------------------------------------
    def share_input(self, call_id: int, x, out=None, owner: int = 0):
        """Pi_<.>^{l,k}(x), k = owner (0: P0, the default).  x: CUDA int64 tensor (device input)
        or numpy uint64 array (host)."""
        if isinstance(x, np.ndarray):
            xh = np.ascontiguousarray(x, dtype=np.uint64)
            n = xh.size
            ptr, on_host = xh.ctypes.data, 1
        else:
            n = x.numel()
            ptr, on_host = _ptr(x), 0
        out = self.shares(n) if out is None else out
        wsb = self.ws_size(OP_SHARE, n)
        ws = self.workspace(wsb)
        if owner == 0:
            rc = self.lib.mpc_share_input(self.h, call_id, C.c_void_p(ptr), on_host, n,
                                          C.c_void_p(_ptr(out)), C.c_void_p(_ptr(ws)), wsb)
        else:
            rc = self.lib.mpc_share_input_from(self.h, call_id, owner, C.c_void_p(ptr), on_host,
                                               n, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(ws)), wsb)
        self._check(rc)
        if on_host:   # the host buffer must stay alive until the copy ran
            self.sync()
        return out

    def share_fixed(self, call_id: int, x, frac_bits: int, out=None, owner: int = 0):
        """mpc_share_fixed: the library encodes floor(x 2^k) and shares it.  x: numpy float64
        (host) or a CUDA float64 tensor (device)."""
        if isinstance(x, np.ndarray):
            xh = np.ascontiguousarray(x, dtype=np.float64)
            n, ptr, on_host = xh.size, xh.ctypes.data, 1
        else:
            n, ptr, on_host = x.numel(), _ptr(x), 0
        out = self.shares(n) if out is None else out
        wsb = self.ws_size(OP_SHARE_FIXED, n)
        ws = self.workspace(wsb)
        self._check(self.lib.mpc_share_fixed(self.h, call_id, owner, C.c_void_p(ptr), on_host, n,
                                             frac_bits, C.c_void_p(_ptr(out)),
                                             C.c_void_p(_ptr(ws)), wsb))
        return out

    def reconstruct_fixed(self, xs, n: int, frac_bits: int) -> np.ndarray:
        """mpc_reconstruct_fixed: Pi_Rec, then the signed value / 2^k (host float64 array)."""
        out = np.empty(n, dtype=np.float64)
        wsb = self.ws_size(OP_RECONSTRUCT_FIXED, n)
        ws = self.workspace(wsb)
        self._check(self.lib.mpc_reconstruct_fixed(self.h, C.c_void_p(_ptr(xs)), n, frac_bits,
                                                   C.c_void_p(out.ctypes.data), 1,
                                                   C.c_void_p(_ptr(ws)), wsb))
        return out

    @staticmethod
    def conv_out(geom):
        """(Ho, Wo) of a convolution, (0, 0) for a geometry the library rejects."""
        B, Cc, H, W, kh, kw, stride, pad = geom
        if stride <= 0 or pad < 0 or H + 2 * pad < kh or W + 2 * pad < kw:
            return 0, 0
        return (H + 2 * pad - kh) // stride + 1, (W + 2 * pad - kw) // stride + 1

    def conv2d(self, call_id: int, xs, ws_, geom, C_out: int, trunc_bits: int = -1,
               row_keys=None):
        """mpc_conv2d.  geom = (B, C, H, W, kh, kw, stride, pad).  Returns (cols, zpre, zout, pq,
        (M, N, K)) with M = B Ho Wo, N = C_out, K = C kh kw (output rows (b, i, j)); row_keys as
        for matmul."""
        B, Cc, H, W, kh, kw, stride, pad = geom
        Ho, Wo = self.conv_out(geom)
        Mr, K = B * Ho * Wo, Cc * kh * kw
        E = Mr * C_out
        cols = self.shares(Mr * K)
        zpre = self.shares(E)
        zout = self.shares(E) if trunc_bits >= 0 else None
        pq = self.empty(12 * E) if trunc_bits >= 0 else None
        wsb = self.ws_size(OP_MATMUL, Mr, C_out, K, trunc_bits)
        ws = self.workspace(wsb)
        g = (C.c_int32 * 8)(*geom)
        rk = self._row_keys(row_keys)
        self._check(self.lib.mpc_conv2d(self.h, call_id, C.c_void_p(_ptr(xs)), C.c_void_p(_ptr(ws_)),
                                        g, C_out, trunc_bits, C.c_void_p(_ptr(rk)),
                                        C.c_void_p(_ptr(cols)),
                                        C.c_void_p(_ptr(zpre)), C.c_void_p(_ptr(zout)),
                                        C.c_void_p(_ptr(pq)), C.c_void_p(_ptr(ws)), wsb))
        if rk is not None:
            self.sync()   # the keys must outlive the enqueued work
        return cols, zpre, (zout if trunc_bits >= 0 else zpre), pq, (Mr, C_out, K)

    def trunc(self, call_id: int, xs, n: int, t: int):
        """mpc_trunc: Pi_Trunc^t of a sharing.  Returns (out sharing, pq)."""
        out, pq = self.shares(n), self.empty(12 * n)
        wsb = self.ws_size(OP_TRUNC, n)
        ws = self.workspace(wsb)
        self._check(self.lib.mpc_trunc(self.h, call_id, C.c_void_p(_ptr(xs)), n, t,
                                       C.c_void_p(_ptr(out)), C.c_void_p(_ptr(pq)),
                                       C.c_void_p(_ptr(ws)), wsb))
        return out, pq

    def verify_trunc(self, verify_id: int, pq, n: int, t: int, trunc_call_id: int, R: int = -1,
                     trace: bool = False):
        tr = self.zeros(self.trace_words(OP_VERIFY_TRUNC, n, 0, 0, t, -1, R)) if trace else None
        wsb = self.ws_size(OP_VERIFY_TRUNC, n, R_trunc=R)
        ws = self.workspace(wsb)
        rc = self.lib.mpc_verify_trunc(self.h, verify_id, C.c_void_p(_ptr(pq)), n, t, trunc_call_id,
                                       R, C.c_void_p(_ptr(ws)), wsb, C.c_void_p(_ptr(tr)))
        if rc not in (MPC_OK, MPC_ERR_VERIFY, MPC_ERR_ABORT):
            self._check(rc)
        return rc, tr

    def mult(self, call_id: int, xs, ys, n: int, out=None):
        out = self.shares(n) if out is None else out
        wsb = self.ws_size(OP_MULT, n)
        ws = self.workspace(wsb)
        self._check(self.lib.mpc_mult(self.h, call_id, C.c_void_p(_ptr(xs)), C.c_void_p(_ptr(ys)),
                                      n, C.c_void_p(_ptr(out)), C.c_void_p(_ptr(ws)), wsb))
        return out

    def _row_keys(self, row_keys):
        """numpy uint64 row keys -> a CUDA tensor (None stays None)."""
        if row_keys is None or not isinstance(row_keys, np.ndarray):
            return row_keys
        return from_u64(self, np.ascontiguousarray(row_keys, dtype=np.uint64))

    def matmul(self, call_id: int, xs, ws_, M: int, N: int, K: int, trunc_bits: int = -1,
               zpre=None, zout=None, pq=None, row_keys=None):
        """mpc_matmul, or mpc_matmul_keyed when row_keys (M object ids, numpy or CUDA) is given."""
        E = M * N
        zpre = self.shares(E) if zpre is None else zpre
        if trunc_bits >= 0:
            zout = self.shares(E) if zout is None else zout
            pq = self.empty(12 * E) if pq is None else pq
        wsb = self.ws_size(OP_MATMUL, M, N, K, trunc_bits)
        ws = self.workspace(wsb)
        rk = self._row_keys(row_keys)
        self._check(self.lib.mpc_matmul_keyed(self.h, call_id, C.c_void_p(_ptr(xs)),
                                              C.c_void_p(_ptr(ws_)), M, N, K, trunc_bits,
                                              C.c_void_p(_ptr(rk)), C.c_void_p(_ptr(zpre)),
                                              C.c_void_p(_ptr(zout)), C.c_void_p(_ptr(pq)),
                                              C.c_void_p(_ptr(ws)), wsb))
        if rk is not None:
            self.sync()   # the keys must outlive the enqueued work
        return zpre, (zout if trunc_bits >= 0 else zpre), pq

    def verify_mult(self, verify_id: int, xs, ys, zs, n: int, mult_call_id: int, R: int = -1,
                    trace: bool = False):
        """Returns (code, trace): code MPC_OK (accept), MPC_ERR_VERIFY or MPC_ERR_ABORT."""
        Rr = default_R(n) if R < 0 else R
        tr = self.zeros((Rr + 1) * TRACE_ROUND) if trace else None
        wsb = self.ws_size(OP_VERIFY_MULT, n, R_main=R)
        ws = self.workspace(wsb)
        rc = self.lib.mpc_verify_mult(self.h, verify_id, C.c_void_p(_ptr(xs)), C.c_void_p(_ptr(ys)),
                                      C.c_void_p(_ptr(zs)), n, mult_call_id, R,
                                      C.c_void_p(_ptr(ws)), wsb, C.c_void_p(_ptr(tr)))
        if rc not in (MPC_OK, MPC_ERR_VERIFY, MPC_ERR_ABORT):
            self._check(rc)
        return rc, tr

    def verify_mult_calls(self, verify_id: int, triples, R: int = -1, trace: bool = False):
        """Deferred Pi_MultVerify over the triples of several mult calls in one batch.
        triples: list of (xs, ys, zs, n, mult_call_id).  Returns (code, trace) as verify_mult."""
        k = len(triples)
        N = sum(int(t[3]) for t in triples)
        Rr = default_R(N) if R < 0 else R
        tr = self.zeros((Rr + 1) * TRACE_ROUND) if trace else None
        wsb = self.ws_size(OP_VERIFY_MULT_CALLS, N, R_main=R)
        ws = self.workspace(wsb)
        ptrs = [(C.c_void_p * k)(*(_ptr(t[j]) for t in triples)) for j in range(3)]
        ns = (C.c_int64 * k)(*(int(t[3]) for t in triples))
        ids = (C.c_uint64 * k)(*(int(t[4]) for t in triples))
        rc = self.lib.mpc_verify_mult_calls(self.h, verify_id, k, ptrs[0], ptrs[1], ptrs[2], ns, ids,
                                            R, C.c_void_p(_ptr(ws)), wsb, C.c_void_p(_ptr(tr)))
        if rc not in (MPC_OK, MPC_ERR_VERIFY, MPC_ERR_ABORT):
            self._check(rc)
        return rc, tr

    def gather(self, xs, n_in: int, idx):
        """out[k] = x[idx[k]] (0 where idx[k] < 0) on every share component; idx: numpy int64."""
        idx_d = self.torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int64)).to(self.device)
        out = self.shares(idx_d.numel())
        self._check(self.lib.mpc_gather(self.h, C.c_void_p(_ptr(xs)), n_in, C.c_void_p(_ptr(idx_d)),
                                        idx_d.numel(), C.c_void_p(_ptr(out))))
        self.sync()   # idx_d must outlive the enqueued gather
        return out

    def hash_u64(self, data) -> bytes:
        """H of Pi_Rec (SHA-256 Merkle root, 1 KiB leaves) of a device u64 tensor."""
        d = (C.c_uint8 * 32)()
        self._check(self.lib.mpc_hash_u64(self.h, C.c_void_p(_ptr(data) if data.numel() else 0),
                                          data.numel(), d))
        return bytes(d)

    @staticmethod
    def nonlinear_R(np_list):
        """Default rounds (R0, R1, R2, R3) of a non-linear layer's four verification batches for
        stage widths np_list (padded): daBit and final products, edaBit inner products, AND
        gates, edaBit bit products."""
        nm = sum(3 * n for n in np_list)
        ne = sum(np_list)
        nand = sum(125 * n for n in np_list)
        return default_R(nm), default_R(64 * ne), default_R(nand), default_R(64 * ne)

    def _nl_trace(self, np_list, trace):
        if not trace:
            return None
        R0, R1, R2, R3 = self.nonlinear_R(np_list)
        return self.zeros((R0 + 1) * TRACE_ROUND + (R1 + 1) * TRACE_ROUND + (R2 + 1) * TRACE_GF_ROUND
                          + (R3 + 1) * TRACE_ROUND)

    def relu(self, call_id: int, verify_id: int, xs, n: int, trace: bool = False):
        """ReLU layer with its verification (Sec. 4.3).  Returns (code, out sharing, trace)."""
        out = self.shares(n)
        np_ = 64 * ((n + 63) // 64)
        tr = self._nl_trace([np_], trace)
        wsb = self.ws_size(OP_RELU, n)
        ws = self.workspace(wsb)
        rc = self.lib.mpc_relu(self.h, call_id, verify_id, C.c_void_p(_ptr(xs)), n,
                               C.c_void_p(_ptr(out)), C.c_void_p(_ptr(ws)), wsb, C.c_void_p(_ptr(tr)))
        if rc not in (MPC_OK, MPC_ERR_VERIFY, MPC_ERR_ABORT):
            self._check(rc)
        return rc, out, tr

    def maxpool2(self, call_id: int, verify_id: int, xs, shape, trace: bool = False):
        """2x2 / stride-2 max-pool of a (B, C, H, W) sharing with its verification."""
        B, Cc, H, W = shape
        nw = B * Cc * (H // 2) * (W // 2)
        out = self.shares(nw)
        nps = [64 * ((2 * nw + 63) // 64), 64 * ((nw + 63) // 64)]
        tr = self._nl_trace(nps, trace)
        wsb = self.ws_size(OP_MAXPOOL2, B * Cc, H, W)
        ws = self.workspace(wsb)
        rc = self.lib.mpc_maxpool2(self.h, call_id, verify_id, C.c_void_p(_ptr(xs)), B, Cc, H, W,
                                   C.c_void_p(_ptr(out)), C.c_void_p(_ptr(ws)), wsb,
                                   C.c_void_p(_ptr(tr)))
        if rc not in (MPC_OK, MPC_ERR_VERIFY, MPC_ERR_ABORT):
            self._check(rc)
        return rc, out, tr

    def verify_matmul(self, verify_id: int, xs, ws_, zpre, pq, M: int, N: int, K: int,
                      trunc_bits: int, matmul_call_id: int, R_main: int = -1, R_trunc: int = -1,
                      trace: bool = False, row_keys=None):
        ntr = self.trace_words(OP_VERIFY_MATMUL, M, N, K, trunc_bits, R_main, R_trunc)
        tr = self.zeros(ntr) if trace else None
        wsb = self.ws_size(OP_VERIFY_MATMUL, M, N, K, trunc_bits, R_main, R_trunc)
        ws = self.workspace(wsb)
        rk = self._row_keys(row_keys)
        rc = self.lib.mpc_verify_matmul_keyed(self.h, verify_id, C.c_void_p(_ptr(xs)),
                                              C.c_void_p(_ptr(ws_)), C.c_void_p(_ptr(zpre)),
                                              C.c_void_p(_ptr(pq)), M, N, K, trunc_bits,
                                              C.c_void_p(_ptr(rk)), matmul_call_id, R_main, R_trunc,
                                              C.c_void_p(_ptr(ws)), wsb, C.c_void_p(_ptr(tr)))
        if rc not in (MPC_OK, MPC_ERR_VERIFY, MPC_ERR_ABORT):
            self._check(rc)
        return rc, tr

    def reconstruct(self, xs, n: int, to_host: bool = True):
        """Pi_Rec; returns a numpy uint64 array (host) or an int64 CUDA tensor."""
        wsb = self.ws_size(OP_RECONSTRUCT, n)
        ws = self.workspace(wsb)
        if to_host:
            out = np.empty(n, dtype=np.uint64)
            rc = self.lib.mpc_reconstruct(self.h, C.c_void_p(_ptr(xs)), n,
                                          C.c_void_p(out.ctypes.data), 1, C.c_void_p(_ptr(ws)), wsb)
        else:
            out = self.empty(n)
            rc = self.lib.mpc_reconstruct(self.h, C.c_void_p(_ptr(xs)), n, C.c_void_p(_ptr(out)),
                                          0, C.c_void_p(_ptr(ws)), wsb)
        self._check(rc)
        return out

    def reconstruct_noalloc(self, xs, n: int, out=None):
        """Pi_Rec through mpc_reconstruct_noalloc: the library uses its fixed device array as
        scratch and allocates nothing (for callers that cannot allocate at this point); n must
        not exceed NOALLOC_MAX_N.  Returns the int64 CUDA tensor it wrote."""
        out = self.empty(n) if out is None else out
        self._check(self.lib.mpc_reconstruct_noalloc(self.h, C.c_void_p(_ptr(xs)), n,
                                                     C.c_void_p(_ptr(out))))
        return out

    def ledger(self):
        b = (C.c_uint64 * 18)()
        m = C.c_uint64()
        self._check(self.lib.mpc_ledger(self.h, b, C.byref(m)))
        out = {(PHASES[i // 6], PROTOS[i % 6]): int(b[i]) for i in range(18)}
        return out, int(m.value)

    def ledger_reset(self):
        self.lib.mpc_ledger_reset(self.h)

    def inject_fault(self, site: str, index: int, xor_mask: int = 1):
        self._check(self.lib.mpc_inject_fault(self.h, SITES[site], index, xor_mask))

    def status(self) -> int:
        return self.lib.mpc_status(self.h)

    def profile(self, enable: bool):
        self._check(self.lib.mpc_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{phase name: (milliseconds, intervals, algorithmic u64 MACs)} since the last read
        (waits for the stream)."""
        ms = (C.c_double * len(PROF_PHASES))()
        cnt = (C.c_uint64 * len(PROF_PHASES))()
        work = (C.c_double * len(PROF_PHASES))()
        self._check(self.lib.mpc_profile_read(self.h, ms, cnt, work))
        return {name: (float(ms[i]), int(cnt[i]), float(work[i]))
                for i, name in enumerate(PROF_PHASES)}

    def launch_count(self) -> int:
        return int(self.lib.mpc_launch_count())

    def sync(self):
        self._check(self.lib.mpc_sync(self.h))


def row_object_ids(call: int, rows: int, first: int = 0) -> np.ndarray:
    """Object ids (call << 20 | batch << 16 | sub, the C-ABI layout) of rows first .. first + rows
    - 1 of one call, the row number r split as batch = r >> 16, sub = r & 0xFFFF (r < 2^20)."""
    r = np.arange(first, first + rows, dtype=np.uint64)
    assert 0 <= call < (1 << 44) and first + rows <= (1 << 20)
    return (np.uint64(call) << np.uint64(20)) | ((r >> np.uint64(16)) << np.uint64(16)) | (r & np.uint64(0xFFFF))


def segment_row_keys(segments, layer: int, rows_per_image: int) -> np.ndarray:
    """Row keys of one layer of a packed batch: segments = [(request id, images), ...] in packing
    order; the rows of request q's images get the object ids of call 2^43 + q * 64 + layer (a
    range apart from ordinary call ids), numbered from 0 within the request, so that a request
    draws the same truncation bits packed or alone."""
    assert 0 <= layer < 64
    return np.concatenate([row_object_ids((1 << 43) + int(q) * 64 + layer, int(b) * rows_per_image)
                           for q, b in segments])


def to_u64(t) -> np.ndarray:
    """Device int64 tensor -> host numpy uint64 (bit pattern)."""
    return t.detach().cpu().numpy().view(np.uint64)


def from_u64(ctx: Context, a: np.ndarray):
    """Host numpy uint64 -> device int64 tensor (bit pattern)."""
    t = ctx.torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64))
    return t.to(ctx.device)

