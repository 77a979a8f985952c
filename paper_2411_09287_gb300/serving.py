"""Continuous-batching server for secure inference on one GPU (config C5 pattern).

Requests (a batch of 1..256 inputs each) arrive over time.  A dispatcher admits arrived requests
while the images in flight fit a device-memory budget, packs the admitted requests of one model
into a single secure forward pass (up to `max_batch` images), and hands it to the first idle
worker.  Each worker owns a libmpc3 context on its own CUDA stream, so packed batches of
different workers run concurrently on the device (the library's calls release the GIL).  Logits
are split back per request; latency is arrival -> opened logits.

The weights are shared once per worker and stay resident.  Each request's truncation bits are
keyed by (request, layer, row of the request), so a request's logits are bit-identical whether it
runs alone or packed with others (the other random values differ, but an opened value depends on
them only through the truncation carry).
"""
from __future__ import annotations

import contextlib
import hashlib
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import mpc as M
from . import secure_cnn as SC
from . import secure_mlp as SM


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    x: np.ndarray             # (b, ...) float inputs
    logits: np.ndarray = None
    done: float = None
    error: BaseException = None   # set when the packed pass that carried the request failed


class Model:
    """A fixed-point model with a secure forward pass and its float64 reference."""

    def __init__(self, kind: str, k: int = 13):
        self.kind, self.k = kind, k
        if kind == "mlp":
            self.w = SM.mlp_weights([784, 128, 128, 10], "C2-weights")
            self.in_shape = (784,)
        elif kind == "neta":
            self.p = SC.net_a_params("C4-netA-weights")
            self.in_shape = (1, 28, 28)
        elif kind == "netb":
            self.p = SC.net_b_params("C4-netB-weights")
            self.in_shape = (3, 32, 32)
        else:
            raise ValueError(kind)

    def share(self, ctx, call_base):
        """P0 shares the weights once; the sharings stay resident for every later pass."""
        if self.kind == "mlp":
            return SM.share_weights(ctx, self.w, self.k, call_base)
        if self.kind == "netb":
            return SC.share_params_b(ctx, self.p, self.k, call_base)
        return SC.share_params(ctx, self.p, self.k, call_base)

    def secure(self, ctx, x, call_base, shared=None, segments=None):
        """Opened logits (float64) of one secure forward pass over the packed inputs x.
        segments = [(request id, images), ...]: truncation bits keyed per request, so that each
        request gets exactly the logits it would get alone."""
        if self.kind == "mlp":
            return SM.secure_forward(ctx, x, self.w, self.k, call_base, shared_weights=shared,
                                     segments=segments)
        if self.kind == "netb":
            return SC.net_b_secure(ctx, x, self.p, self.k, call_base, shared=shared,
                                   segments=segments)
        return SC.net_a_secure(ctx, x, self.p, self.k, call_base, shared=shared, segments=segments)

    def fp64(self, x):
        q = lambda a: SM.quantized(a, self.k)
        if self.kind == "mlp":
            return SM.fp64_forward(q(x), [q(w) for w in self.w])
        ref = SC.net_b_fp64 if self.kind == "netb" else SC.net_a_fp64
        return ref(q(x), {n: q(w) for n, w in self.p.items()})

    def bytes_per_image(self, ctx, b: int) -> float:
        """Peak workspace of one packed batch of b images (the largest single call) / b."""
        if self.kind == "mlp":
            sizes = [784, 128, 128, 10]
            ws = []
            for i in range(3):
                ws.append(ctx.ws_size(M.OP_MATMUL, b, sizes[i + 1], sizes[i], self.k))
                ws.append(ctx.ws_size(M.OP_VERIFY_MATMUL, b, sizes[i + 1], sizes[i], self.k))
                if i < 2:
                    ws.append(ctx.ws_size(M.OP_RELU, b * sizes[i + 1]))
        elif self.kind == "neta":
            ws = [ctx.ws_size(M.OP_VERIFY_MATMUL, b * 576, 16, 25, self.k),
                  ctx.ws_size(M.OP_VERIFY_MATMUL, b * 64, 16, 400, self.k),
                  ctx.ws_size(M.OP_MAXPOOL2, SC.pool_planes(SC.NL_CHUNK, 24, 24, b * 16), 24, 24),
                  ctx.ws_size(M.OP_RELU, min(SC.NL_CHUNK, b * 16 * 12 * 12))]
        else:
            ws = [ctx.ws_size(M.OP_VERIFY_MATMUL, b * 1024, 64, 576, self.k),
                  ctx.ws_size(M.OP_MAXPOOL2, SC.pool_planes(SC.NL_CHUNK, 32, 32, b * 64), 32, 32),
                  ctx.ws_size(M.OP_RELU, min(SC.NL_CHUNK, b * 64 * 32 * 32))]
        return max(ws) / b


class _Worker(threading.Thread):
    def __init__(self, wid, server, ctx=None, stream=None):
        super().__init__(daemon=True)
        self.wid, self.server = wid, server
        if ctx is None:   # the same three parties (one seed) on every worker, own call ids
            import torch
            stream = torch.cuda.Stream()
            ctx = M.Context(server.seed, gemm_path=server.gemm_path, stream=stream)
        self.ctx, self.stream = ctx, stream
        self.inbox = queue.Queue()
        self.calls = 1 + wid * (1 << 36)          # disjoint call-id spaces per worker
        self.busy = threading.Event()

    def _on_stream(self):
        if self.stream is None:
            return contextlib.nullcontext()
        import torch
        return torch.cuda.stream(self.stream)

    def run(self):
        shared = None
        while True:
            job = self.inbox.get()
            if job is None:
                return
            reqs = job
            n = sum(r.x.shape[0] for r in reqs)
            try:
                x = np.concatenate([r.x for r in reqs], axis=0)
                with self._on_stream():
                    if shared is None:   # weights shared once, resident for the worker's life
                        shared = self.server.model.share(self.ctx, self.calls)
                        self.calls += 1 << 16
                    logits = self.server.model.secure(self.ctx, x, self.calls, shared,
                                                      [(r.rid, r.x.shape[0]) for r in reqs])
                t = time.perf_counter() - self.server.t0
                off = 0
                for r in reqs:
                    b = r.x.shape[0]
                    r.logits = logits[off: off + b]
                    r.done = t
                    off += b
            except BaseException as ex:   # an aborted protocol, a CUDA error, an OOM ...
                t = time.perf_counter() - self.server.t0
                for r in reqs:
                    r.error, r.done = ex, t
                with self.server.lock:
                    self.server.errors.append(ex)
            finally:
                self.calls += 1 << 16
                with self.server.lock:
                    self.server.in_flight -= n
                self.busy.clear()
                self.server.wake.set()


def pack_requests(pending: list, limit: int):
    """Admit the longest prefix of the arrival-ordered `pending` whose images fit `limit`; the
    admitted requests leave `pending`.  Returns (requests, images)."""
    pack, n = [], 0
    while pending and n + pending[0].x.shape[0] <= limit:
        r = pending.pop(0)
        pack.append(r)
        n += r.x.shape[0]
    return pack, n


def check_admissible(requests, max_batch: int, max_in_flight: int):
    """Every request must fit one packed pass and the memory budget on its own; otherwise it could
    never be admitted and the server would wait for it forever."""
    cap = min(max_batch, max_in_flight)
    for r in requests:
        if r.x.shape[0] > cap:
            raise ValueError(f"request {r.rid} has {r.x.shape[0]} images; at most {cap} fit "
                             f"(max_batch {max_batch}, memory budget {max_in_flight} images)")


class Server:
    SEED = hashlib.sha256(b"mpc3-serving-parties").digest()

    def __init__(self, model: Model, n_workers: int = 2, max_batch: int = 256,
                 mem_budget_bytes: float = 64e9, gemm_path: int = M.GEMM_LIMB_TC,
                 make_context=None, seed: bytes = None):
        """make_context(worker id) -> (context, CUDA stream or None) replaces the default context
        per worker (one on a new stream, keyed by `seed`: every worker runs the same three
        parties, in its own range of call ids)."""
        self.model, self.max_batch, self.gemm_path = model, max_batch, gemm_path
        self.seed = seed or self.SEED
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.in_flight = 0
        self.errors = []
        self.workers = [_Worker(i, self, *(make_context(i) if make_context else (None, None)))
                        for i in range(n_workers)]
        per = model.bytes_per_image(self.workers[0].ctx, max_batch)
        self.max_in_flight = max(1, int(mem_budget_bytes // max(per, 1.0)))
        self.t0 = None

    def serve(self, requests):
        """Run all requests (sorted by arrival); returns them with logits and completion times.
        If a packed pass fails, no further requests are admitted, the workers are shut down and
        the first failure is raised (the failed requests carry it in .error)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        check_admissible(reqs, self.max_batch, self.max_in_flight)
        for w in self.workers:
            w.start()
        self.t0 = time.perf_counter()
        pending = []
        i = 0
        while (i < len(reqs) or pending) and not self.errors:
            now = time.perf_counter() - self.t0
            while i < len(reqs) and reqs[i].arrival <= now:
                pending.append(reqs[i])
                i += 1
            idle = [w for w in self.workers if not w.busy.is_set()]
            if pending and idle:
                with self.lock:
                    room = self.max_in_flight - self.in_flight
                pack, n = pack_requests(pending, min(self.max_batch, room))
                if pack:
                    with self.lock:
                        self.in_flight += n
                    w = idle[0]
                    w.busy.set()
                    w.inbox.put(pack)
                    continue
            # sleep until the next arrival or a worker finishes
            nxt = reqs[i].arrival - now if i < len(reqs) else 0.05
            self.wake.wait(timeout=max(0.0005, min(nxt, 0.05)))
            self.wake.clear()
        for w in self.workers:
            while w.busy.is_set():
                time.sleep(0.001)
            w.inbox.put(None)
        for w in self.workers:
            w.join()
        if self.errors:
            raise RuntimeError(f"a packed secure pass failed: {self.errors[0]!r}") from self.errors[0]
        return reqs

    def close(self):
        """Release the workers' contexts and their workspaces (after serve)."""
        for w in self.workers:
            ctx = getattr(w, "ctx", None)
            if ctx is None:
                continue
            if hasattr(ctx, "_ws"):
                ctx._ws = None
            if hasattr(ctx, "close"):
                ctx.close()
        try:
            import torch
            if torch.cuda.is_available():
                torch.cuda.empty_cache()
        except ImportError:
            pass

    @staticmethod
    def stats(reqs):
        lat = np.array([r.done - r.arrival for r in reqs])
        imgs = sum(r.x.shape[0] for r in reqs)
        span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
        return {"requests": len(reqs), "images": int(imgs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "images_per_s": imgs / span}


def poisson_requests(model: Model, n: int, rate: float, max_b: int, seed: str):
    from .workloads import rng
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += g.exponential(1.0 / rate)
        b = int(g.integers(1, max_b + 1))
        out.append(Request(i, t, g.uniform(0.0, 1.0, (b,) + model.in_shape)))
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="secure-inference serving run")
    ap.add_argument("--model", choices=["mlp", "neta", "netb"], default="mlp")
    ap.add_argument("--rate", type=float, nargs="+", default=[200.0])
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--max-b", type=int, default=256)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--workers", type=int, default=2)
    a = ap.parse_args()
    model = Model(a.model)
    for rate in a.rate:
        reqs = poisson_requests(model, a.requests, rate, a.max_b, f"C5-{a.model}-{rate}")
        srv = Server(model, a.workers, a.max_batch)
        try:
            out = srv.serve(reqs)
        finally:
            srv.close()   # each rate's workers hold workspaces sized for the largest call
        st = Server.stats(out)
        err = max(float(np.max(np.abs(r.logits - model.fp64(r.x)))) for r in out)
        st.update({"model": a.model, "rate": rate, "max_abs_err_vs_fp64": err})
        print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
