"""Benchmark: one secure Z_2^64 GEMM layer per step on GB300, through libmpc3's C-ABI.

Step = the whole hot path on one batch of synthetic input (default n = M = N = K = 8192):
  input sharing of X (M x K) and W (K x N)          Pi_<.>^{l,0}
  Pi_Inner for all M N outputs + Pi_Trunc^13         (offline Gamma, trunc pairs, online products)
  Pi_BIVerify of the layer (batch 0: the M N inner products; batch 1: the truncation pairs, in
  chunks of 2^24 outputs)
  Pi_Rec of the M x N output
Metric: secure ring-MAC/s = M N K / step time (plaintext-equivalent multiply-accumulates of the
secure product, verification included).  Inputs are resident in HBM when timing starts ("value");
"e2e" repeats the step through the same C-ABI with the inputs and the output in pinned host
memory: each step's inputs are uploaded by mpc_h2d_async one step ahead and its output downloaded
by mpc_d2h_async one step behind, on the context's copy stream.

The same step also runs on the other GEMM path (the u64 CUDA-core products when the main path is
the limb-split tensor-core one) on the same layer and inputs, reported under "other_path".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 8192 | --shape MxNxK]
                  [--gemm-path tc|u64] [--other-path-steps S] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("secure Z_2^64 ring-MAC/s incl. verification (limb-INT8 TC vs u64 path); "
          "CNN images/s")
UNIT = "ring-MAC/s"


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The job's time: the maximum of a per-rank time over all ranks (replicas)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n: int, world: int, seconds_per_step: float, shape=None) -> float:
    """Whole-job secure ring-MAC/s: every rank runs one n x n x n (or M x N x K) layer per step."""
    M, N, K = shape if shape else (n, n, n)
    return world * float(M) * N * K / seconds_per_step


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--shape", default=None, help="MxNxK instead of a square n (e.g. 16384x256x4096)")
    ap.add_argument("--other-path-steps", type=int, default=1,
                    help="timed steps of the other GEMM path on the same layer (0: skip)")
    ap.add_argument("--other-path-warmup", type=int, default=1)
    ap.add_argument("--trunc", type=int, default=13)
    ap.add_argument("--gemm-path", choices=["u64", "tc"], default="tc")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default tuning instead of the autotuner's picks")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle timed on the host on a bounded slab of the workload
# ---------------------------------------------------------------------------------------------
def oracle_step(n: int, rows: int, cols: int, t: int, seed: bytes, call: int):
    from oracle import protocols as OP
    from oracle import verify as OV
    from oracle.shares import Session
    from paper_2411_09287_gb300 import workloads
    X, W = workloads.gemm_square(n) if n <= 1024 else workloads.gemm_shape(rows, cols, n, "slab")
    X, W = X[:rows, :n], W[:n, :cols]
    s = Session(seed)
    SX = OP.share_input(s, X, call)
    SW = OP.share_input(s, W, call + 1)
    res = OP.matmul(s, SX, SW, call + 2, trunc_bits=t)
    ok = OV.matmul_verify(s, SX, SW, res, call + 3, t)
    out = OP.reconstruct(s, res.out)
    assert ok and out.shape == (rows, cols)


def _oracle_slab(job):
    oracle_step(*job)
    return True


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """One single-threaded oracle process per host core (spawned, so that it is safe after CUDA
    has been initialised in this process); run() times one slab per core, concurrently."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        self.cores = cores
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})   # inherited by the spawned workers
        try:
            self.pool = mp.get_context("spawn").Pool(cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, n, rows, cols, t, seed, call0) -> float:
        jobs = [(n, rows, cols, t, seed, call0 + 10 * i) for i in range(self.cores)]
        t0 = time.perf_counter()
        assert all(self.pool.map(_oracle_slab, jobs, chunksize=1))
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(n: int, t: int, rows: int = 2, cols: int = 32):
    from paper_2411_09287_gb300 import workloads
    seed = workloads.master_seed("C3-cpu")
    pool = OraclePool(host_cores())
    try:
        pool.run(n, rows, cols, t, seed, 10)                  # warm-up: imports, first slab
        dt = pool.run(n, rows, cols, t, seed, 10 + 10 * pool.cores)
    finally:
        pool.close()
    macs = pool.cores * rows * cols * n
    return {"value": macs / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{pool.cores} x one {rows}x{cols} output slab of the {n}x{n}x{n} layer "
                      f"(K = {n}), one per core at once: share, Pi_Inner + Pi_Trunc^{t}, "
                      f"Pi_BIVerify (both batches), Pi_Rec; {dt:.1f} s wall, numpy single-threaded "
                      f"per process"}


def layer_config(M: int, N: int, K: int, t: int, gemm_path: str, world: int) -> dict:
    """The workload both arms report (identical objects, so that their lines compare)."""
    return {"workload": f"secure GEMM {M}x{N}x{K} (M x N x K) over Z_2^64 (uniform u64 shares) + "
                        f"Pi_Trunc^{t} + Pi_BIVerify (2 batches, trunc batch in chunks of 2^24 "
                        f"outputs) + Pi_Rec",
            "M": M, "N": N, "K": K, "trunc_bits": t, "gemm_path": gemm_path,
            "parallelism": f"replicas x{world}", "l2": "inputs larger than L2"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    M, N, K = parse_shape(args)
    rows, cols = 1, 16
    pool = OraclePool(host_cores())
    try:
        for i in range(warm):
            pool.run(K, rows, cols, args.trunc, b"\x01" * 32, 100 + i * 1000)
        dt = sum(pool.run(K, rows, cols, args.trunc, b"\x02" * 32, 100000 + i * 1000)
                 for i in range(steps)) / steps
    finally:
        pool.close()
    v = pool.cores * rows * cols * K / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": layer_config(M, N, K, args.trunc, args.gemm_path, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": f"per step, {pool.cores} x one {rows}x{cols} output slab "
                                       f"of the layer (K = {K}), one per core at once; the rate "
                                       f"is the slabs' plaintext-equivalent MACs per second"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
# DRAM bytes (read + write) per step of each kernel, summed over its launches, from one ncu
# capture of the n = 1024 layer (E = 2^20 outputs); every one of these kernels streams data in
# proportion to E (operand digit planes, folded vectors, bit words, tables), so the bench scales
# the figure by E / 2^20.  The summaries, with the commands that produced them: profiles/.
NCU_TRAFFIC_E = 2 ** 20
NCU_TRAFFIC = {   # bytes per step at E = 2^20 (profiles/traffic_gr_kernels_n1024.md)
    "k_trunc_s": 0.3965e9,
    "k_limb_gemm": 0.7628e9,
    "k_gr_matmul": 10.066e9,
    "k_gram": 2.165e9,
    "k_gr_mul_rows": None,   # not launched at these sizes (the tensor-core form replaces it)
}
ALU_NOTE = "peak derived: 152 SMs x 64 IMAD/clk x max SM clock; a u64 MAC is 3 IMAD"


def rooflines(phases, steps, peaks, clk, M, N, K, E, gemm_path):
    """Roofline records of the dominant kernels: CUDA-event time of each kernel inside the step
    and the algorithmic u64 multiply-accumulates the library attributes to it.  Tensor kernels
    count the digit products they form (36 f16 digit pairs per u64 MAC for the 8-bit balanced
    digits, 8 where one operand is a bit; 16 e4m3 limbs per bit-times-u64 MAC for the S matrix;
    the library reports the work in 36-pair units), 2 FLOP each, against
    the measured cuBLAS bf16 rate (sustained: they run inside a long step) or twice it for e4m3
    (the nominal fp8 : bf16 ratio).  CUDA-core kernels count 3 IMAD per u64 MAC."""
    bf16 = peaks.get("bf16_tflops_sustained")
    src = "of measured" if bf16 else "of fallback"
    bf16 = bf16 or 1700.0
    sm_max = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    alu = 152 * 64 * sm_max * 1e6 / 1e12   # T IMAD/s
    out = {}

    def rec(name, ops_per_mac, peak, unit, bound, note, work=None):
        ms, _, w = phases.get(name, (0.0, 0, 0.0))
        ms /= steps
        w = (w / steps) if work is None else work
        if not ms or not w:
            return
        ach = ops_per_mac * w / (ms * 1e-3) / 1e12
        tr = NCU_TRAFFIC.get(name)
        out[name] = {"bound": bound, "kernel": name, "achieved": ach, "peak": peak, "unit": unit,
                     "frac": ach / peak, "traffic": tr * E / NCU_TRAFFIC_E if tr else None,
                     "ms_per_step": ms, "u64_macs_per_step": w, "peak_source": src, "note": note}

    rec("k_trunc_s", 2 * 16, 2 * bf16, "TFLOP/s", "tensor",
        "tcgen05 kind::f8f6f4, 16 e4m3 limbs per MAC; peak = 2 x measured bf16 (sustained)")
    if gemm_path == "tc":
        for k, what in (("k_limb_gemm", "limb-split products"), ("k_gr_matmul", "GR-matrix products"),
                        ("k_gram", "Gram sums")):
            rec(k, 2 * 36, bf16, "TFLOP/s", "tensor",
                f"tcgen05 kind::f16 {what}, 36 f16 digit pairs per MAC; peak = measured bf16 (sustained)")
        rec("k_gr_mul_rows", 3, alu, "Tops/s (int32 IMAD)", "alu", ALU_NOTE)
    else:
        rec("gemm", 3, alu, "Tops/s (int32 IMAD)", "alu", "u64 CUDA-core GEMM; " + ALU_NOTE,
            work=5.0 * M * N * K)
    return out


class Layer:
    """One secure GEMM layer per step through the C-ABI on one context: buffers, workspace and the
    step itself (the same call sequence for both GEMM paths)."""

    def __init__(self, mpc, torch, M, N, K, t, seed, device, gemm_path, X, W, Xd, Wd):
        import ctypes as C
        self.mpc, self.torch, self.C = mpc, torch, C
        self.M, self.N, self.K, self.t = M, N, K, t
        self.E = E = M * N
        self.ctx = ctx = mpc.Context(seed, device=device, gemm_path=gemm_path)
        self.X, self.W = X, W
        self.xs, self.wsh = ctx.shares(M * K), ctx.shares(K * N)
        self.zpre, self.zout, self.pq = ctx.shares(E), ctx.shares(E), ctx.empty(12 * E)
        self.out_dev = ctx.empty(E)
        # one workspace for every call of the step
        self.wsb = self.ws_bytes(ctx)
        self.ws = ctx.workspace(self.wsb)
        self.lib, self.h = ctx.lib, ctx.h
        self.call = 1
        self.dev_args = (self.P(Xd), self.P(Wd), 0, self.P(self.out_dev), 0)

    def P(self, tt):
        return self.C.c_void_p(tt.data_ptr())

    def check(self, rc, what):
        if rc != self.mpc.MPC_OK:
            raise self.mpc.MpcError(rc, f"{what}: {self.lib.mpc_last_error(self.h).decode()}")

    def ws_bytes(self, ctx):
        mpc, M, N, K, t = self.mpc, self.M, self.N, self.K, self.t
        return max(ctx.ws_size(mpc.OP_SHARE, max(M * K, K * N)), ctx.ws_size(mpc.OP_MATMUL, M, N, K, t),
                   ctx.ws_size(mpc.OP_VERIFY_MATMUL, M, N, K, t), ctx.ws_size(mpc.OP_RECONSTRUCT, self.E))

    def retune(self, picks):
        """The tuning the autotuner picked, on this layer's context (workspace re-sized)."""
        self.ctx.set_tuning(**picks)
        self.wsb = self.ws_bytes(self.ctx)
        self.ws = None
        self.ws = self.ctx.workspace(self.wsb)

    def tune_step(self, ctx, trace):
        """One step on another context (same seed, fixed call ids) with this layer's buffers and a
        verification trace; returns the host copy of the trace (the autotuner's runs)."""
        wsb = self.ws_bytes(ctx)
        if self.ws.numel() * 8 < wsb + 256:
            self.ws = None
            self.ws = self.ctx.workspace(wsb)
        return self.step(*self.dev_args, ctx=ctx, call=1, trace=trace, wsb=wsb)

    def step(self, x_ptr, w_ptr, on_host, out_ptr, out_host, ctx=None, call=None, trace=None,
             wsb=None):
        lib, P, M, N, K, t = self.lib, self.P, self.M, self.N, self.K, self.t
        h = ctx.h if ctx is not None else self.h
        ws = self.ws
        wsb = self.wsb if wsb is None else wsb
        if call is None:
            c = self.call
            self.call += 8
        else:
            c = call
        self.check(lib.mpc_share_input(h, c, x_ptr, on_host, M * K, P(self.xs), P(ws), wsb), "share X")
        self.check(lib.mpc_share_input(h, c + 1, w_ptr, on_host, K * N, P(self.wsh), P(ws), wsb),
                   "share W")
        self.check(lib.mpc_matmul(h, c + 2, P(self.xs), P(self.wsh), M, N, K, t, P(self.zpre),
                                  P(self.zout), P(self.pq), P(ws), wsb), "matmul")
        self.check(lib.mpc_verify_matmul(h, c + 3, P(self.xs), P(self.wsh), P(self.zpre),
                                         P(self.pq), M, N, K, t, c + 2, -1, -1, P(ws), wsb,
                                         P(trace) if trace is not None else None),
                   "verify")
        self.check(lib.mpc_reconstruct(h, P(self.zout), self.E, out_ptr, out_host, P(ws), wsb),
                   "reconstruct")
        if trace is not None:
            return self.mpc.to_u64(trace).copy()

    def sampled_check(self, nsamples: int = 16):
        """On sampled outputs (a, b): the pre-truncation product reconstructs to (X W)_ab mod 2^64
        (Python integers), and the opened truncated output is (X W)_ab >>_arith t up to Pi_Trunc's
        error (Fig. trunc, Sec. 4.2): with m = x + r, (m >>_a t) - (r >>_a t) = (x >>_a t) + c -
        2^(l-t) w, c in {0, 1} the carry and w in {-1, 0, 1} the wrap of x + r; a wrap has
        probability about |x| / 2^l, common for the uniform 64-bit words of this workload, so the
        check is the residue mod 2^(l-t) and the wraps are counted."""
        mpc, M, N, K, t, E = self.mpc, self.M, self.N, self.K, self.t, self.E
        zp = self.torch.empty(E, dtype=self.torch.int64, device=self.out_dev.device)
        self.check(self.lib.mpc_reconstruct(self.h, self.P(self.zpre), E, self.P(zp), 0,
                                            self.P(self.ws), self.wsb), "reconstruct zpre")
        zp = mpc.to_u64(zp)
        o = mpc.to_u64(self.out_dev)
        g = np.random.default_rng(0)
        wraps = 0
        for _ in range(nsamples):
            a, b = int(g.integers(0, M)), int(g.integers(0, N))
            ref = sum(int(self.X[a, k]) * int(self.W[k, b]) for k in range(K)) % (1 << 64)
            assert int(zp[a * N + b]) == ref, f"secure product differs from X W at ({a}, {b})"
            sref = ref - (1 << 64) if ref >> 63 else ref
            got = int(o[a * N + b])
            got = got - (1 << 64) if got >> 63 else got
            d = (got - (sref >> t)) % (1 << 64)
            assert d % (1 << (64 - t)) in (0, 1), f"truncated output off at ({a}, {b}): {d:#x}"
            wraps += d > 1
        return wraps

    def timed(self, steps, world, dist):
        """`steps` steps on resident inputs, CUDA events on the context's stream; returns ms per
        step and the library's kernel launches per step."""
        torch = self.torch
        stream = torch.cuda.current_stream()
        l0 = self.ctx.launch_count()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            self.step(*self.dev_args)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return ev0.elapsed_time(ev1) / steps, (self.ctx.launch_count() - l0) // steps

    def close(self):
        self.ws = None
        self.ctx.close()


def run_autotune(mpc, torch, L, seed, device, path, M, N, K, t):
    """The autotuner's picks for this layer (cached per device, shape and path): each candidate
    runs one whole step on a fresh context of the same seed and call ids, and must reproduce the
    default's verification transcript."""
    from paper_2411_09287_gb300 import autotune as AT
    key = AT._key(torch.cuda.get_device_name(device), M, N, K, t, path)
    hit = AT.load_cached(key)
    if hit is not None:
        return {**hit, "cached": True}
    trace = L.ctx.zeros(L.ctx.trace_words(mpc.OP_VERIFY_MATMUL, M, N, K, t))

    def make_ctx(tuning):
        return mpc.Context(seed, device=device, gemm_path=path, tuning=tuning or None,
                           stream=L.ctx.stream)

    rec = AT.autotune(make_ctx, lambda ctx: L.tune_step(ctx, trace), AT.search_space(M, N, K))
    AT.store_cached(key, rec)
    return {**rec, "cached": False}


def parse_shape(args):
    if args.shape:
        M, N, K = (int(v) for v in args.shape.lower().split("x"))
    else:
        M = N = K = args.n
    return M, N, K


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    from paper_2411_09287_gb300 import mpc, workloads

    M, N, K = parse_shape(args)
    t = args.trunc
    E = M * N
    name = f"{M}x{N}x{K}"
    seed = workloads.master_seed(f"C3-{M}" if M == N == K else f"C3-{name}")
    X, W = workloads.gemm_square(M) if M == N == K else workloads.gemm_shape(M, N, K)
    main_path = mpc.GEMM_U64 if args.gemm_path == "u64" else mpc.GEMM_LIMB_TC
    Xd, Wd = (torch.from_numpy(a.reshape(-1).view(np.int64)).to(f"cuda:{local}") for a in (X, W))
    L = Layer(mpc, torch, M, N, K, t, seed, local, main_path, X, W, Xd, Wd)
    tuned = None
    if not args.no_autotune:
        tuned = run_autotune(mpc, torch, L, seed, local, main_path, M, N, K, t)
        L.retune(tuned["picks"])
    for _ in range(args.warmup):
        L.step(*L.dev_args)
    torch.cuda.synchronize()
    if args.warmup > 0:   # (with no warm-up step there is no product to check yet)
        L.sampled_check()

    # ---- timed region: inputs resident in HBM ----
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    L.ctx.profile(True)
    ms, launches = L.timed(args.steps, world, dist)
    phases = L.ctx.profile_read()
    L.ctx.profile(False)
    clk = clocks.stop()
    wraps = L.sampled_check()

    # ---- e2e: host inputs (pinned) -> device, output -> pinned host ----
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X.reshape(-1).view(np.int64)).pin_memory()
        Wh = torch.from_numpy(W.reshape(-1).view(np.int64)).pin_memory()
        Oh = torch.empty(E, dtype=torch.int64).pin_memory()
        host_args = (L.P(Xh), L.P(Wh), 1, L.P(Oh), 1)
        L.step(*host_args)
        torch.cuda.synchronize()
        e_steps = max(1, args.steps)
        # pipelined copies: step k + 1's inputs go up on the context's copy stream
        # (mpc_h2d_async) while step k runs, and step k's output comes down on it
        # (mpc_d2h_async) while step k + 1 runs; mpc_h2d_wait orders each step after its
        # upload, and the reuse of an output buffer after its download
        Xu = [L.ctx.empty(M * K) for _ in range(2)]
        Wu = [L.ctx.empty(K * N) for _ in range(2)]
        Od = [L.ctx.empty(E) for _ in range(2)]
        Ohs = [Oh, torch.empty(E, dtype=torch.int64).pin_memory()]

        def upload(k):
            L.ctx.h2d_async(Xu[k % 2], Xh, k % 2)
            L.ctx.h2d_async(Wu[k % 2], Wh, k % 2)

        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        upload(0)
        for k in range(e_steps):
            L.ctx.h2d_wait(k % 2)
            if k + 1 < e_steps:
                upload(k + 1)
            if k >= 2:
                L.ctx.h2d_wait(2 + k % 2)
            L.step(L.P(Xu[k % 2]), L.P(Wu[k % 2]), 0, L.P(Od[k % 2]), 0)
            L.ctx.d2h_async(Ohs[k % 2], Od[k % 2], 2 + k % 2)
        torch.cuda.synchronize()   # the device, copy stream included
        dt = max_over_ranks((time.perf_counter() - t0) / e_steps, world)
        L.sampled_check()
        # the last download equals the last step's output opened again on the device
        od = torch.empty(E, dtype=torch.int64, device=L.out_dev.device)
        L.check(L.lib.mpc_reconstruct(L.h, L.P(L.zout), E, L.P(od), 0, L.P(L.ws), L.wsb),
                "reconstruct e2e output")
        if not torch.equal(od.cpu(), Ohs[(e_steps - 1) % 2]):
            raise SystemExit("e2e: the downloaded output differs from the device-side opening")
        del od
        e2e = {"value": job_value(0, world, dt, (M, N, K)), "unit": UNIT, "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": (M * K + K * N) * 8, "d2h_bytes_per_step": E * 8,
               "steps": e_steps, "copies": "pinned host buffers; each step's inputs uploaded by "
                                           "mpc_h2d_async one step ahead and its output "
                                           "downloaded by mpc_d2h_async one step behind, on the "
                                           "context's copy stream"}
        del Xh, Wh, Oh, Ohs, Xu, Wu, Od

    ms = max_over_ranks(ms, world)
    value = job_value(0, world, ms * 1e-3, (M, N, K))
    wsb = L.wsb
    L.close()
    del L

    # ---- the other GEMM path on the same layer and inputs ----
    other = None
    if args.other_path_steps > 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        o_path = mpc.GEMM_LIMB_TC if main_path == mpc.GEMM_U64 else mpc.GEMM_U64
        O = Layer(mpc, torch, M, N, K, t, seed, local, o_path, X, W, Xd, Wd)
        for _ in range(args.other_path_warmup):
            O.step(*O.dev_args)
        torch.cuda.synchronize()
        oclk = ClockSampler(torch.cuda.current_device())
        oclk.start()
        O.ctx.profile(True)
        oms, olaunch = O.timed(args.other_path_steps, world, dist)
        ophases = O.ctx.profile_read()
        O.ctx.profile(False)
        oc = oclk.stop()
        O.sampled_check()
        oms = max_over_ranks(oms, world)
        oname = "u64" if o_path == mpc.GEMM_U64 else "tc"
        other = {"gemm_path": oname, "value": job_value(0, world, oms * 1e-3, (M, N, K)),
                 "unit": UNIT, "ms_per_step": oms, "steps": args.other_path_steps,
                 "warmup": args.other_path_warmup, "gpu_launches": olaunch, "clocks": oc,
                 "phases_ms": {k: round(v[0] / args.other_path_steps, 3)
                               for k, v in ophases.items() if v[0] > 0},
                 "speedup_of_main_path": oms / ms}
        O.close()
        del O

    # ---- roofline of the dominant kernel ----
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else open(os.devnull) as f:
        try:
            peaks = json.load(f)
        except Exception:
            peaks = {}
    per = {k: v[0] / args.steps for k, v in phases.items()}
    roofs = rooflines(phases, args.steps, peaks, clk, M, N, K, E, args.gemm_path)
    roof = max(roofs.values(), key=lambda r: r["ms_per_step"]) if roofs else None
    if other is not None:
        opk = "u64" if other["gemm_path"] == "u64" else "tc"
        other["rooflines"] = rooflines(ophases, args.other_path_steps, peaks, oc, M, N, K, E, opk)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": layer_config(M, N, K, t, args.gemm_path, world),
        "working_set_gib": round((wsb + 8 * 6 * (M * K + K * N + 4 * E)) / 2**30, 1),
        "roofline": roof,
        "rooflines": roofs,
        "phases_ms": {k: round(v, 3) for k, v in per.items() if v > 0},
        "gpu_launches": launches,
        "clocks": clk,
        "trunc_wraps_sampled": wraps,
    }
    if tuned is not None:
        line["autotune"] = tuned
    if other is not None:
        line["other_path"] = other
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(K, t)
        except Exception as ex:   # reported, never silently replaced
            line["cpu_baseline"] = {"error": str(ex)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
