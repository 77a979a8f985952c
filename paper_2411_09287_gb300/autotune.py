"""Autotuner for libmpc3's launch shapes and verification layout (mpc_set_tuning).

The knobs change no protocol value: every setting must give the same verification transcript
(every revealed challenge, every round's <h(0)>, <h(p2)>, every opened Delta).  The tuner runs
the caller's step -- one whole layer: sharing, Pi_Inner + Pi_Trunc, Pi_BIVerify, Pi_Rec -- once
per candidate on the real shape, times it with CUDA events on the context's stream, compares
its transcript with the first (default) run's, and keeps the fastest.  Knob groups are searched
one after another, each with the others at their best so far (coordinate descent):

  gr        the GR-matrix product kernel: producers (register loads / TMA / A in tensor
            memory) and drain warps (8 / 16)
  split     fewest 32-deep K chunks per split-K slice of the thin tensor-core products
  gram      split-K slices of the tensor-core Gram sums
  rowsplit  L', the row split of the blocked truncation batch's folded-vector products
  foldbatch the longest folded vectors whose folds share one launch

Picks are cached per (device, shape, GEMM path) in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np


def _row_split_candidates(E: int):
    """0 (the library's own choice) and odd multiples of 128 around sqrt(E)/2 .. 2 sqrt(E)."""
    out = [0]
    a0 = max(1, math.ceil(math.sqrt(max(E, 1)) / 128))
    for a in (a0 // 2, a0 * 2):
        a |= 1
        if a >= 1 and 128 * a <= E:
            out.append(128 * a)
    return out


def search_space(M: int, N: int, K: int):
    E = M * N
    return [
        ("gr", [dict(gr_producers=1, gr_drain_warps=8), dict(gr_producers=2, gr_drain_warps=8),
                dict(gr_producers=1, gr_drain_warps=16), dict(gr_producers=3)]),
        ("split", [dict(gemm_split_min=v) for v in (8, 4, 16)]),
        ("gram", [dict(gram_split=v) for v in (76, 152, 38)]),
        ("rowsplit", [dict(row_split=v) for v in _row_split_candidates(E)]),
        ("foldbatch", [dict(fold_batch_max=v) for v in (65536, 16384, 262144)]),
    ]


def cache_path() -> str:
    return os.environ.get("MPC3_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                                       "autotune.json"))


def _key(device_name: str, M, N, K, t, path) -> str:
    return f"{device_name}|{M}x{N}x{K}|t{t}|path{path}"


def load_cached(key: str):
    try:
        with open(cache_path()) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def store_cached(key: str, rec) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        data = {}
        if os.path.exists(p):
            with open(p) as f:
                data = json.load(f)
        data[key] = rec
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, p)
    except (OSError, ValueError):
        pass


class TranscriptMismatch(RuntimeError):
    """A tuning candidate changed a protocol value: a bug in the kernel it selects."""


def cuda_clock(ctx, fn):
    """(milliseconds, result) of fn() between CUDA events on the context's stream."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    out = fn()
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def autotune(make_ctx, run_step, space, reps: int = 1, budget_s: float = 120.0, log=None,
             clock=cuda_clock):
    """Coordinate descent over `space` (list of (group, [tuning dicts])).
    make_ctx(tuning) returns a fresh context with the given tuning and always the same seed, so
    that every candidate runs the same protocol instance; run_step(ctx) runs one layer step on it
    (always the same call ids) and returns the host copy of its verification transcript; the
    step is timed here with CUDA events on the context's stream.  Returns {"picks": tuning dict,
    "trials": [...], "seconds": s}.  Raises TranscriptMismatch when a candidate's transcript
    differs from the default's."""
    best = {}
    ref = None
    trials = []
    t_start = time.perf_counter()

    def timed(cand):
        nonlocal ref
        ms, tr = [], None
        for _ in range(reps):
            ctx = make_ctx({**best, **cand})
            t, tr = clock(ctx, lambda: run_step(ctx))
            ms.append(t)
            ctx.close()
        if ref is None:
            ref = tr
        elif not np.array_equal(tr, ref):
            raise TranscriptMismatch(f"tuning {dict(**best, **cand)} changed the transcript")
        return float(np.median(ms))

    warm = make_ctx({})   # first-use costs (kernel attributes, tensor-map setup) out of the timings
    run_step(warm)
    warm.close()
    for group, cands in space:
        scores = []
        for cand in cands:
            if time.perf_counter() - t_start > budget_s and scores:
                break
            ms = timed(cand)
            trials.append({"group": group, "tuning": cand, "ms": round(ms, 3)})
            scores.append((ms, cand))
            if log:
                log(f"autotune {group} {cand}: {ms:.2f} ms")
        best.update(min(scores, key=lambda x: x[0])[1])
    return {"picks": best, "trials": trials, "seconds": round(time.perf_counter() - t_start, 2)}
